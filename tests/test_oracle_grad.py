"""Pins for the oracle's gradients of L = sum_i w_i . a_i (Newton and table).

Independent checks: L recomputed from scratch with plain numpy pair loops on
tiny sets and differenced; translation invariance (sum_k dL/dx_k = 0); degree-1
homogeneity in the masses (sum_k m_k dL/dm_k = L); linearity in the knot
values (sum_b v_b dL/dv_b = L); and agreement of the incremental central
differences with the analytic gradient.
"""

import numpy as np
import pytest

import gen


def _L_numpy(x, m, w, kern):
    """L = sum_i sum_{j != i} m_j K(r_ij^2) w_i . (x_j - x_i), plain loops."""
    n = len(x)
    L = 0.0
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d = x[j] - x[i]
            L += m[j] * kern(float(d @ d)) * float(w[i] @ d)
    return L


def _newton_kern(eps):
    return lambda r2: (r2 + eps * eps) ** -1.5


def _table_kern(orc, E, F, r_cut, v):
    G0, G1 = orc.table_from_values(E, F, v)
    return lambda r2: orc.table_eval(E, F, r_cut, G0, G1, r2)


def _small_set(n, seed):
    x, m = gen.plummer(n, seed)
    m = m * np.exp(np.random.default_rng(seed).uniform(-1, 1, n))
    w = gen.unit_vectors(n, seed + 1)
    return x, m, w


def test_newton_gradient_against_brute_force_L(orc):
    x, m, w = _small_set(9, 101)
    eps = 0.2
    dx, dm, L = orc.grad_newton(x, m, w, eps)
    kern = _newton_kern(eps)
    assert L == pytest.approx(_L_numpy(x, m, w, kern), rel=1e-13)
    h = 1e-5
    for k in range(9):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (_L_numpy(xp, m, w, kern) - _L_numpy(xm, m, w, kern)) / (2 * h)
            assert dx[k, c] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (_L_numpy(x, mp, w, kern) - _L_numpy(x, mm, w, kern)) / (2 * h)
        assert dm[k] == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_table_gradient_against_brute_force_L(orc):
    x, m, w = _small_set(8, 202)
    E, F, r_cut = 3, 5, 2.5
    par = [0.8, 0.3]       # r_s, eps of the Gaussian-split shape
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    dx, dm, L = orc.grad_table(x, m, w, E, F, r_cut, v)
    kern = _table_kern(orc, E, F, r_cut, v)
    assert L == pytest.approx(_L_numpy(x, m, w, kern), rel=1e-6)
    dv = orc.grad_table_v(x, m, w, E, F, r_cut, v)
    # L is linear in v: probe a few knots by full recomputation
    for b in np.nonzero(dv)[0][:6]:
        vp, vm = v.copy(), v.copy()
        hb = 1e-2 * max(abs(float(v[b])), 1e-3)
        vp[b] += hb
        vm[b] -= hb
        hb_eff = (float(vp[b]) - float(vm[b])) / 2
        fd = (_L_numpy(x, m, w, _table_kern(orc, E, F, r_cut, vp)) -
              _L_numpy(x, m, w, _table_kern(orc, E, F, r_cut, vm))) / (2 * hb_eff)
        assert dv[b] == pytest.approx(fd, rel=1e-4, abs=1e-9)
    # positions: away from knots the interpolant is linear in s, so a short
    # central difference agrees unless a pair changes bin
    h = 1e-7
    for k in range(8):
        for c in range(3):
            val, kinked = orc.fd_table(x, m, w, E, F, r_cut, v, k, c, h=h)
            if kinked:
                continue
            assert dx[k, c] == pytest.approx(val, rel=1e-5, abs=1e-9)


def test_invariants_newton(orc):
    x, m, w = _small_set(400, 303)
    dx, dm, L = orc.grad_newton(x, m, w, 1 / 64)
    assert np.abs(dx.sum(axis=0)).max() <= 1e-11 * np.abs(dx).sum()
    assert (m * dm).sum() == pytest.approx(L, rel=1e-11)


def test_invariants_table(orc):
    x, m, w = _small_set(400, 404)
    E, F, r_cut = 3, 5, 0.6
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
    dx, dm, L = orc.grad_table(x, m, w, E, F, r_cut, v)
    assert np.abs(dx.sum(axis=0)).max() <= 1e-11 * np.abs(dx).sum()
    assert (m * dm).sum() == pytest.approx(L, rel=1e-11)
    dv = orc.grad_table_v(x, m, w, E, F, r_cut, v)
    assert (v.astype(np.float64) * dv).sum() == pytest.approx(L, rel=1e-11)


def test_incremental_fd_agrees(orc):
    x, m, w = _small_set(300, 505)
    eps = 1 / 64
    dx, dm, _ = orc.grad_newton(x, m, w, eps)
    for k in (0, 123, 299):
        for c in range(3):
            fd = orc.fd_newton(x, m, w, eps, k, c, h=1e-6)
            assert fd == pytest.approx(dx[k, c], rel=1e-7, abs=1e-12)
        assert orc.fd_newton(x, m, w, eps, k, 3, h=1e-6) == pytest.approx(dm[k], rel=1e-9)
    idx = np.array([5, 77])
    gx, gm = orc.grad_newton_at(x, m, w, eps, idx)
    assert np.allclose(gx, dx[idx], rtol=1e-14) and np.allclose(gm, dm[idx], rtol=1e-14)
    E, F, r_cut = 3, 5, 0.6
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
    dv = orc.grad_table_v(x, m, w, E, F, r_cut, v)
    probes = np.nonzero(dv)[0][::7]
    fdv = orc.fd_table_v(x, m, w, E, F, r_cut, v, probes, h=1e-6)
    assert np.allclose(fdv, dv[probes], rtol=1e-7, atol=1e-12)
    tx, tm, _ = orc.grad_table(x, m, w, E, F, r_cut, v)
    gx, gm = orc.grad_table_at(x, m, w, E, F, r_cut, v, idx)
    assert np.allclose(gx, tx[idx], rtol=1e-14) and np.allclose(gm, tm[idx], rtol=1e-14)
