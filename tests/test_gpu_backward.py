"""Backward pass of L = sum_i w_i . a_i (hand-written kernel behind
torch.autograd) against the oracle's analytic FP64 gradients and its
incremental central differences (h = 1e-6): small sets in full for Newton
and the tabulated force, and the 65536-particle Plummer set on 64 sampled
coordinates and 64 knots, relative error <= 1e-4 norm-wise."""

import numpy as np
import pytest

import gen
from pgtest import need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def grads(pg, torch, x, m, w, eps=None, table=None):
    from paper_1203_4037_gb300 import autograd as AG
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    mt = torch.tensor(m, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda")
    if table is None:
        a = AG.newton_force(xt, mt, eps)
        vt = None
    else:
        v, r_cut, E, F = table
        vt = torch.tensor(v, device="cuda", requires_grad=True)
        a = AG.table_force(xt, mt, vt, r_cut, E, F)
    L = (a * wt).sum()
    L.backward()
    out = [xt.grad.cpu().numpy(), mt.grad.cpu().numpy(), float(L.item())]
    out.append(vt.grad.cpu().numpy() if vt is not None else None)
    return out


def normrel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_newton_small_full(pg, torch, orc):
    x, m = gen.plummer(700, 11)
    m = m * np.exp(np.random.default_rng(1).uniform(-1, 1, len(m)))
    w = gen.unit_vectors(700, 12)
    dx, dm, L, _ = grads(pg, torch, x, m, w, eps=1 / 64)
    ox, om, oL = orc.grad_newton(x, m, w, 1 / 64)
    assert L == pytest.approx(oL, rel=1e-5)
    assert normrel(dx, ox) <= 1e-5 and normrel(dm, om) <= 1e-5
    assert np.abs(dx.sum(axis=0)).max() <= 1e-5 * np.abs(dx).sum()


def test_newton_diagonal_subtiles(pg, torch, orc):
    # The Newton kernel takes the j records in the i-particles' tile order
    # and tests for the own pair only in the j sub-tiles that overlap the
    # thread's i-tile. A Morton-ordered set (20011 particles: a ragged last
    # tile) at eps = 1/64, sampled against the oracle's analytic gradient
    n = 20011
    x, m = gen.plummer(n, 7411)
    m = m * np.exp(np.random.default_rng(7412).uniform(-1, 1, n))
    w = gen.unit_vectors(n, 7413)
    dx, dm, _, _ = grads(pg, torch, x, m, w, eps=1 / 64)
    idx = gen.sample_indices(n, 256, 7414)
    ox, om = orc.grad_newton_at(x, m, w, 1 / 64, idx)
    assert normrel(dx[idx], ox) <= 1e-5 and normrel(dm[idx], om) <= 1e-5


def test_newton_eps0_full(pg, torch, orc):
    # eps = 0 tests every sub-tile (a coincident pair would have r^2 = 0): a
    # jittered 14^3 lattice (no two particles closer than a fifth of the
    # spacing; 2744 = 5 tiles of 512 and a ragged one) in full
    rng = np.random.default_rng(7415)
    g = np.stack(np.meshgrid(*[np.arange(14)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g + rng.uniform(-0.4, 0.4, g.shape)) / 14.0
    m = rng.uniform(0.5, 1.5, len(x)) / len(x)
    w = gen.unit_vectors(len(x), 7416)
    dx, dm, L, _ = grads(pg, torch, x, m, w, eps=0.0)
    ox, om, oL = orc.grad_newton(x, m, w, 0.0)
    assert L == pytest.approx(oL, rel=1e-5)
    assert normrel(dx, ox) <= 1e-5 and normrel(dm, om) <= 1e-5


def test_table_small_full(pg, torch, orc):
    # a compact set: with fewer i-particles than a few tiles the FP32 offsets
    # are taken from centres of tiles that span the whole set
    rng = np.random.default_rng(13)
    x = rng.random((1500, 3)) * 0.3
    m = rng.uniform(0.5, 1.5, 1500) / 1500
    w = gen.unit_vectors(1500, 14)
    E, F, r_cut = 3, 5, 0.1
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
    dx, dm, L, dv = grads(pg, torch, x, m, w, table=(v, r_cut, E, F))
    ox, om, oL = orc.grad_table(x, m, w, E, F, r_cut, v)
    odv = orc.grad_table_v(x, m, w, E, F, r_cut, v)
    assert L == pytest.approx(oL, rel=1e-4)
    assert normrel(dx, ox) <= 1e-4 and normrel(dm, om) <= 1e-4
    assert normrel(dv, odv) <= 1e-4


def test_plummer_65536_against_finite_differences(pg, torch, orc):
    n = 65536
    x, m = gen.plummer(n, gen.CONFIG_SEEDS[5])
    w = gen.unit_vectors(n, gen.CONFIG_SEEDS[5] + 1)
    rng = np.random.default_rng(5)
    ks = rng.choice(n, 64, replace=False)
    comps = rng.integers(0, 3, 64)
    # Newton, eps = 1/64
    dx, dm, _, _ = grads(pg, torch, x, m, w, eps=1 / 64)
    fd = np.array([orc.fd_newton(x, m, w, 1 / 64, k, c, h=1e-6) for k, c in zip(ks, comps)])
    assert normrel(dx[ks, comps], fd) <= 1e-4
    fdm = np.array([orc.fd_newton(x, m, w, 1 / 64, k, 3, h=1e-6) for k in ks])
    assert normrel(dm[ks], fdm) <= 1e-4
    ax, am = orc.grad_newton_at(x, m, w, 1 / 64, ks)
    assert normrel(dx[ks], ax) <= 1e-4 and normrel(dm[ks], am) <= 1e-4
    # table, r_cut = 0.1, 256 knots (E = 3, F = 5)
    E, F, r_cut = 3, 5, 0.1
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
    dx, dm, _, dv = grads(pg, torch, x, m, w, table=(v, r_cut, E, F))
    pool = rng.choice(n, 512, replace=False)
    vals, want = [], []
    for k in pool:
        c = int(rng.integers(0, 3))
        val, kinked = orc.fd_table(x, m, w, E, F, r_cut, v, k, c, h=1e-6)
        if kinked:
            continue
        vals.append(dx[k, c])
        want.append(val)
        if len(vals) == 64:
            break
    assert len(vals) == 64
    assert normrel(vals, want) <= 1e-4
    odv = orc.grad_table_v(x, m, w, E, F, r_cut, v)
    bins = np.nonzero(odv)[0]
    probe = rng.choice(bins, min(64, len(bins)), replace=False)
    fdv = orc.fd_table_v(x, m, w, E, F, r_cut, v, probe, h=1e-6)
    assert normrel(dv[probe], fdv) <= 1e-4
