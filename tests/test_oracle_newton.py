"""Pins for the FP64 Newton oracle (Eq. 1), each against something other than
the oracle's own formula: hand-derived two-body and lattice values, momentum
conservation, and the analytic fields of a uniform sphere and a Plummer model.
"""

import math

import numpy as np
import pytest

import gen


def test_two_body_hand_values(orc):
    # j at (3, 4, 0) with unit mass acting on i at the origin: r = 5.
    xi = np.array([[0.0, 0.0, 0.0]])
    xj = np.array([[3.0, 4.0, 0.0]])
    a, p = orc.newton(xi, xj, [1.0], eps=0.0)
    assert np.allclose(a[0], [3 / 125, 4 / 125, 0.0], rtol=0, atol=1e-16)
    assert p[0] == pytest.approx(-0.2, rel=1e-15)
    # eps^2 = 11 gives r^2 + eps^2 = 36: a = d / 216, phi = -1/6.
    a, p = orc.newton(xi, xj, [1.0], eps=math.sqrt(11.0))
    assert np.allclose(a[0], [3 / 216, 4 / 216, 0.0], rtol=1e-14, atol=0)
    assert p[0] == pytest.approx(-1 / 6, rel=1e-14)
    # mass scales the result linearly and the sign points from i to j
    a, _ = orc.newton(xj, xi, [2.0], eps=0.0)
    assert np.allclose(a[0], [-6 / 125, -8 / 125, 0.0], rtol=1e-14, atol=0)


def test_all_pairs_leaves_self_out(orc):
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([2.0, 1.0])
    a, p = orc.newton_allpairs(x, m, eps=0.0)   # eps = 0 would be NaN with a self term
    assert np.allclose(a, [[3 / 125, 4 / 125, 0], [-6 / 125, -8 / 125, 0]], rtol=1e-14, atol=0)
    assert np.allclose(p, [-1 / 5, -2 / 5], rtol=1e-14)


def test_cube_corner_lattice(orc):
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    m = np.ones(8)
    # centre: every component cancels by symmetry; phi = -8 / sqrt(3)
    a, p = orc.newton(np.zeros((1, 3)), corners, m, eps=0.0)
    assert np.all(np.abs(a) < 1e-15)
    assert p[0] == pytest.approx(-8 / math.sqrt(3), rel=1e-15)
    # corner (1,1,1) from the other seven: 3 edges (r=2), 3 face diagonals
    # (r=2 sqrt 2), 1 body diagonal (r=2 sqrt 3), worked out by hand
    k = 7
    assert np.all(corners[k] == [1, 1, 1])
    others = np.delete(corners, k, axis=0)
    a, p = orc.newton(corners[k:k + 1], others, np.ones(7), eps=0.0)
    ax = -(1 / 4 + 1 / (4 * math.sqrt(2)) + 1 / (12 * math.sqrt(3)))
    assert np.allclose(a[0], [ax, ax, ax], rtol=1e-14, atol=0)
    assert p[0] == pytest.approx(-(1.5 + 1.5 / math.sqrt(2) + 0.5 / math.sqrt(3)), rel=1e-14)
    # skip[] leaves exactly one j out
    a2, p2 = orc.newton(corners[k:k + 1], corners, m, eps=0.0, skip=[k])
    assert np.allclose(a2, a, rtol=1e-15) and p2[0] == pytest.approx(p[0], rel=1e-15)


def test_momentum_conservation(orc):
    x, _ = gen.plummer(512, 11)
    m = np.exp(np.random.default_rng(5).uniform(-3, 0, 512))
    a, _ = orc.newton_allpairs(x, m, eps=1 / 64)
    net = np.abs((m[:, None] * a).sum(axis=0)).max()
    scale = (m * np.linalg.norm(a, axis=1)).sum()
    assert net / scale <= 1e-13


def test_uniform_sphere_field(orc):
    nj = 100_000
    xs, ms = gen.uniform_sphere(nj, 21, radius=1.0, total_mass=1.0)
    probes_r = np.array([0.3, 0.6, 1.5, 3.0])
    probes = np.stack([probes_r / math.sqrt(3)] * 3, axis=1)  # along the diagonal
    a, p = orc.newton(probes, xs, ms, eps=1e-4)
    for r, ai, pi, pos in zip(probes_r, a, p, probes):
        if r < 1.0:
            phi_exact = -(3 - r * r) / 2
            a_exact = -pos          # -M r / R^3, radial
        else:
            phi_exact = -1 / r
            a_exact = -pos / r**3
        tol = 5 / math.sqrt(nj)
        assert abs(pi - phi_exact) <= tol * abs(phi_exact)
        # inside, the near neighbours' graininess dominates the force noise
        atol = 3 * tol if r > 1.0 else 0.1
        assert np.linalg.norm(ai - a_exact) <= atol * np.linalg.norm(a_exact)


def _fibonacci_sphere(k):
    t = np.arange(k) + 0.5
    mu = 1 - 2 * t / k
    ph = math.pi * (1 + 5 ** 0.5) * t
    st = np.sqrt(1 - mu * mu)
    return np.stack([st * np.cos(ph), st * np.sin(ph), mu], axis=1)


def test_plummer_sample_shell_theorem(orc):
    """Averaged over a sphere of radius r, the potential of any point set is
    -sum_j m_j / max(r, r_j) and the inward radial force is M(<r) / r^2
    (Newton's shell theorem), computed here from the sample's radii alone."""
    n = 1 << 16
    x, m = gen.plummer(n, 31)
    rj = np.linalg.norm(x, axis=1)
    dirs = _fibonacci_sphere(4000)
    for r in (0.5, 1.0, 2.0):
        a, p = orc.newton(r * dirs, x, m, eps=0.0)
        phi_shell = -(m / np.maximum(r, rj)).sum()
        ar_shell = m[rj < r].sum() / r**2
        assert p.mean() == pytest.approx(phi_shell, rel=2e-5)
        assert -(a * dirs).sum(axis=1).mean() == pytest.approx(ar_shell, rel=5e-3)
        # and the drawn model follows the analytic Plummer field
        assert p.mean() == pytest.approx(-1 / math.sqrt(r * r + 1), rel=5e-3)
        assert ar_shell == pytest.approx(r / (r * r + 1) ** 1.5, rel=3e-2)


def test_subset_matches_full(orc):
    x, m = gen.plummer(600, 41)
    a, p = orc.newton_allpairs(x, m, eps=1 / 64)
    idx = np.array([0, 17, 599])
    a2, p2 = orc.newton_subset(x, m, 1 / 64, idx)
    assert np.allclose(a2, a[idx], rtol=1e-15, atol=0) and np.allclose(p2, p[idx], rtol=1e-15)


def test_groups_raw_list_sum(orc):
    # one group with a listed self pair: zero force from it and -m/eps potential
    xj = np.array([[0.0, 0, 0], [3.0, 4, 0]])
    mj = np.array([2.0, 1.0])
    xi = np.array([[0.0, 0, 0]])
    eps = math.sqrt(11.0)
    a, p = orc.newton_groups([0, 1], [0, 2], [0, 1], xi, xj, mj, eps)
    assert np.allclose(a[0], [3 / 216, 4 / 216, 0], rtol=1e-14, atol=1e-18)
    assert p[0] == pytest.approx(-2 / eps - 1 / 6, rel=1e-14)
    # two groups, repeated and reordered indices: each group sums its own list
    x, mm = gen.plummer(64, 51)
    i_off = [0, 3, 5]
    j_off = [0, 4, 7]
    jl = [5, 9, 9, 60, 1, 2, 3]
    xi = x[[10, 11, 12, 40, 41]]
    a, p = orc.newton_groups(i_off, j_off, jl, xi, x, mm, 0.01)
    for g in range(2):
        for i in range(i_off[g], i_off[g + 1]):
            lst = jl[j_off[g]:j_off[g + 1]]
            ai, pi = orc.newton(xi[i:i + 1], x[lst], mm[lst], 0.01)
            assert np.allclose(a[i], ai[0], rtol=1e-14) and p[i] == pytest.approx(pi[0], rel=1e-14)
