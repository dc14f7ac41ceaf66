"""Pins of the oracle's extensions beyond Eq. (1) and (2) as the paper runs
them:

- Per-i softening. The i-particle structure of Section 3.1 carries eps^2 per
  i, and the Newton kernel of Section 3.3 adds the i-particle's eps^2.
  Pinned by hand-derived two-body values with unequal softenings and by the
  all-equal case.
- Table-mode potential. A second table of the same layout for a potential
  shape psi(r); the paper's tabulated kernel stores accelerations only.
  Pinned by:
  - exact reproduction of a psi linear in r^2;
  - the knot values;
  - zero at and beyond r_cut;
  - the tabulated Newton potential against the Newton oracle's potential.
"""

import numpy as np
import pytest


def test_per_i_softening_two_body_hand_values(orc):
    # |d| = 3. Particle 0 has eps = 4, so r_hat = 5; particle 1 has eps = 0,
    # so r_hat = 3. Masses 2 and 5.
    x = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    m = np.array([2.0, 5.0])
    a, phi = orc.newton_epsi(x, [4.0, 0.0], x, m, skip=np.arange(2))
    assert a[0] == pytest.approx([0.12, 0.0, 0.0], abs=1e-15)          # 5 * 3 / 125
    assert phi[0] == pytest.approx(-1.0, abs=1e-15)                    # -5 / 5
    assert a[1] == pytest.approx([-2.0 / 9.0, 0.0, 0.0], abs=1e-15)    # 2 * (-3) / 27
    assert phi[1] == pytest.approx(-2.0 / 3.0, abs=1e-15)              # -2 / 3


def test_per_i_softening_three_bodies_use_own_eps_only(orc):
    # probe at the origin with eps = 1.5, sources at distance 2 and sqrt(8)
    # whose own softenings must not matter: r_hat^2 = 4 + 2.25 and 8 + 2.25
    xi = np.zeros((1, 3))
    xj = np.array([[2.0, 0.0, 0.0], [0.0, 2.0, 2.0]])
    mj = np.array([1.0, 3.0])
    a, phi = orc.newton_epsi(xi, [1.5], xj, mj)
    k0 = 1.0 / 6.25 ** 1.5
    k1 = 3.0 / 10.25 ** 1.5
    assert a[0] == pytest.approx([2.0 * k0, 2.0 * k1, 2.0 * k1], rel=1e-14)
    assert phi[0] == pytest.approx(-(1.0 / 2.5 + 3.0 / 10.25 ** 0.5), rel=1e-14)


def test_per_i_softening_all_equal_is_the_global_case(orc):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((200, 3))
    m = rng.uniform(0.5, 1.5, 200) / 200
    a1, p1 = orc.newton_epsi(x, np.full(200, 0.07), x, m, skip=np.arange(200))
    a2, p2 = orc.newton(x, x, m, 0.07, skip=np.arange(200))
    assert np.allclose(a1, a2, rtol=1e-14, atol=0)
    assert np.allclose(p1, p2, rtol=1e-14, atol=0)


def test_per_i_softening_rejects_negative(orc):
    with pytest.raises(ValueError):
        orc.newton_epsi(np.zeros((1, 3)), [-1.0], np.ones((1, 3)), [1.0])


def _pairs_at(r, n_i=1):
    """i-particles at the origin and one j per distance in r along a diagonal."""
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    return np.zeros((n_i, 3)), np.outer(r, u)


@pytest.mark.parametrize("E,F", [(3, 5), (4, 8)])
def test_potential_table_linear_in_r2_is_exact(orc, E, F):
    # psi = alpha + beta r^2 is linear in s, so the interpolant is exact
    # (up to the FP32 rounding of the stored values) below r_cut, and the
    # T5 reading makes it zero at and beyond r_cut
    r_cut, alpha, beta = 0.3, -2.5, 7.0
    P0, P1 = orc.table_build(E, F, r_cut, orc.SHAPE_LINEAR, [alpha, beta])
    rng = np.random.default_rng(E + F)
    r = np.concatenate([rng.uniform(0.0, r_cut * 0.999, 400), [r_cut * 1.001, 1.0, 5.0]])
    xi, xj = _pairs_at(r)
    mj = rng.uniform(0.5, 2.0, len(r))
    for k in range(len(r)):
        phi, _ = orc.table_potential(xi, xj[k:k + 1], mj[k:k + 1], E, F, r_cut, P0, P1)
        want = mj[k] * (alpha + beta * r[k] ** 2) if r[k] < r_cut else 0.0
        assert phi[0] == pytest.approx(want, rel=2e-6, abs=1e-300)


def test_potential_table_knot_values(orc):
    # a pair placed exactly at knot k (s = s_k) reads the stored knot value
    E, F, r_cut = 3, 4, 1.0
    eps = 0.05
    v = orc.table_values(E, F, r_cut, orc.SHAPE_NEWTON_POT, [eps])
    P0, P1 = orc.table_from_values(E, F, v)
    n = orc.table_size(E, F)
    sc2 = (orc.s_max(E, F) - 2.0) / r_cut ** 2
    for k in (0, 1, 5, n // 2, n - 2):
        r = np.sqrt((orc.knot(E, F, k) - 2.0) / sc2)
        xi, xj = _pairs_at(np.array([r]))
        phi, _ = orc.table_potential(xi, xj, [1.0], E, F, r_cut, P0, P1)
        assert phi[0] == pytest.approx(float(v[k]), rel=1e-12, abs=1e-12)
    # at and beyond the cutoff: nothing
    xi, xj = _pairs_at(np.array([r_cut, 2.0 * r_cut]))
    phi, _ = orc.table_potential(xi, xj, [1.0, 1.0], E, F, r_cut, P0, P1)
    assert phi[0] == 0.0


def test_tabulated_newton_potential_matches_newton_oracle(orc):
    # psi = -(r^2 + eps^2)^(-1/2) tabulated with r_cut beyond every pair: the
    # table-mode potential equals Eq. (1)'s potential within the table error
    rng = np.random.default_rng(21)
    x = rng.random((300, 3))
    m = rng.uniform(0.5, 1.5, 300) / 300
    eps, r_cut, E, F = 0.05, 2.0, 4, 8
    P0, P1 = orc.table_build(E, F, r_cut, orc.SHAPE_NEWTON_POT, [eps])
    skip = np.arange(300)
    pt, _ = orc.table_potential(x, x, m, E, F, r_cut, P0, P1, skip=skip)
    _, pn = orc.newton_allpairs(x, m, eps)
    rel = np.abs(pt - pn) / np.abs(pn)
    assert np.max(rel) < 2e-5
    # and the skip leaves the own pair out: without it the sum gains m_i psi(0)
    pa, _ = orc.table_potential(x, x, m, E, F, r_cut, P0, P1)
    assert np.allclose(pa - pt, m * float(orc.table_values(E, F, r_cut, orc.SHAPE_NEWTON_POT,
                                                               [eps])[0]), rtol=1e-9)
