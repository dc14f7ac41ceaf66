"""Pins for the oracle's tabulated-force side (Section 3.4): the worked bit
example of Table 4, the index against the paper's bit recipe done with numpy
bit views, the knot walk of the table builder, exact reproduction of shapes
linear in r^2, the S2 profile's continuity, the Section 4.2 accuracy run, the
Gaussian-split shape against a quadrature of the Gaussian cloud, and the
Newton-shaped table against the Newton oracle.
"""

import json
import math
import os

import numpy as np
import pytest

import gen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bits(s):
    return np.asarray(s, dtype=np.float32).view(np.uint32).astype(np.int64)


def _paper_index(s, E, F):
    """Section 3.4.1: shift the FP32 pattern right by 23-F and mask E+F bits."""
    return (_bits(s) >> (23 - F)) & ((1 << (E + F)) - 1)


def test_table4_worked_example(orc):
    g = json.load(open(os.path.join(GOLD, "table4_E4F6.json")))
    E, F = g["E"], g["F"]
    smax = orc.s_max(E, F)
    assert smax == 130048.0
    assert smax == pytest.approx(g["s_max_printed"], rel=5e-5)
    assert orc.table_size(E, F) * 8 == g["table_bytes_printed"]
    r_cut = 0.37
    sc2 = orc.scale2(E, F, r_cut)
    for row in g["rows"]:
        r = row["r_over_rcut"] * r_cut
        s = r * r * sc2 + 2.0
        assert s == pytest.approx(row["s_printed"], rel=5e-5)
        b = format(int(_bits(s)), "032b")
        assert b[1:9] == row["exponent_bits"]
        assert b[9:] == row["fraction_bits"]
        assert orc.bin_index(E, F, min(s, smax)) == row["index"]
        assert _paper_index(s, E, F) == row["index"]


@pytest.mark.parametrize("E,F", [(4, 6), (4, 5), (4, 8), (3, 5), (2, 2), (5, 3), (0, 4), (4, 0)])
def test_index_matches_bit_recipe(orc, E, F):
    rng = np.random.default_rng(E * 100 + F)
    smax = orc.s_max(E, F)
    # random FP32 values of s across [2, s_max] plus every knot and its neighbours
    s = np.exp(rng.uniform(math.log(2.0), math.log(smax), 4000)).astype(np.float32)
    n = orc.table_size(E, F)
    knots = (0x40000000 + np.arange(n, dtype=np.int64) * (1 << (23 - F))).astype(np.uint32).view(np.float32)
    s = np.concatenate([s, knots, np.nextafter(knots, np.float32(np.inf))])
    s = s[(s >= 2) & (s <= smax)]
    got = np.array([orc.bin_index(E, F, float(v)) for v in s])
    assert np.array_equal(got, _paper_index(s, E, F))


@pytest.mark.parametrize("E,F", [(4, 6), (3, 5), (4, 8)])
def test_knots_are_the_builder_tick_walk(orc, E, F):
    # the builder starts at the FP32 pattern of 2.0 and adds 2^(23-F) per knot
    n = orc.table_size(E, F)
    walk = (0x40000000 + np.arange(n, dtype=np.int64) * (1 << (23 - F))).astype(np.uint32).view(np.float32)
    got = np.array([orc.knot(E, F, k) for k in range(n)])
    assert np.array_equal(got, walk.astype(np.float64))
    assert got[-1] == orc.s_max(E, F)


def test_spacing_laws(orc):
    E, F = 5, 6
    smax = orc.s_max(E, F)
    nF = 1 << F

    def r_of(k):
        return math.sqrt((orc.knot(E, F, k) - 2.0) / (smax - 2.0))

    # log spacing across exponents: r ratio tends to sqrt 2 for large bE
    for bF in (0, 17, 63):
        ratios = [r_of((bE + 1) * nF + bF) / r_of(bE * nF + bF) for bE in range(4, 30)]
        assert abs(ratios[-1] - math.sqrt(2)) < 1e-4
        assert abs(ratios[-1] - math.sqrt(2)) < abs(ratios[0] - math.sqrt(2))
    # linear spacing inside an octave: the interval approximation of Section 3.4.1
    bE = 25
    for bF in (8, 30, 62):
        dr = r_of(bE * nF + bF + 1) - r_of(bE * nF + bF)
        approx = (1 / math.sqrt(nF + bF)) * math.sqrt(2.0 ** (bE + 1) / 2.0 ** (F + 2) / (smax - 2.0))
        assert dr == pytest.approx(approx, rel=2e-2)


def test_linear_in_r2_shape_is_exact(orc):
    E, F, r_cut = 4, 6, 0.25
    alpha, beta = 3.0, -17.0
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_LINEAR, [alpha, beta])
    rng = np.random.default_rng(3)
    r = rng.uniform(0, r_cut * 0.999, 2000)
    for rr in r:
        g = orc.table_eval(E, F, r_cut, G0, G1, rr * rr)
        assert g == pytest.approx(alpha + beta * rr * rr, rel=2e-6, abs=2e-6)


def test_table_hits_closed_form_at_knots_and_zero_beyond(orc):
    E, F, r_cut = 4, 8, 4.5 / 256
    par = [1 / 256, 1 / 256 / 16]
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    n = orc.table_size(E, F)
    sc2 = orc.scale2(E, F, r_cut)
    for k in range(0, n - 1, 37):
        rk2 = (orc.knot(E, F, k) - 2.0) / sc2
        want = np.float32(orc.shape(orc.SHAPE_GAUSS_SPLIT, par, math.sqrt(rk2)))
        assert orc.table_eval(E, F, r_cut, G0, G1, rk2) == pytest.approx(float(want), rel=1e-6)
    # the last knot is the cutoff: zero at and beyond r_cut
    assert G0[-1] == 0 and G1[-1] == 0
    for r in (r_cut, 1.01 * r_cut, 5 * r_cut):
        assert orc.table_eval(E, F, r_cut, G0, G1, r * r) == 0.0
    # just inside the cutoff the last bin reaches the closed form's left limit
    r = r_cut * (1 - 1e-7)
    g_in = orc.table_eval(E, F, r_cut, G0, G1, r * r)
    assert g_in == pytest.approx(orc.shape(orc.SHAPE_GAUSS_SPLIT, par, r_cut), rel=1e-5)
    # the interpolant is continuous at interior knots up to FP32 rounding
    for k in range(1, n - 1, 53):
        sk = orc.knot(E, F, k)
        left = float(G0[k - 1]) + (sk - orc.knot(E, F, k - 1)) * float(G1[k - 1])
        assert left == pytest.approx(float(G0[k]), rel=1e-6)


def test_s2_profile_continuity(orc):
    a = 0.7
    # R = 1 / r^2 at and beyond r = a (xi = 2)
    for r in (a, 1.3 * a, 4 * a):
        assert orc.s2_profile(r, a) == pytest.approx(1 / r**2, rel=1e-14)
    # value and slope continuous at xi = 2 and value continuous at xi = 1
    for r0 in (a, a / 2):
        h = 1e-7 * a
        lo, hi = orc.s2_profile(r0 - h, a), orc.s2_profile(r0 + h, a)
        assert lo == pytest.approx(hi, rel=1e-6)
    h = 1e-5 * a
    slope_in = (orc.s2_profile(a - h, a) - orc.s2_profile(a - 2 * h, a)) / h
    slope_out = -2 / a**3
    assert slope_in == pytest.approx(slope_out, rel=1e-4)
    # small r: R grows linearly, R / r -> 448 / (35 a^3)
    assert orc.s2_profile(1e-9 * a, a) / (1e-9 * a) == pytest.approx(448 / 35 / a**3, rel=1e-8)


def test_section_4_2_accuracy_run(orc):
    """S2 PP shape, eps = 3.125e-3, r_cut = 4.6875e-2, E = 4, F = 5, unit masses,
    4K pairs log-uniform in (5e-3, 1) r_cut: the PP (table) + PM (closed form)
    force stays within 1e-3 of R(r, eps)."""
    eps, r_cut, E, F = 3.125e-3, 4.6875e-2, 4, 5
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_S2PP, [eps, r_cut])
    d = gen.log_pairs(4096, 77) * r_cut
    worst = 0.0
    for v in d:
        r = float(np.linalg.norm(v))
        f_pp = orc.table_eval(E, F, r_cut, G0, G1, r * r) * r
        total = f_pp + orc.s2_profile(r, r_cut)
        exact = orc.s2_profile(r, eps)
        worst = max(worst, abs(total - exact) / exact)
    assert worst < 1e-3


def test_gauss_split_against_gaussian_cloud(orc):
    """Short-range shape = Newton minus the force of a Gaussian cloud of unit
    mass, density proportional to exp(-r^2 / 4 r_s^2); the cloud's enclosed
    mass comes from quadrature, not from erf."""
    from scipy import integrate

    rs = 1 / 256
    norm = (4 * math.pi * rs * rs) ** 1.5

    def enclosed(r):
        val, _ = integrate.quad(lambda u: 4 * math.pi * u * u * math.exp(-u * u / (4 * rs * rs)), 0, r,
                                epsabs=0, epsrel=1e-13, limit=200)
        return val / norm

    for r in (0.3 * rs, rs, 2.5 * rs, 4.5 * rs, 9 * rs):
        g = orc.shape(orc.SHAPE_GAUSS_SPLIT, [rs, 0.0], r)
        assert g == pytest.approx((1 - enclosed(r)) / r**3, rel=1e-9)
    # softening multiplies by (r^2/(r^2+eps^2))^{3/2}; r_s -> infinity gives Newton
    eps = rs / 16
    r = 2 * rs
    g0 = orc.shape(orc.SHAPE_GAUSS_SPLIT, [rs, 0.0], r)
    assert orc.shape(orc.SHAPE_GAUSS_SPLIT, [rs, eps], r) == pytest.approx(
        g0 * (r * r / (r * r + eps * eps)) ** 1.5, rel=1e-13)
    assert orc.shape(orc.SHAPE_GAUSS_SPLIT, [1e12, eps], r) == pytest.approx(
        orc.shape(orc.SHAPE_NEWTON, [eps], r), rel=1e-10)


def test_newton_table_matches_newton_oracle(orc):
    rng = np.random.default_rng(9)
    x = rng.random((300, 3))
    m = rng.uniform(0.5, 1.5, 300) / 300
    eps, r_cut, E, F = 0.05, 2.0, 4, 8
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_NEWTON, [eps])
    skip = np.arange(300)
    at, _ = orc.table_forces(x, x, m, E, F, r_cut, G0, G1, skip=skip)
    an, _ = orc.newton_allpairs(x, m, eps)
    rel = np.linalg.norm(at - an, axis=1) / np.linalg.norm(an, axis=1)
    assert np.max(rel) < 2e-5


def test_closed_form_cutoff_and_periodic_image(orc):
    # i near 0.01, j near 0.99 in a unit periodic box: the image at -0.01 acts
    rs = 1 / 256
    r_cut, eps = 4.5 * rs, rs / 16
    par = [rs, eps]
    xi = np.array([[0.01, 0.5, 0.5]])
    xj = np.array([[0.99, 0.5, 0.5]])
    a, _ = orc.shape_forces(xi, xj, [1.0], orc.SHAPE_GAUSS_SPLIT, par, r_cut, box=1.0)
    g = orc.shape(orc.SHAPE_GAUSS_SPLIT, par, 0.02)
    assert 0.02 > r_cut  # beyond the cutoff: nothing
    assert np.all(a == 0)
    xj = np.array([[0.995, 0.5, 0.5]])
    a, _, absum = orc.shape_forces(xi, xj, [1.0], orc.SHAPE_GAUSS_SPLIT, par, r_cut, box=1.0,
                                   with_absum=True)
    g = orc.shape(orc.SHAPE_GAUSS_SPLIT, par, 0.015)
    assert a[0, 0] == pytest.approx(-0.015 * g, rel=1e-12)
    assert absum[0] == pytest.approx(0.015 * g, rel=1e-12)
    # the table path takes the same image
    E, F = 4, 8
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    at, _ = orc.table_forces(xi, xj, [1.0], E, F, r_cut, G0, G1, box=1.0)
    assert at[0, 0] == pytest.approx(a[0, 0], rel=1e-4)


def test_cutoff_ambiguity_record(orc):
    rs = 1 / 256
    r_cut, eps = 4.5 * rs, rs / 16
    E, F = 4, 8
    G0, G1 = orc.table_build(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [rs, eps])
    xi = np.zeros((1, 3))
    xj = np.array([[r_cut * (1 + 1e-8), 0, 0], [0.5 * r_cut, 0, 0]])
    a, amb = orc.table_forces(xi, xj, [1.0, 1.0], E, F, r_cut, G0, G1, window=1e-6)
    assert amb[0] > 0
    a, amb = orc.table_forces(xi, xj, [1.0, 1.0], E, F, r_cut, G0, G1, window=0.0)
    assert amb[0] == 0
