"""Pins of the PM oracle (the long-range part of the PPPM / TreePM methods
whose short-range part the paper's arbitrary-shape force loop evaluates,
Section 4.2).

- The direct k-space sum (the definition) against closed forms: near a mass
  in a periodic box the long-range field is the isolated split force plus
  the neutralising background's (4 pi / 3) (m / L^3) r; the lattice images
  add nothing at first order (cubic symmetry). For the Gaussian split the
  isolated long-range force is m [erf(r / 2 r_s) - r / (r_s sqrt pi)
  e^(-r^2 / 4 r_s^2)] / r^2; for S2 it is R(r, a), the paper's profile.
- The mesh method against the direct sum, and its invariances (a shift by
  whole cells, linearity in the masses).
- PP (the exact short-range pair force) plus PM against the Ewald sum of
  the full Newton force, as the paper measures its PP accuracy.
"""

import math

import numpy as np
import pytest

import gen
from oracle import pm

L = 1.0


def _closed_form_gauss(r, rs):
    return (math.erf(r / (2 * rs)) - r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs))) / r ** 2


@pytest.mark.parametrize("r_over_rs", [0.5, 1.0, 2.0, 4.0])
def test_kspace_gauss_is_the_long_range_force(r_over_rs):
    rs = 0.02
    src = np.array([[0.5, 0.5, 0.5]])
    u = np.array([0.48, -0.6, 0.64])
    r = r_over_rs * rs
    t = src + r * u[None, :]
    a, _ = pm.kspace_forces(src, np.array([1.0]), L, "gauss", rs, 32, targets=t)
    want = -_closed_form_gauss(r, rs) * u + (4 * math.pi / 3) * r * u
    assert np.allclose(a[0], want, rtol=1e-4, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("r_over_a", [0.3, 0.7, 1.0, 2.0])
def test_kspace_s2_is_the_s2_profile(orc, r_over_a):
    a_ = 0.05
    src = np.array([[0.25, 0.5, 0.75]])
    u = np.array([0.0, 0.6, -0.8])
    r = r_over_a * a_
    t = src + r * u[None, :]
    a, _ = pm.kspace_forces(src, np.array([1.0]), L, "s2", a_, 64, targets=t)
    want = -orc.s2_profile(r, a_) * u + (4 * math.pi / 3) * r * u
    assert np.allclose(a[0], want, rtol=2e-4, atol=1e-12 * np.abs(want).max())


def test_s2_form_factor_series_is_continuous():
    # the series below q = 0.1 and the closed form above meet, and the series
    # agrees with the closed form where both are accurate
    q = np.array([0.1 * (1 - 1e-10), 0.1 * (1 + 1e-10)])
    v = pm.split_factor(2 * q, "s2", 1.0)
    assert abs(v[0] - v[1]) < 1e-9
    for qq in (0.05, 0.08):
        series = pm.split_factor(np.array([2 * qq]), "s2", 1.0)[0]
        direct = (12 * (2 - 2 * math.cos(qq) - qq * math.sin(qq)) / qq ** 4) ** 2
        assert series == pytest.approx(direct, rel=1e-8)


@pytest.mark.parametrize("split,scale_cells", [("gauss", 1.25), ("s2", 4.0)])
def test_mesh_matches_the_kspace_sum(split, scale_cells):
    N = 64
    rng = np.random.default_rng(21)
    x = rng.random((24, 3))
    m = rng.uniform(0.5, 1.5, 24)
    scale = scale_cells * L / N
    am, pm_ = pm.mesh_forces(x, m, L, N, split, scale)
    ak, pk = pm.kspace_forces(x, m, L, split, scale, N // 2 - 1)
    err = np.linalg.norm(am - ak, axis=1) / np.linalg.norm(ak, axis=1)
    assert np.median(err) < 3e-3 and err.max() < 2e-2
    # potentials agree up to the mesh's own error
    assert np.max(np.abs(pm_ - pk)) < 2e-2 * np.max(np.abs(pk))


def test_mesh_shift_by_cells_and_mass_linearity():
    N = 32
    x, m = gen.clustered_box(500, 22, nclump=5, sigma=0.05)
    a0, p0 = pm.mesh_forces(x, m, L, N, "gauss", 1.25 / N)
    a1, p1 = pm.mesh_forces((x + np.array([3, -5, 7]) / N) % 1.0, m, L, N, "gauss", 1.25 / N)
    assert np.allclose(a0, a1, rtol=1e-9, atol=1e-9 * np.abs(a0).max())
    a2, p2 = pm.mesh_forces(x, 2.5 * m, L, N, "gauss", 1.25 / N)
    assert np.allclose(a2, 2.5 * a0, rtol=1e-12, atol=1e-12 * np.abs(a0).max())


def _pp_exact(x, m, rs, rcut, L=1.0):
    """Short-range Gaussian-split pair force, minimum image, within rcut."""
    acc = np.zeros_like(x)
    for i in range(len(x)):
        d = x - x[i]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=1)
        s = (r > 0) & (r < rcut)
        rr = r[s]
        g = (np.array([math.erfc(v / (2 * rs)) for v in rr]) +
             rr / (rs * math.sqrt(math.pi)) * np.exp(-rr ** 2 / (4 * rs ** 2))) / rr ** 3
        acc[i] = np.sum((m[s] * g)[:, None] * d[s], axis=0)
    return acc


def test_pp_plus_pm_is_the_ewald_sum():
    # the Gaussian split is an Ewald split: PP (real space, cut at 4.5 r_s
    # where erfc is below 1e-6 of the force) plus the k-space sum is the
    # periodic Newton force; PP plus the mesh agrees with it to the mesh
    # accuracy (the paper's PP + PM check, here with random particles)
    N = 64
    rs = 1.25 / N
    rng = np.random.default_rng(23)
    x = rng.random((200, 3))
    m = rng.uniform(0.5, 1.5, 200)
    pp = _pp_exact(x, m, rs, 4.5 * rs * 1.6)
    ak, _ = pm.kspace_forces(x, m, L, "gauss", rs, 40)
    am, _ = pm.mesh_forces(x, m, L, N, "gauss", rs)
    ewald, total = pp + ak, pp + am
    err = np.linalg.norm(total - ewald, axis=1) / np.linalg.norm(ewald, axis=1)
    assert np.median(err) < 2e-3 and np.percentile(err, 99) < 2e-2
