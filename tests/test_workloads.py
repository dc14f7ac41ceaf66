"""The synthetic inputs: the King (1966) models the paper's tree runs use
(Section 5.1, W0 = 9) against their published structure, and the sampled
sets against their own profiles."""

import numpy as np
import pytest

import gen


@pytest.mark.parametrize("W0,c", [(6.0, 1.25), (7.0, 1.53), (9.0, 2.12)])
def test_king_concentration(W0, c):
    # the concentration log10(r_t / r0) of King's models
    xi, W, frac = gen.king_profile(W0)
    assert np.log10(xi[-1]) == pytest.approx(c, abs=0.01)
    assert W[0] == pytest.approx(W0) and W[-1] == pytest.approx(0.0, abs=1e-8)
    assert np.all(np.diff(frac) >= 0) and frac[-1] == 1.0


def test_king_core_is_isothermal_sphere_like():
    # near the centre the density is flat: W = W0 - 1.5 xi^2 to second order
    xi, W, _ = gen.king_profile(9.0)
    small = (xi > 0) & (xi < 0.05)
    assert np.allclose(W[small], 9.0 - 1.5 * xi[small] ** 2, atol=1e-5)


def test_king_sample_follows_the_mass_profile():
    x, m = gen.king(200000, 31)
    xi, _, frac = gen.king_profile(9.0)
    r = np.sort(np.linalg.norm(x, axis=1))
    emp = np.arange(1, len(r) + 1) / len(r)
    model = np.interp(r, xi, frac)
    assert np.max(np.abs(emp - model)) < 0.01          # Kolmogorov-Smirnov distance
    assert r[-1] <= xi[-1] and m.sum() == pytest.approx(1.0)
    # isotropic: the mean direction vanishes
    assert np.linalg.norm((x / r.max()).mean(axis=0)) < 0.02
