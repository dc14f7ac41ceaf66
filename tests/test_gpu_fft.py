"""The hand-written FFT solve of the particle mesh (power-of-two meshes from
8 to 512) against the PM oracle (the same method in FP64, numpy's FFT) and
against the cuFFT solve of the same mesh on the GPU.

Tolerance as in the PM tests: per particle |a - a_ref| against the RMS
acceleration, median <= 1e-5 and max <= 1e-4 (both GPU solves are FP32).
Covered: every power of two from 8 to 512 (512 against cuFFT only), the
Gaussian and S2 splits, a box of side 3, the fallback to cuFFT for a mesh
that is not a power of two, and the mode's errors.
"""

import numpy as np
import pytest

import gen
from oracle import pm as opm
from pgtest import need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def rms(a):
    return float(np.sqrt(np.mean(np.sum(np.asarray(a).reshape(len(a), -1) ** 2, axis=1))))


def assert_mesh_parity(a, ao, what):
    err = np.linalg.norm((a - ao).reshape(len(a), -1), axis=1) / rms(ao)
    med, mx = float(np.median(err)), float(err.max())
    assert med <= 1e-5 and mx <= 1e-4, f"{what}: median {med:.2e} max {mx:.2e} of the RMS"


def both_solves(pg, x, m, L, N, split, scale):
    with pg.Context(0) as c:
        c.set_periodic(L)
        c.set_pm(N, pg.PG_SPLIT_GAUSS if split == "gauss" else pg.PG_SPLIT_S2, scale)
        a1, p1 = c.pm_forces(x, m)
        k1 = c.pm_fft()
        c.set_pm_fft(pg.PG_FFT_LIBRARY)
        a2, p2 = c.pm_forces(x, m)
        k2 = c.pm_fft()
    return a1, p1, k1, a2, p2, k2


@pytest.mark.parametrize("N,split,scale_cells,L", [(8, "gauss", 1.25, 1.0), (16, "gauss", 1.25, 1.0),
                                                   (32, "s2", 4.0, 1.0), (64, "gauss", 1.5, 3.0),
                                                   (128, "gauss", 1.25, 1.0), (256, "s2", 4.0, 1.0)])
def test_hand_fft_against_oracle_and_cufft(pg, N, split, scale_cells, L):
    x, m = gen.clustered_box(20000, 7200 + N, nclump=30, sigma=0.03)
    x = x * L
    m = m * np.random.default_rng(N).uniform(0.5, 2.0, len(m))
    scale = scale_cells * L / N
    a1, p1, k1, a2, p2, k2 = both_solves(pg, x, m, L, N, split, scale)
    assert k1 == 1 and k2 == 2
    ao, po = opm.mesh_forces(x, m, L, N, split, scale)
    assert_mesh_parity(a1, ao, f"hand-written a, N={N}")
    assert_mesh_parity(p1[:, None], po[:, None], f"hand-written phi, N={N}")
    assert_mesh_parity(a1, a2, f"hand-written against cuFFT a, N={N}")
    assert_mesh_parity(p1[:, None], p2[:, None], f"hand-written against cuFFT phi, N={N}")


def test_hand_fft_512_against_cufft(pg):
    x, m = gen.clustered_box(300000, 7301, nclump=60, sigma=0.02)
    a1, p1, k1, a2, p2, k2 = both_solves(pg, x, m, 1.0, 512, "gauss", 1.25 / 512)
    assert k1 == 1 and k2 == 2
    assert_mesh_parity(a1, a2, "a, N=512")
    assert_mesh_parity(p1[:, None], p2[:, None], "phi, N=512")


def test_other_sizes_use_cufft(pg):
    x, m = gen.clustered_box(5000, 7302, nclump=10, sigma=0.03)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        assert c.pm_fft() == 0
        c.set_pm(48, pg.PG_SPLIT_GAUSS, 1.5 / 48)
        c.pm_forces(x, m)
        assert c.pm_fft() == 2
        c.set_pm(32, pg.PG_SPLIT_GAUSS, 1.5 / 32)
        c.pm_forces(x, m)
        assert c.pm_fft() == 1
        with pytest.raises(pg.PGError) as e:
            c.set_pm_fft(5)
        assert e.value.code == pg.PG_EINVAL
