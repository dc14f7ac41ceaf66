"""Parity of the periodic cutoff path (cell list of side >= r_cut, 27
neighbour cells with minimum-image shifts, tabulated Gaussian-split force)
with the oracle's brute-force minimum-image sums over all j: a small
clustered box in full, boundary-crossing pairs, and the 2^21-particle
clustered box on a 4096-particle sample."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda

pytestmark = pytest.mark.gpu

RS = 1 / 256


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def run_cells(pg, x, m, v, r_cut, E, F, box=1.0):
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_table_values(v, r_cut, E, F)
        c.set_self(True)
        c.set_periodic(box)
        a, p = c.forces(x, x, m)
        info = c.info()
        return a, p, info


def check_sample(orc, x, m, a, idx, v, r_cut, E, F, par):
    G0, G1 = orc.table_from_values(E, F, v)
    ao, amb = orc.table_forces(x[idx], x, m, E, F, r_cut, G0, G1, box=1.0, skip=idx, window=1e-6)
    norm = np.linalg.norm(ao, axis=1)
    ok = norm > 0
    assert np.all(np.linalg.norm(a[idx][~ok], axis=1) == 0)
    rel = np.maximum(np.linalg.norm(a[idx] - ao, axis=1) - amb, 0)[ok] / norm[ok]
    assert_parity(rel, what="a vs table semantics")
    # the table's own error is at most 1e-3 of each pair term
    ac, ambc, absum = orc.shape_forces(x[idx], x, m, orc.SHAPE_GAUSS_SPLIT, par, r_cut, box=1.0,
                                       skip=idx, window=1e-6, with_absum=True)
    err = np.maximum(np.linalg.norm(a[idx] - ac, axis=1) - ambc, 0)
    assert np.all(err <= 1e-3 * absum)


def test_small_clustered_box(pg, orc):
    n = 1 << 15
    x, m = gen.clustered_box(n, 123, nclump=20, sigma=0.01)
    r_cut, E, F = 0.05, 4, 8
    par = [r_cut / 4.5, r_cut / 72]
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    a, p, info = run_cells(pg, x, m, v, r_cut, E, F)
    assert np.all(p == 0)
    assert info["pairs"] > 0
    check_sample(orc, x, m, a, np.arange(0, n, 4), v, r_cut, E, F, par)


def test_pairs_across_the_boundary(pg, orc):
    r_cut, E, F = 0.1, 3, 5
    par = [r_cut / 4.5, 0.01]
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    rng = np.random.default_rng(1)
    # particles hugging faces, edges and corners of the unit box
    x = np.mod(rng.normal(0.0, 0.03, (4000, 3)), 1.0)
    m = np.full(len(x), 1.0 / len(x))
    a, _, _ = run_cells(pg, x, m, v, r_cut, E, F)
    check_sample(orc, x, m, a, np.arange(len(x)), v, r_cut, E, F, par)


def test_clustered_2e21_sampled(pg, orc):
    """2^21 particles, 200 clumps, Gaussian split with r_s = 1/256,
    r_cut = 4.5 r_s, E = 4, F = 8, cells of side 1/56: 4096-particle sample
    against brute force over all particles with minimum image."""
    n = 1 << 21
    x, m = gen.clustered_box(n, gen.CONFIG_SEEDS[3])
    r_cut, E, F = 4.5 * RS, 4, 8
    par = [RS, RS / 16]
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    a, _, info = run_cells(pg, x, m, v, r_cut, E, F)
    idx = gen.sample_indices(n, 4096, 31)
    check_sample(orc, x, m, a, idx, v, r_cut, E, F, par)


def test_cell_path_errors(pg):
    x, m = gen.clustered_box(1000, 3)
    with pg.Context(0) as c:
        c.set_self(True)
        c.set_periodic(1.0)
        c.set_j(x, m)
        c.set_i(x)
        with pytest.raises(pg.PGError) as e:      # Newton mode
            c.run()
        assert e.value.code == pg.PG_ESTATE
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: 1.0, 0.5, 3, 5)      # r_cut > box / 3
        with pytest.raises(pg.PGError) as e:
            c.run()
        assert e.value.code == pg.PG_ESTATE
