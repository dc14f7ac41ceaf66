"""The autotuner (pg_tune) on each path: it keeps one of its candidate launch
shapes, later runs use it, and their forces match the oracle as untuned
ones do. Every compiled j-tile depth x block size of the batched kernel at
every i-per-thread count gives the oracle's group forces. Also the split and
tile setters' ranges."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def test_tune_tiled_allpairs(pg, orc):
    x, m = gen.plummer(8192, 77)
    with pg.Context(0) as c:
        c.set_eps(1 / 64)
        c.set_self(True)
        c.set_allpairs_path(pg.PG_PATH_TILED)
        c.set_j(x, m)
        c.set_i(x)
        c.tune()
        c.run()
        a, p = c.get_force(len(x))
        info = c.info()
    assert info["i_per_thread"] in (2, 4, 8)
    assert info["packed"] in (0, 1)
    assert info["split"] == 0
    ao, po = orc.newton_allpairs(x, m, 1 / 64)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_tune_narrow_split(pg, orc):
    xj, mj = gen.plummer(1 << 16, 78)
    xi = xj[np.argsort(np.linalg.norm(xj, axis=1))[:16]].copy()
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_j(xj, mj)
        c.set_i(xi)
        c.tune()
        c.run()
        a, p = c.get_force(len(xi))
        info = c.info()
    assert info["split"] in (1, 2, 4)
    assert info["slots"] > 1
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("split", [1, 3, 8])
def test_narrow_split_values(pg, orc, split):
    xj, mj = gen.plummer(1 << 15, 79)
    xi = gen.plummer(40, 80)[0]
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_split(split)
        c.set_j(xj, mj)
        c.set_i(xi)
        c.run()
        a, p = c.get_force(len(xi))
        assert c.info()["split"] == split
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_tune_groups(pg, orc):
    d = gen.tree_groups(gen.CONFIG_SEEDS[4] + 11, n=1 << 15, ngroups=200,
                        n_monopoles=1 << 11, nj_range=(64, 3000))
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_j(d["xj"], d["mj"])
        c.set_i(d["xi"])
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        c.tune()
        c.run()
        a, p = c.get_force(len(d["xi"]))
        info = c.info()
    assert info["i_per_thread"] in (2, 4, 8)
    assert (info["j_tile"], info["block_threads"]) in ((512, 128), (256, 128), (1024, 256), (512, 256))
    ao, po = orc.newton_groups(d["i_off"], d["j_off"], d["jlist"], d["xi"], d["xj"], d["mj"], 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("np_", [1, 2, 4])
@pytest.mark.parametrize("tile", [(512, 128), (256, 128), (1024, 256), (512, 256)])
def test_groups_every_tile_shape(pg, orc, tile, np_):
    # lists from 64 to 3000 j and groups of every size: CTA-mode and
    # warp-mode items, one- and multi-pass i sets
    d = gen.tree_groups(gen.CONFIG_SEEDS[4] + 12, n=1 << 15, ngroups=300,
                        n_monopoles=1 << 11, nj_range=(64, 3000))
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_shape(np_, 0, 1)
        c.set_groups_tile(*tile)
        c.set_j(d["xj"], d["mj"])
        c.set_i(d["xi"])
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        c.run()
        a, p = c.get_force(len(d["xi"]))
        info = c.info()
    assert (info["j_tile"], info["block_threads"]) == tile
    assert info["i_per_thread"] == 2 * np_
    ao, po = orc.newton_groups(d["i_off"], d["j_off"], d["jlist"], d["xi"], d["xj"], d["mj"], 1e-3)
    assert_parity(rel_vec(a, ao), what=f"a {tile} np={np_}")
    assert_parity(rel_scalar(p, po), what=f"phi {tile} np={np_}")


def test_groups_tile_range(pg):
    with pg.Context(0) as c:
        for bad in ((128, 128), (512, 64), (2048, 256)):
            with pytest.raises(pg.PGError) as e:
                c.set_groups_tile(*bad)
            assert e.value.code == pg.PG_EINVAL
        c.set_groups_tile(0, 0)


def test_split_range(pg):
    with pg.Context(0) as c:
        for bad in (-1, 9):
            with pytest.raises(pg.PGError) as e:
                c.set_split(bad)
            assert e.value.code == pg.PG_EINVAL
        c.set_split(0)


def test_tune_tree(pg, orc):
    x, m = gen.plummer(20000, 83)
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_self(True)
        c.set_tree(0.75, 64, 8)
        c.set_j(x, m)
        c.set_i(x)
        c.tune()
        c.run()
        a, p = c.get_force(len(x))
        assert c.info()["i_per_thread"] in (2, 4, 8)
    ao, po = orc.tree_forces(x, m, 1e-3, 0.75, 64, 8)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_tune_cell_list(pg, orc):
    n = 1 << 14
    x, m = gen.clustered_box(n, 84, nclump=10, sigma=0.01)
    r_cut, E, F = 0.05, 4, 8
    par = [r_cut / 4.5, r_cut / 72]
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_table_values(v, r_cut, E, F)
        c.set_self(True)
        c.set_periodic(1.0)
        c.set_j(x, m)
        c.set_i(x)
        c.tune()
        c.run()
        a, _ = c.get_force(n)
        assert c.info()["i_per_thread"] in (2, 4, 8)
    idx = np.arange(0, n, 8)
    G0, G1 = orc.table_from_values(E, F, v)
    ao, amb = orc.table_forces(x[idx], x, m, E, F, r_cut, G0, G1, box=1.0, skip=idx, window=1e-6)
    norm = np.linalg.norm(ao, axis=1)
    ok = norm > 0
    rel = np.maximum(np.linalg.norm(a[idx] - ao, axis=1) - amb, 0)[ok] / norm[ok]
    assert_parity(rel, what="a vs table semantics")
