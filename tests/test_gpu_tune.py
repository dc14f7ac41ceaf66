"""The autotuner (pg_tune) on each path: it keeps one of its candidate launch
shapes, later runs use it, and their forces match the oracle as untuned
ones do. Also the split setter's range."""

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
    ao, po = orc.newton_groups(d["i_off"], d["j_off"], d["jlist"], d["xi"], d["xj"], d["mj"], 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_split_range(pg):
    with pg.Context(0) as c:
        for bad in (-1, 9):
            with pytest.raises(pg.PGError) as e:
                c.set_split(bad)
            assert e.value.code == pg.PG_EINVAL
        c.set_split(0)
