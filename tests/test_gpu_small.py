"""The one-launch path for small i-sets (double-float pair differences, pair
loop and the last block's combine in one kernel) against the FP64 oracle and
against the multi-launch tiled path: ragged tile and chunk counts, self and
non-self modes, a self offset, eps = 0, per-i softening, and repeated graph
replays (each replay must find every tile's ticket back at zero). A run's
launch count is checked on its second run: the first also packs the j
records' double-float pairs, which later runs reuse."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def run(pg, xi, xj, mj, eps, self_=False, off=None, np_=0, epsi=None, graph=False, reps=1):
    with pg.Context(0) as c:
        c.set_eps(eps)
        if off is not None:
            c.set_self_offset(off)
        else:
            c.set_self(self_)
        if np_:
            c.set_shape(np_, 0, 1)
        c.set_graph(graph)
        c.set_j(xj, mj)
        c.set_i(xi)
        if epsi is not None:
            c.set_eps_i(epsi)
        for _ in range(reps):
            c.run()
        a, p = c.get_force(len(xi))
        return a, p, c.info()


@pytest.mark.parametrize("n", [2, 255, 257, 1000, 4096, 9999])
def test_small_allpairs(pg, orc, n):
    x, m = gen.plummer(n, 5100 + n)
    a, p, info = run(pg, x, x, m, 1 / 64, self_=True, reps=2)
    assert info["launches"] == 1 and info["df"] == 1
    ao, po = orc.newton_allpairs(x, m, 1 / 64)
    assert_parity(rel_vec(a, ao), what=f"a n={n}")
    if n > 2:
        assert_parity(rel_scalar(p, po), what=f"phi n={n}")
    a2, p2, info2 = run(pg, x, x, m, 1 / 64, self_=True, np_=1)      # the multi-launch path
    assert info2["launches"] > 1
    assert_parity(rel_vec(a, a2), what=f"a small vs tiled n={n}")


@pytest.mark.parametrize("ni,nj", [(700, 3000), (3000, 700), (300, 40000)])
def test_small_non_self(pg, orc, ni, nj):
    xj, mj = gen.plummer_cube_mix(nj, 5200 + nj)
    xi = gen.plummer(ni, 5300 + ni)[0]
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_TILED)
        c.set_eps(1e-3)
        c.set_j(xj, mj)
        c.set_i(xi)
        c.run()
        c.run()
        a, p = c.get_force(ni)
        assert c.info()["launches"] == 1
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_small_eps_zero_and_per_i(pg, orc):
    x, m = gen.plummer(3000, 54)
    a, p, _ = run(pg, x, x, m, 0.0, self_=True)
    ao, po = orc.newton_allpairs(x, m, 0.0)
    assert_parity(rel_vec(a, ao), what="a eps=0")
    assert_parity(rel_scalar(p, po), what="phi eps=0")
    e = np.exp(np.random.default_rng(5).uniform(np.log(1 / 256), np.log(1 / 16), len(x)))
    a, p, _ = run(pg, x, x, m, 0.0, self_=True, epsi=e)
    ao, po = orc.newton_epsi(x, e, x, m, skip=np.arange(len(x)))
    assert_parity(rel_vec(a, ao), what="a per-i eps")
    assert_parity(rel_scalar(p, po), what="phi per-i eps")


def test_small_self_offset(pg, orc):
    x, m = gen.plummer(6000, 55)
    lo, hi = 2000, 4500
    a, p, info = run(pg, x[lo:hi], x, m, 1 / 64, off=lo, reps=2)
    assert info["launches"] == 1
    ao, po = orc.newton(x[lo:hi], x, m, 1 / 64, skip=np.arange(lo, hi))
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_small_graph_replays(pg, orc):
    x, m = gen.plummer(4096, gen.CONFIG_SEEDS[1])
    a, p, info = run(pg, x, x, m, 1 / 64, self_=True, graph=True, reps=7)
    ao, po = orc.newton_allpairs(x, m, 1 / 64)
    assert_parity(rel_vec(a, ao), what="a after replays")
    assert_parity(rel_scalar(p, po), what="phi after replays")
