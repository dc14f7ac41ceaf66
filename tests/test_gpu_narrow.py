"""Parity of the narrow all-pairs path (a few i-particles against many j, the
individual time step regime of Section 5) with the FP64 oracle through the
C ABI: i-sets from 1 to 1000 particles (one warp per item up to CTA items,
ragged last chunks of i and j), Newton and tabulated forces, the self mode
with eps > 0 and eps = 0, agreement with the tiled path, graph replay with
kernel timing, and empty sets. Tolerances as for the tiled path: per-particle
relative error median <= 2e-6 and max <= 1e-4."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


@pytest.fixture(scope="module")
def jset():
    return gen.plummer_cube_mix(50000, 4242)


def run(pg, xi, xj, mj, eps, path, self_=False, graph=False, reps=1, table=None):
    with pg.Context(0) as c:
        c.set_allpairs_path(path)
        c.set_eps(eps)
        c.set_self(self_)
        c.set_graph(graph)
        if table is not None:
            c.set_mode(pg.PG_TABLE)
            c.set_table_values(*table)
        c.set_j(xj, mj)
        c.set_i(xi)
        for _ in range(reps):
            c.run()
        a, p = c.get_force(len(xi))
        return a, p, c.info()


def core_set(ni, seed):
    """ni particles of the dense core of a Plummer sphere: the ones with the
    shortest time steps, which an individual time step code updates most
    often. Compact, as the FP32 offsets from an i chunk's FP64 centre need
    for eps well below the interparticle spacing."""
    x = gen.plummer(20 * ni + 100, seed)[0]
    return x[np.argsort(np.linalg.norm(x, axis=1))[:ni]]


# 64 and 65 straddle the switch from the warp-mode kernel (one warp pass of
# at most 64 i) to CTA-mode items
@pytest.mark.parametrize("ni", [1, 16, 33, 64, 65, 100, 513, 1000])
def test_narrow_newton(pg, orc, jset, ni):
    xj, mj = jset
    xi = core_set(ni, 900 + ni)
    a, p, info = run(pg, xi, xj, mj, 1e-3, pg.PG_PATH_NARROW)
    assert info["slots"] > 1           # the j records were split into chunks
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("ni", [16, 513, 1000])
def test_narrow_newton_spread_i(pg, orc, jset, ni):
    # i spread over the whole sphere: softening of the 4096-body case
    xj, mj = jset
    xi = gen.plummer(ni, 900 + ni)[0]
    a, p, _ = run(pg, xi, xj, mj, 1 / 64, pg.PG_PATH_NARROW)
    ao, po = orc.newton(xi, xj, mj, 1 / 64)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_auto_path_takes_narrow_for_few_i(pg, orc, jset):
    xj, mj = jset
    xi = core_set(24, 77)
    a, p, info = run(pg, xi, xj, mj, 1e-3, pg.PG_PATH_AUTO)
    assert info["slots"] > 1 and info["pairs"] == 24 * len(xj)
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")


@pytest.mark.parametrize("eps", [0.02, 0.0])
def test_narrow_self_mode(pg, orc, eps):
    # i-particle k is j-particle k: the self pair is left out; the j-set is
    # ordered by radius so that the i-set is its compact core
    x, m = gen.plummer(5000, 31)
    x = x[np.argsort(np.linalg.norm(x, axis=1))]
    xi = x[:700]
    a, p, _ = run(pg, xi, x, m, eps, pg.PG_PATH_NARROW, self_=True)
    ao, po = orc.newton(xi, x, m, eps, skip=np.arange(700, dtype=np.int64))
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_narrow_equals_tiled(pg, jset):
    xj, mj = jset
    xi = core_set(300, 5)
    a1, p1, _ = run(pg, xi, xj, mj, 1e-3, pg.PG_PATH_NARROW)
    a2, p2, _ = run(pg, xi, xj, mj, 1e-3, pg.PG_PATH_TILED)
    assert_parity(rel_vec(a1, a2), what="a narrow vs tiled")
    assert_parity(rel_scalar(p1, p2), what="phi narrow vs tiled")


@pytest.mark.parametrize("ni", [7, 400])
def test_narrow_table(pg, orc, ni):
    rng = np.random.default_rng(ni)
    r_cut, E, F = 0.1, 3, 5
    xj = rng.random((20000, 3)) * 0.4
    mj = rng.uniform(0.5, 1.5, len(xj)) / len(xj)
    xi = rng.random((ni, 3)) * 0.4
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
    G0, G1 = orc.table_from_values(E, F, v)
    a, p, _ = run(pg, xi, xj, mj, 0.0, pg.PG_PATH_NARROW, table=(v, r_cut, E, F))
    assert np.all(p == 0)
    ao, amb = orc.table_forces(xi, xj, mj, E, F, r_cut, G0, G1, window=1e-6)
    rel = np.maximum(np.linalg.norm(a - ao, axis=1) - amb, 0) / np.linalg.norm(ao, axis=1)
    assert_parity(rel, what="a vs table semantics")


@pytest.mark.parametrize("path", ["narrow", "tiled"])
def test_graph_replay_and_kernel_time(pg, jset, path):
    xj, mj = jset
    xi = gen.plummer(64, 3)[0]
    p_ = pg.PG_PATH_NARROW if path == "narrow" else pg.PG_PATH_TILED
    a1, q1, _ = run(pg, xi, xj, mj, 1e-3, p_)
    with pg.Context(0) as c:
        c.set_allpairs_path(p_)
        c.set_eps(1e-3)
        c.set_graph(True)
        c.set_timing(True)
        c.set_j(xj, mj)
        c.set_i(xi)
        for _ in range(3):          # first call uncaptured, then capture, replay
            c.run()
            assert c.kernel_time() > 0.0
        a2, q2 = c.get_force(len(xi))
    assert np.array_equal(a1, a2) and np.array_equal(q1, q2)


def test_narrow_new_j_between_calls(pg, orc, jset):
    xj, mj = jset
    xi = core_set(40, 8)
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_eps(1e-3)
        c.set_j(xj, mj)
        c.set_i(xi)
        c.run()
        c.set_j(xj[:, ::-1].copy(), mj)     # new records: the cached packing is stale
        c.run()
        a, p = c.get_force(len(xi))
    ao, po = orc.newton(xi, xj[:, ::-1].copy(), mj, 1e-3)
    assert_parity(rel_vec(a, ao), what="a")


def test_graph_replay_sees_new_j(pg, orc, jset):
    # the double-float j packing is not part of the captured graph: a replay
    # after new records (same count) packs them first
    xj, mj = jset
    xi = core_set(24, 9)
    xj2 = xj[:, ::-1].copy()
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_eps(1e-3)
        c.set_graph(True)
        c.set_j(xj, mj)
        c.set_i(xi)
        for _ in range(3):          # uncaptured, captured, replayed
            c.run()
        a1, p1 = c.get_force(len(xi))
        c.set_j(xj2, mj)
        c.run()                     # replay with new records
        a2, p2 = c.get_force(len(xi))
        c.set_j(xj, mj)
        c.run()
        a3, p3 = c.get_force(len(xi))
    ao, po = orc.newton(xi, xj, mj, 1e-3)
    ao2, po2 = orc.newton(xi, xj2, mj, 1e-3)
    assert_parity(rel_vec(a1, ao), what="a")
    assert_parity(rel_vec(a2, ao2), what="a after new j")
    assert_parity(rel_scalar(p2, po2), what="phi after new j")
    assert np.array_equal(a1, a3) and np.array_equal(p1, p3)


def test_narrow_empty_sets(pg):
    xj, mj = gen.plummer(5000, 2)
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_eps(0.01)
        c.set_j(xj, mj)
        c.set_i(np.zeros((0, 3)))
        c.run()
        a, p = c.get_force(0)
        assert a.shape == (0, 3)
        c.set_n(0)
        c.set_i(xj[:10])
        c.run()
        a, p = c.get_force(10)
        assert np.all(a == 0) and np.all(p == 0)
