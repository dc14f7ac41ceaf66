"""The tree call's two walks and its read-back discipline on the GPU.

- The group walk (one warp per group, breadth first) and the level walk (all
  groups level by level) make the same lists, bit for bit, and both equal
  the oracle's; forces from them are bit-identical.
- A call for a particle count seen before runs from the room the last exact
  call left, with one read-back; the first call, and one whose counts
  outgrow that room, read each count back before the stage that needs it
  (the fast attempt's results are then discarded), with the same lists.
- A group that opens more nodes on one level than the warp's queue holds
  (theta = 0 and leaves of one particle: every node of two or more is
  opened, 961 on level 8 of a 6000-particle Plummer tree) makes the call
  take the level walk.
"""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def same_lists(t, o):
    assert np.array_equal(t["perm"], o["perm"])
    assert np.array_equal(t["g_i0"], o["g_i0"]) and np.array_equal(t["g_ni"], o["g_ni"])
    assert np.array_equal(t["j_off"], o["j_off"])
    assert np.array_equal(t["jlist"], o["jlist"])


def room(x):
    return x + x // 8 + 256


def run_once(pg, c, x, m):
    c.set_j(x, m)
    c.set_i(x)
    c.run()
    a, p = c.get_force(len(x))
    return a, p, c.get_tree(), c.tree_stats()


@pytest.mark.parametrize("ncrit,quad", [(64, False), (256, False), (64, True)])
def test_group_walk_matches_level_walk_and_oracle(pg, orc, ncrit, quad):
    x, m = gen.plummer(20000, 7101)
    o = orc.tree_build(x, m, 0.75, ncrit, 8, quadrupole=quad)
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_self(True)
        c.set_tree(0.75, ncrit, 8, quadrupole=quad)
        a1, p1, t1, s1 = run_once(pg, c, x, m)
        a2, p2, t2, s2 = run_once(pg, c, x, m)
        c.set_tree_walk(pg.PG_TREE_WALK_LEVEL)
        a3, p3, t3, s3 = run_once(pg, c, x, m)
    # first call exact (keys, groups, list length, end), then from room
    assert s1["walk"] == 1 and s1["exact"] == 1 and s1["reads"] == 4
    assert s2["walk"] == 1 and s2["exact"] == 0 and s2["reads"] == 1
    assert s3["walk"] == 2 and s3["exact"] == 1
    assert 0 < s1["queue_peak"] <= pg.PG_TREE_WALK_QUEUE and s2["queue_peak"] == s1["queue_peak"]
    for t in (t1, t2, t3):
        same_lists(t, o)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    assert np.array_equal(a1, a3) and np.array_equal(p1, p3)
    ao, po = orc.tree_forces(x, m, 1e-3, 0.75, ncrit, 8, quadrupole=quad)
    assert_parity(rel_vec(a1, ao), what="a")
    assert_parity(rel_scalar(p1, po), what="phi")


def test_counts_beyond_the_room_rerun_exact(pg, orc):
    # the same particle count, four sets: a Plummer sphere, a clustered set
    # (twice the nodes, shorter lists), another sphere (its lists outgrow
    # the clustered set's room), the first sphere again (fits)
    n = 16384
    first = gen.plummer(n, 7102)
    xs = [first, gen.clustered_box(n, 7103, nclump=30, sigma=3e-4, periodic=False),
          gen.plummer(n, 7104), first]
    builds = [orc.tree_build(x, m, 0.75, 64, 8) for x, m in xs]
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_self(True)
        c.set_tree(0.75, 64, 8)
        prev = None        # (nodes, groups, list entries) of the last exact call
        outcomes = []
        for (x, m), o in zip(xs, builds):
            a, p, t, s = run_once(pg, c, x, m)
            same_lists(t, o)
            cnt = (len(o["nM"]), len(o["g_i0"]), len(o["jlist"]))
            if prev is None:
                assert s["exact"] == 1 and s["reads"] == 4
            else:
                over = any(k > min(room(q), bound) for k, q, bound in
                           zip(cnt, prev, (11 * n + 1, n, 1 << 32)))
                assert s["exact"] == int(over)
                outcomes.append(over)
                # the fast attempt's end read, then the exact call's four
                assert s["reads"] == (5 if over else 1)
            if s["exact"]:
                prev = cnt
            ao, po = orc.tree_forces(x, m, 1e-3, 0.75, 64, 8)
            assert_parity(rel_vec(a, ao), what="a")
            assert_parity(rel_scalar(p, po), what="phi")
        # both outcomes were met
        assert outcomes == [True, True, False]


def test_queue_overflow_takes_the_level_walk(pg, orc):
    x, m = gen.plummer(6000, 7105)
    o = orc.tree_build(x, m, 0.0, 64, 1)
    with pg.Context(0) as c:
        c.set_eps(0.01)
        c.set_self(True)
        c.set_tree(0.0, 64, 1)
        for _ in range(2):
            a, p, t, s = run_once(pg, c, x, m)
            same_lists(t, o)
            assert s["walk"] == 2 and s["exact"] == 1
            assert s["queue_peak"] > pg.PG_TREE_WALK_QUEUE
        # back to a theta whose groups fit their queues: the group walk again
        c.set_tree(0.75, 64, 8)
        a2, p2, t2, s2 = run_once(pg, c, x, m)
        same_lists(t2, orc.tree_build(x, m, 0.75, 64, 8))
        assert s2["walk"] == 1
    ao, po = orc.newton_allpairs(x, m, 0.01)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_parameter_and_size_changes(pg, orc):
    # new ncrit, theta and pseudo-particle count on the same particles, then
    # another particle count: every call's lists equal the oracle's
    x, m = gen.king(12000, 7106, W0=9.0)
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_self(True)
        for theta, ncrit, quad in [(0.75, 64, False), (0.75, 128, False), (0.5, 128, False),
                                   (0.5, 128, True), (1.0, 32, True)]:
            c.set_tree(theta, ncrit, 8, quadrupole=quad)
            _, _, t, s = run_once(pg, c, x, m)
            same_lists(t, orc.tree_build(x, m, theta, ncrit, 8, quadrupole=quad))
        x2, m2 = x[:7001], m[:7001] * (12000 / 7001)
        pg.pg_set_n(c.h, len(x2))         # the j memory keeps its high-water mark
        _, _, t, s = run_once(pg, c, x2, m2)
        assert s["exact"] == 1            # a new particle count
        same_lists(t, orc.tree_build(x2, m2, 1.0, 32, 8, quadrupole=True))


def test_tree_walk_mode_errors(pg):
    with pg.Context(0) as c:
        with pytest.raises(pg.PGError) as e:
            c.set_tree_walk(7)
        assert e.value.code == pg.PG_EINVAL
        c.set_tree_walk(pg.PG_TREE_WALK_LEVEL)
        c.set_tree_walk(pg.PG_TREE_WALK_AUTO)


def test_keys_on_and_beside_cell_edges(pg, orc):
    # Coordinates k / 256 in [0, 1] (span 1): 1024 (x - lo) / span is an
    # integer, where the key takes the exact quotient; the same points one
    # ulp below and above, where the rounded quotient decides the cell; and
    # random points, where the product with 1024 / span does. The lists
    # (keys, groups, entries) equal the oracle's, which divides.
    rng = np.random.default_rng(7107)
    k = rng.integers(0, 257, size=(3000, 3)).astype(np.float64) / 256.0
    lo_ulp = np.nextafter(k, -np.inf)
    hi_ulp = np.nextafter(k, np.inf)
    x = np.concatenate([k, np.clip(lo_ulp, 0.0, 1.0), np.clip(hi_ulp, 0.0, 1.0),
                        rng.uniform(0.0, 1.0, size=(3000, 3)),
                        np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])])
    m = np.full(len(x), 1.0 / len(x))
    for theta in (0.75, 0.4):
        with pg.Context(0) as c:
            c.set_eps(1e-3)
            c.set_self(True)
            c.set_tree(theta, 32, 4)
            a, p, t, s = run_once(pg, c, x, m)
        same_lists(t, orc.tree_build(x, m, theta, 32, 4))
        ao, po = orc.tree_forces(x, m, 1e-3, theta, 32, 4)
        assert_parity(rel_vec(a, ao), what="a")
        assert_parity(rel_scalar(p, po), what="phi")


def test_recorded_and_rewalked_groups(pg, orc):
    # a call from room replays the count pass's recorded emitters (accepted
    # nodes and leaves) in the fill pass; a group with more than 4096 of them
    # (186 of the 1149 groups here, theta = 0.3) is walked again instead. The
    # lists of both kinds equal the oracle's
    x, m = gen.plummer(20000, 7108)
    o = orc.tree_build(x, m, 0.3, 64, 8)
    assert np.max(np.diff(o["j_off"])) > 4096
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_self(True)
        c.set_tree(0.3, 64, 8)
        a1, p1, t1, s1 = run_once(pg, c, x, m)
        a2, p2, t2, s2 = run_once(pg, c, x, m)
    assert s1["exact"] == 1 and s2["exact"] == 0 and s2["walk"] == 1
    same_lists(t1, o)
    same_lists(t2, o)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
