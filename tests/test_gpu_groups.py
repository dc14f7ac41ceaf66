"""Parity of the batched tree-style groups (each group of i-particles sums
its own j-list, Section 5.1 usage) with the oracle's list-mode sums, through
the C ABI: a small clustered workload in full, ragged and empty groups,
single-group and split-list identities, the tabulated force in list mode,
CUDA-graph replay, and the 20000-group workload on a sample of groups."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def run_groups(pg, d, eps, graph=False, reps=1, table=None, np_=0):
    with pg.Context(0) as c:
        c.set_eps(eps)
        if np_:
            c.set_shape(np_)
        if table is not None:
            c.set_mode(pg.PG_TABLE)
            c.set_table_values(*table)
        c.set_graph(graph)
        c.set_j(d["xj"], d["mj"])
        c.set_i(d["xi"])
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        for _ in range(reps):
            c.run()
        return c.get_force(len(d["xi"]))


@pytest.fixture(scope="module")
def small():
    return gen.tree_groups(gen.CONFIG_SEEDS[4] + 10, n=1 << 16, ngroups=300,
                           n_monopoles=1 << 12, nj_range=(64, 4000))


@pytest.mark.parametrize("np_", [1, 2, 4])
def test_small_tree_workload(pg, orc, small, np_):
    d = small
    a, p = run_groups(pg, d, 1e-3, np_=np_)
    ao, po = orc.newton_groups(d["i_off"], d["j_off"], d["jlist"], d["xi"], d["xj"], d["mj"], 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_graph_replay_matches(pg, small):
    a1, p1 = run_groups(pg, small, 1e-3)
    a2, p2 = run_groups(pg, small, 1e-3, graph=True, reps=3)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


def test_graph_replay_sees_new_j(pg, orc, small):
    d = small
    xj2 = d["xj"][:, [1, 2, 0]].copy()
    with pg.Context(0) as c:
        c.set_eps(1e-3)
        c.set_graph(True)
        c.set_j(d["xj"], d["mj"])
        c.set_i(d["xi"])
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        for _ in range(3):          # uncaptured, captured, replayed
            c.run()
        c.set_j(xj2, d["mj"])
        c.run()                     # replay with new records
        a, p = c.get_force(len(d["xi"]))
    ao, po = orc.newton_groups(d["i_off"], d["j_off"], d["jlist"], d["xi"], xj2, d["mj"], 1e-3)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_ragged_and_empty_groups(pg, orc):
    rng = np.random.default_rng(3)
    xj, mj = gen.plummer(6000, 5)
    # the last two are small items with empty lists, which run one after the
    # other in warp mode
    sizes_i = [1, 15, 16, 17, 0, 511, 512, 513, 1500, 3, 5, 2]
    sizes_j = [1, 7, 511, 512, 513, 3000, 0, 1025, 64, 6000, 0, 0]
    i_off = np.concatenate([[0], np.cumsum(sizes_i)])
    j_off = np.concatenate([[0], np.cumsum(sizes_j)])
    jlist = np.concatenate([rng.integers(0, len(xj), k) for k in sizes_j]).astype(np.int32)
    xi = gen.plummer(int(i_off[-1]), 6)[0]
    d = dict(xj=xj, mj=mj, xi=xi, i_off=i_off, j_off=j_off, jlist=jlist)
    a, p = run_groups(pg, d, 0.01)
    ao, po = orc.newton_groups(i_off, j_off, jlist, xi, xj, mj, 0.01)
    nz = np.linalg.norm(ao, axis=1) > 0
    assert np.all(a[~nz] == 0) and np.all(p[~nz] == 0)
    assert_parity(rel_vec(a[nz], ao[nz]), what="a")
    assert_parity(rel_scalar(p[nz], po[nz]), what="phi")


def test_single_group_equals_all_pairs_and_lists_add(pg, orc):
    x, m = gen.plummer(3000, 7)
    n = len(x)
    probes = gen.plummer(200, 8)[0]
    one = dict(xj=x, mj=m, xi=probes, i_off=[0, 200], j_off=[0, n],
               jlist=np.arange(n, dtype=np.int32))
    a1, p1 = run_groups(pg, one, 0.02)
    ao, po = orc.newton(probes, x, m, 0.02)
    assert_parity(rel_vec(a1, ao), what="a")
    half = n // 2
    two = dict(xj=x, mj=m, xi=np.concatenate([probes, probes]), i_off=[0, 200, 400],
               j_off=[0, half, n], jlist=np.arange(n, dtype=np.int32))
    a2, p2 = run_groups(pg, two, 0.02)
    assert_parity(rel_vec(a2[:200] + a2[200:], ao), what="a (split)")
    assert_parity(rel_scalar(p2[:200] + p2[200:], po), what="phi (split)")


def test_table_force_in_list_mode(pg, orc, small):
    d = small
    E, F, r_cut = 4, 8, 0.05
    par = [r_cut / 4.5, 1e-3]
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    G0, G1 = orc.table_from_values(E, F, v)
    a, _ = run_groups(pg, d, 0.0, table=(v, r_cut, E, F))
    rel = []
    for g in range(0, len(d["i_off"]) - 1, 7):
        i0, i1 = d["i_off"][g], d["i_off"][g + 1]
        lst = d["jlist"][d["j_off"][g]:d["j_off"][g + 1]]
        ao, amb = orc.table_forces(d["xi"][i0:i1], d["xj"][lst], d["mj"][lst], E, F, r_cut, G0, G1,
                                   window=1e-6)
        norm = np.linalg.norm(ao, axis=1)
        ok = norm > 0
        err = np.maximum(np.linalg.norm(a[i0:i1] - ao, axis=1) - amb, 0)
        rel.extend((err[ok] / norm[ok]).tolist())
    assert_parity(np.array(rel), what="a (table list mode)")


def test_bad_lists_are_rejected(pg):
    x, m = gen.plummer(100, 9)
    with pg.Context(0) as c:
        c.set_j(x, m)
        c.set_i(x[:10])
        with pytest.raises(pg.PGError) as e:
            c.set_groups([0, 10], [0, 2], np.array([3, -1], np.int32))
        assert e.value.code == pg.PG_EINVAL
        with pytest.raises(pg.PGError) as e:
            c.set_groups([1, 10], [0, 2], np.array([3, 4], np.int32))
        assert e.value.code == pg.PG_EINVAL
        c.set_groups([0, 10], [0, 2], np.array([3, 100], np.int32))   # j 100 not written
        with pytest.raises(pg.PGError) as e:
            c.run()
        assert e.value.code == pg.PG_ESTATE


def test_tree_workload_20000_groups_sampled(pg, orc):
    """The 20000-group workload on its 2^22-particle set, in the launch
    configuration the benchmark row uses, checked on 600 sampled groups."""
    d = gen.tree_groups(gen.CONFIG_SEEDS[4])
    eps = 1e-3
    a, p = run_groups(pg, d, eps)
    rng = np.random.default_rng(4)
    gs = np.sort(rng.choice(len(d["i_off"]) - 1, 600, replace=False))
    ni = d["i_off"][gs + 1] - d["i_off"][gs]
    nj = d["j_off"][gs + 1] - d["j_off"][gs]
    i_off = np.concatenate([[0], np.cumsum(ni)])
    j_off = np.concatenate([[0], np.cumsum(nj)])
    xi = np.concatenate([d["xi"][d["i_off"][g]:d["i_off"][g + 1]] for g in gs])
    jl = np.concatenate([d["jlist"][d["j_off"][g]:d["j_off"][g + 1]] for g in gs])
    ao, po = orc.newton_groups(i_off, j_off, jl, xi, d["xj"], d["mj"], eps)
    sel = np.concatenate([np.arange(d["i_off"][g], d["i_off"][g + 1]) for g in gs])
    assert_parity(rel_vec(a[sel], ao), what="a")
    assert_parity(rel_scalar(p[sel], po), what="phi")
