"""Parity of the two extensions with the FP64 oracle through the C ABI, on
every path that evaluates them:

- Per-i softening (PG_NEWTON). The i-particle structure of Section 3.1
  carries eps^2 per i, and the kernel of Section 3.3 adds the i-particle's
  eps^2. Covered: the tiled all-pairs path in self mode (zero softenings
  included), the narrow path, tree groups in list mode, host and device
  setters, clearing, graph replay with new values, and the errors.
- Table-mode potential (PG_TABLE). phi_i = sum_j m_j psi~ from a second
  table on the force table's knots. Covered: tiled all-pairs, narrow, list
  mode, the periodic cell list in self mode, graph replay, and the errors.

Tolerances as for the base paths: per-particle relative error median <=
2e-6 and max <= 1e-4. For the potential, the allowance of pair terms within
rounding distance of the cutoff is applied as for forces.
"""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def eps_for(n, seed, zero_every=0):
    e = np.random.default_rng(seed).uniform(0.005, 0.05, n)
    if zero_every:
        e[::zero_every] = 0.0
    return e


# ------------------------------------------------------------ per-i softening

@pytest.mark.parametrize("zero_every", [0, 7])
def test_eps_i_tiled_self_mode(pg, orc, zero_every):
    x, m = gen.uniform_sphere(3000, 61)     # compact: unsorted tiles stay small
    e = eps_for(len(x), 1, zero_every)
    with pg.Context(0) as c:
        c.set_eps(0.02)                     # overridden by the per-i values
        c.set_self(True)
        c.set_allpairs_path(pg.PG_PATH_TILED)
        c.set_eps_i(e)
        a, p = c.forces(x, x, m)
    ao, po = orc.newton_epsi(x, e, x, m, skip=np.arange(len(x)))
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_eps_i_narrow_path(pg, orc):
    xj, mj = gen.plummer_cube_mix(50000, 4242)
    x = gen.plummer(6000, 905)[0]
    xi = x[np.argsort(np.linalg.norm(x, axis=1))[:300]]
    e = eps_for(300, 2)
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_NARROW)
        c.set_eps_i(e)
        a, p = c.forces(xi, xj, mj)
    ao, po = orc.newton_epsi(xi, e, xj, mj)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_eps_i_groups(pg, orc):
    d = gen.tree_groups(gen.CONFIG_SEEDS[4] + 20, n=1 << 15, ngroups=120, n_monopoles=1 << 11,
                        nj_range=(64, 3000))
    e = eps_for(len(d["xi"]), 3)
    with pg.Context(0) as c:
        c.set_eps_i(e)
        c.set_j(d["xj"], d["mj"])
        c.set_i(d["xi"])
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        c.run()
        a, p = c.get_force(len(d["xi"]))
    ao = np.empty_like(a)
    po = np.empty_like(p)
    for g in range(len(d["i_off"]) - 1):
        i0, i1 = d["i_off"][g], d["i_off"][g + 1]
        jl = d["jlist"][d["j_off"][g]:d["j_off"][g + 1]]
        ao[i0:i1], po[i0:i1] = orc.newton_epsi(d["xi"][i0:i1], e[i0:i1], d["xj"][jl], d["mj"][jl])
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_eps_i_device_clear_and_graph(pg, orc):
    torch = pytest.importorskip("torch")
    x, m = gen.uniform_sphere(2000, 62)
    e1, e2 = eps_for(2000, 4), eps_for(2000, 5)
    with pg.Context(0) as c:
        c.set_self(True)
        c.set_eps(0.03)
        c.set_graph(True)
        c.set_j(x, m)
        c.set_i(x)
        c.set_eps_i_dev(torch.tensor(e1, device="cuda"))
        for _ in range(3):                  # uncaptured, captured, replayed
            c.run()
        a1, _ = c.get_force(2000)
        c.set_eps_i(e2)                     # new values, same graph
        c.run()
        a2, _ = c.get_force(2000)
        c.set_eps_i(None)                   # back to the global eps
        c.run()
        a3, p3 = c.get_force(2000)
    skip = np.arange(2000)
    assert_parity(rel_vec(a1, orc.newton_epsi(x, e1, x, m, skip=skip)[0]), what="a, eps 1")
    assert_parity(rel_vec(a2, orc.newton_epsi(x, e2, x, m, skip=skip)[0]), what="a, eps 2")
    ao, po = orc.newton(x, x, m, 0.03, skip=skip)
    assert_parity(rel_vec(a3, ao), what="a, global eps")
    assert_parity(rel_scalar(p3, po), what="phi, global eps")


def test_eps_i_errors(pg):
    x, m = gen.plummer(100, 63)
    with pg.Context(0) as c:
        with pytest.raises(pg.PGError) as ex:
            c.set_eps_i(np.array([0.1, -1.0]))
        assert ex.value.code == pg.PG_EINVAL
        c.set_eps_i(np.full(50, 0.1))       # 50 values against 100 i
        c.set_j(x, m)
        c.set_i(x)
        with pytest.raises(pg.PGError) as ex:
            c.run()
        assert ex.value.code == pg.PG_ESTATE
        c.set_eps_i(np.full(100, 0.1))
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: 1.0, 0.3, 3, 5)
        with pytest.raises(pg.PGError) as ex:
            c.run()
        assert ex.value.code == pg.PG_ESTATE


# ------------------------------------------------------ table-mode potential

R_CUT, E, F = 0.1, 3, 5
PAR_F = [R_CUT / 4.5, 1 / 64]
PAR_P = [0.02]


def tables(orc):
    vf = orc.table_values(E, F, R_CUT, orc.SHAPE_GAUSS_SPLIT, PAR_F)
    vp = orc.table_values(E, F, R_CUT, orc.SHAPE_NEWTON_POT, PAR_P)
    return vf, vp, orc.table_from_values(E, F, vf), orc.table_from_values(E, F, vp)


def check_pot(orc, p, xi, xj, mj, P, skip=None, box=0.0):
    po, amb = orc.table_potential(xi, xj, mj, E, F, R_CUT, P[0], P[1], skip=skip, box=box,
                                  window=1e-6)
    rel = np.maximum(np.abs(p - po) - amb, 0) / np.abs(po)
    assert_parity(rel, what="phi vs table semantics")


def dense_box(n, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * 0.35, rng.uniform(0.5, 1.5, n) / n


@pytest.mark.parametrize("path", ["tiled", "narrow"])
def test_table_potential_all_pairs(pg, orc, path):
    x, m = dense_box(3000, 71)
    vf, vp, G, P = tables(orc)
    n_i = 3000 if path == "tiled" else 200
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_allpairs_path(pg.PG_PATH_TILED if path == "tiled" else pg.PG_PATH_NARROW)
        c.set_table_values(vf, R_CUT, E, F)
        c.set_table_pot_values(vp)
        c.set_self(True)
        c.set_j(x, m)
        c.set_i(x[:n_i])
        c.run()
        a, p = c.get_force(n_i)
    skip = np.arange(n_i)
    check_pot(orc, p, x[:n_i], x, m, P, skip=skip)
    ao, amb = orc.table_forces(x[:n_i], x, m, E, F, R_CUT, G[0], G[1], skip=skip, window=1e-6)
    rel = np.maximum(np.linalg.norm(a - ao, axis=1) - amb, 0) / np.linalg.norm(ao, axis=1)
    assert_parity(rel, what="a vs table semantics (with the potential)")


def test_table_potential_groups_list_mode(pg, orc):
    x, m = dense_box(4000, 72)
    vf, vp, G, P = tables(orc)
    rng = np.random.default_rng(5)
    sizes_i, sizes_j = [20, 300, 7, 600], [900, 3000, 50, 4000]
    i_off = np.concatenate([[0], np.cumsum(sizes_i)])
    j_off = np.concatenate([[0], np.cumsum(sizes_j)])
    jlist = np.concatenate([rng.integers(0, len(x), k) for k in sizes_j]).astype(np.int32)
    xi = x[rng.integers(0, len(x), i_off[-1])]
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_table_values(vf, R_CUT, E, F)
        c.set_table_pot_values(vp)
        c.set_j(x, m)
        c.set_i(xi)
        c.set_groups(i_off, j_off, jlist)
        c.run()
        _, p = c.get_force(len(xi))
    po = np.empty(len(xi))
    amb = np.empty(len(xi))
    for g in range(len(sizes_i)):
        i0, i1 = i_off[g], i_off[g + 1]
        jl = jlist[j_off[g]:j_off[g + 1]]
        po[i0:i1], amb[i0:i1] = orc.table_potential(xi[i0:i1], x[jl], m[jl], E, F, R_CUT, P[0],
                                                    P[1], window=1e-6)
    rel = np.maximum(np.abs(p - po) - amb, 0) / np.abs(po)
    assert_parity(rel, what="phi (list mode)")


def test_table_potential_cells(pg, orc):
    n = 1 << 15
    x, m = gen.clustered_box(n, 123, nclump=20, sigma=0.01)
    r_cut, Ec, Fc = 0.05, 4, 8
    vf = orc.table_values(Ec, Fc, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, r_cut / 72])
    vp = orc.table_values(Ec, Fc, r_cut, orc.SHAPE_NEWTON_POT, [r_cut / 72])
    P = orc.table_from_values(Ec, Fc, vp)
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_table_values(vf, r_cut, Ec, Fc)
        c.set_table_pot_values(vp)
        c.set_self(True)
        c.set_periodic(1.0)
        _, p = c.forces(x, x, m)
    idx = np.arange(0, n, 5)
    po, amb = orc.table_potential(x[idx], x, m, Ec, Fc, r_cut, P[0], P[1], skip=idx, box=1.0,
                                  window=1e-6)
    rel = np.maximum(np.abs(p[idx] - po) - amb, 0) / np.abs(po)
    assert_parity(rel, what="phi (cells)")


def test_table_potential_graph_and_api(pg, orc):
    x, m = dense_box(1500, 73)
    vf, vp, G, P = tables(orc)
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        with pytest.raises(pg.PGError) as ex:
            c.set_table_pot_values(vp)      # no force table yet
        assert ex.value.code == pg.PG_ESTATE
        c.set_table_values(vf, R_CUT, E, F)
        with pytest.raises(pg.PGError) as ex:
            c.set_table_pot_values(vp[:-1])
        assert ex.value.code == pg.PG_EINVAL
        c.set_table_pot(lambda r: orc.shape(orc.SHAPE_NEWTON_POT, PAR_P, r))
        c.set_self(True)
        c.set_graph(True)
        c.set_j(x, m)
        c.set_i(x)
        for _ in range(3):
            c.run()
        _, p = c.get_force(len(x))
        check_pot(orc, p, x, x, m, P, skip=np.arange(len(x)))
        c.set_table_pot(None)               # dropped: phi is zero again
        c.run()
        _, p0 = c.get_force(len(x))
        assert np.all(p0 == 0)
        c.set_table_pot_values(vp)
        c.set_table_values(vf, 2 * R_CUT, E, F)   # other knots: the potential goes
        c.run()
        _, p1 = c.get_force(len(x))
        assert np.all(p1 == 0)
