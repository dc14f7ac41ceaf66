"""The particle-mesh long-range force on the GPU against the PM oracle (the
same method in FP64), and PP + PM against the Ewald sum.

Tolerance: the GPU mesh is FP32 (atomic assignment, cuFFT, interpolation),
so its error is a small multiple of 2^-24 times log2(N^3) of the field's
typical size: per particle |a_gpu - a_oracle| is compared with the RMS
acceleration, median <= 1e-5 and max <= 1e-4 (about 10 and 100 times the
~1e-6 expected).
"""

import math

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


@pytest.mark.parametrize("split,N,scale_cells,L", [("gauss", 64, 1.25, 1.0), ("s2", 32, 4.0, 1.0),
                                                   ("gauss", 48, 1.5, 3.0)])
def test_pm_matches_the_oracle(pg, split, N, scale_cells, L):
    x, m = gen.clustered_box(20000, 61, nclump=30, sigma=0.03)
    x = x * L
    m = m * np.random.default_rng(3).uniform(0.5, 2.0, len(m))
    scale = scale_cells * L / N
    with pg.Context(0) as c:
        c.set_periodic(L)
        c.set_pm(N, pg.PG_SPLIT_GAUSS if split == "gauss" else pg.PG_SPLIT_S2, scale)
        a, p = c.pm_forces(x, m)
    ao, po = opm.mesh_forces(x, m, L, N, split, scale)
    assert_mesh_parity(a, ao, "a")
    assert_mesh_parity(p[:, None], po[:, None], "phi")


def test_deposit_runs_of_one_mesh_point(pg):
    # The one-call deposit reads the particles in mesh order, where those of
    # one mesh point are consecutive lanes whose weights a warp sums before
    # its atomics. Runs of 1 to 70 particles around 300 points (runs that
    # cross warps and end at lane 31), each particle a little off its point
    # (distinct weights), plus a uniform background: the one-call forces
    # against the oracle, and against the two-step form, which deposits in
    # input order without the runs
    rng = np.random.default_rng(7501)
    N = 32
    pts = rng.integers(0, N, size=(300, 3))
    sizes = rng.integers(1, 71, size=300)
    cl = np.repeat(pts, sizes, axis=0) / N + rng.uniform(-0.3, 0.3, (sizes.sum(), 3)) / N
    x = np.mod(np.concatenate([cl, rng.random((3000, 3))]), 1.0)
    x = x[rng.permutation(len(x))]
    m = rng.uniform(0.5, 1.5, len(x)) / len(x)
    scale = 1.25 / N
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(N, pg.PG_SPLIT_GAUSS, scale)
        a, p = c.pm_forces(x, m)
    ao, po = opm.mesh_forces(x, m, 1.0, N, "gauss", scale)
    assert_mesh_parity(a, ao, "a")
    assert_mesh_parity(p[:, None], po[:, None], "phi")
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(N, pg.PG_SPLIT_GAUSS, scale)
        r = torch.empty(N ** 3, dtype=torch.float32, device=dev)
        c.pm_deposit_dev(xd, md, r)
        a2 = torch.empty_like(xd)
        p2 = torch.empty_like(md)
        c.pm_solve_dev(r, xd, a2, p2)
        torch.cuda.synchronize()
    assert_mesh_parity(a2.cpu().numpy(), a, "two steps against one call")


def test_positions_outside_the_box_wrap(pg):
    x, m = gen.clustered_box(5000, 62, nclump=10, sigma=0.02)
    shift = np.random.default_rng(4).integers(-3, 4, size=x.shape).astype(np.float64)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(32, pg.PG_SPLIT_GAUSS, 1.25 / 32)
        a0, _ = c.pm_forces(x, m)
        a1, _ = c.pm_forces(x + shift, m)
    assert_mesh_parity(a1, a0, "wrapped")


def _table_run(pg, x, m, v, r_cut, E, F, pm_args=None):
    with pg.Context(0) as c:
        c.set_mode(pg.PG_TABLE)
        c.set_table_values(v, r_cut, E, F)
        c.set_self(True)
        c.set_periodic(1.0)
        if pm_args:
            c.set_pm(*pm_args)
        a, _ = c.forces(x, x, m)
    return a


def test_run_adds_the_mesh_to_the_pp_forces(pg, orc):
    # a periodic table-mode run with the mesh set returns PP + PM: the
    # difference from the PP-only run is the mesh force of the oracle
    x, m = gen.clustered_box(1 << 15, 63, nclump=20, sigma=0.01)
    N, rs = 128, 1.25 / 128
    r_cut, E, F = 4.5 * rs, 4, 8
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [rs, rs / 16])
    pp = _table_run(pg, x, m, v, r_cut, E, F)
    tot = _table_run(pg, x, m, v, r_cut, E, F, (N, pg.PG_SPLIT_GAUSS, rs))
    ao, _ = opm.mesh_forces(x, m, 1.0, N, "gauss", rs)
    assert_mesh_parity(tot - pp, ao, "run - PP")


def _pp_exact(x, m, shape, r_cut, L=1.0):
    acc = np.zeros_like(x)
    for i in range(len(x)):
        d = x - x[i]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=1)
        s = (r > 0) & (r < r_cut)
        acc[i] = np.sum((m[s] * np.array([shape(v) for v in r[s]]))[:, None] * d[s], axis=0)
    return acc


@pytest.mark.parametrize("split", ["gauss", "s2"])
def test_pp_plus_pm_against_ewald(pg, orc, split):
    # the paper's check of PP + PM (Section 4.2), here with random particles
    # in a periodic box: the GPU's tabulated PP plus its mesh against the
    # exact short-range sum plus the exact k-space sum
    n, N = 1500, 64
    rng = np.random.default_rng(64)
    x = rng.random((n, 3))
    m = rng.uniform(0.5, 1.5, n)
    E, F = 4, 8
    if split == "gauss":
        rs = 1.25 / N
        r_cut, scale, eps = 4.5 * rs, rs, rs / 16
        v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [rs, eps])
        def shape(r):
            return (math.erfc(r / (2 * rs)) + r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs))) / (r * r + eps * eps) ** 1.5
        sp = pg.PG_SPLIT_GAUSS
    else:
        # an S2 diameter the mesh resolves (about 10 cells): the S2 form
        # factor falls only as k^-8, so at 4 cells the modes beyond the
        # mesh's Nyquist frequency still hold about 1e-3 of the force
        r_cut = 0.15
        scale, eps = r_cut, r_cut / 15
        v = orc.table_values(E, F, r_cut, orc.SHAPE_S2PP, [eps, r_cut])
        def shape(r):
            return (orc.s2_profile(r, eps) - orc.s2_profile(r, r_cut)) / r
        sp = pg.PG_SPLIT_S2
    tot = _table_run(pg, x, m, v, r_cut, E, F, (N, sp, scale))
    ak, _ = opm.kspace_forces(x, m, 1.0, split, scale, 32)
    ref = _pp_exact(x, m, shape, r_cut) + ak
    err = np.linalg.norm(tot - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(err) < 2e-3 and np.percentile(err, 99) < 2e-2


def test_pm_errors(pg):
    x, m = gen.clustered_box(100, 65)
    with pg.Context(0) as c:
        with pytest.raises(pg.PGError) as e:
            c.pm_forces(x, m)                  # no mesh set
        assert e.value.code == pg.PG_ESTATE
        c.set_pm(32, pg.PG_SPLIT_GAUSS, 0.04)
        with pytest.raises(pg.PGError) as e:
            c.pm_forces(x, m)                  # no periodic box
        assert e.value.code == pg.PG_ESTATE
        for bad in ((33, pg.PG_SPLIT_GAUSS, 0.04), (32, 7, 0.04), (32, pg.PG_SPLIT_S2, 0.0), (4, 0, 0.1)):
            with pytest.raises(pg.PGError) as e:
                c.set_pm(*bad)
            assert e.value.code == pg.PG_EINVAL
        c.set_pm(0)                            # off


def test_pm_edge_cases(pg):
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(16, pg.PG_SPLIT_GAUSS, 1.25 / 16)
        a, p = c.pm_forces(np.zeros((0, 3)), np.zeros(0))      # no particles
        assert a.shape == (0, 3)
        # zero masses: no field anywhere
        x, _ = gen.clustered_box(500, 66)
        a, p = c.pm_forces(x, np.zeros(500))
        assert np.all(a == 0) and np.all(p == 0)
        # one particle: the oracle's mesh gives the same (tiny) self-force
        x1, m1 = np.array([[0.37, 0.52, 0.81]]), np.array([1.0])
        a, p = c.pm_forces(x1, m1)
    ao, po = opm.mesh_forces(x1, m1, 1.0, 16, "gauss", 1.25 / 16)
    assert np.allclose(a, ao, rtol=1e-4, atol=1e-5 * np.abs(po).max())
    assert np.allclose(p, po, rtol=1e-4)


def test_deposit_and_solve_in_two_steps(pg):
    # the two-step form of the multi-rank path on one GPU: the meshes of two
    # halves, summed, solved for all particles, give the one-call forces
    torch = pytest.importorskip("torch")
    x, m = gen.clustered_box(20000, 67, nclump=20, sigma=0.02)
    N = 64
    dev = torch.device("cuda:0")
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(N, pg.PG_SPLIT_GAUSS, 1.25 / N)
        a1 = torch.empty_like(xd)
        p1 = torch.empty_like(md)
        c.pm_forces_dev(xd, md, a1, p1)
        r0 = torch.empty(N ** 3, dtype=torch.float32, device=dev)
        r1 = torch.empty_like(r0)
        h = len(x) // 2
        c.pm_deposit_dev(xd[:h].contiguous(), md[:h].contiguous(), r0)
        c.pm_deposit_dev(xd[h:].contiguous(), md[h:].contiguous(), r1)
        a2 = torch.empty_like(xd)
        p2 = torch.empty_like(md)
        c.pm_solve_dev(r0 + r1, xd, a2, p2)
        # the sharded helper on a single rank is the one-call result too
        a3, p3 = c.pm_forces_sharded(xd, md, N)
        torch.cuda.synchronize()
    a1, a2, a3 = a1.cpu().numpy(), a2.cpu().numpy(), a3.cpu().numpy()
    assert_mesh_parity(a2, a1, "two steps")
    assert_mesh_parity(p2.cpu().numpy()[:, None], p1.cpu().numpy()[:, None], "two steps phi")
    assert_mesh_parity(a3, a1, "sharded helper")


def test_bench_size_mesh(pg):
    # the bench's mesh workload (2^21 clustered particles, 256^3, r_s = h):
    # the oracle's mesh from every particle, solved at a sample of them
    torch = pytest.importorskip("torch")
    x, m = gen.clustered_box(1 << 21, gen.CONFIG_SEEDS[3])
    N, rs = 256, 1.0 / 256
    dev = torch.device("cuda:0")
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    a = torch.empty_like(xd)
    p = torch.empty_like(md)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(N, pg.PG_SPLIT_GAUSS, rs)
        c.pm_forces_dev(xd, md, a, p)
        torch.cuda.synchronize()
    idx = np.random.default_rng(97).choice(len(x), 2000, replace=False)
    ao, po = opm.solve(opm.deposit(x, m, 1.0, N), x[idx], 1.0, N, "gauss", rs)
    a, p = a.cpu().numpy()[idx], p.cpu().numpy()[idx]
    assert_mesh_parity(a, ao, "a")
    assert_mesh_parity(p[:, None], po[:, None], "phi")


def test_pp_plus_pm_under_a_graph(pg, orc):
    # a periodic run with the mesh, captured in a CUDA graph and replayed,
    # gives the forces of the uncaptured run (up to the FP32 atomics' order)
    x, m = gen.clustered_box(1 << 14, 68, nclump=10, sigma=0.01)
    N, rs = 64, 1.25 / 64
    r_cut, E, F = 4.5 * rs, 4, 8
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, [rs, rs / 16])
    out = []
    for graph in (False, True):
        with pg.Context(0) as c:
            c.set_mode(pg.PG_TABLE)
            c.set_table_values(v, r_cut, E, F)
            c.set_self(True)
            c.set_periodic(1.0)
            c.set_pm(N, pg.PG_SPLIT_GAUSS, rs)
            c.set_graph(graph)
            c.set_j(x, m)
            c.set_i(x)
            for _ in range(3):            # capture, then replays
                c.run()
            out.append(c.get_force(len(x))[0])
    assert_mesh_parity(out[1], out[0], "graph")


def test_deposit_scalar_paths(pg):
    # the deposit adds a stencil row with vector atomics only when the mesh
    # side is a multiple of four and the mesh 16-byte aligned: a side of 18,
    # and a mesh that starts 4 bytes into its buffer, take the scalar atomics
    torch = pytest.importorskip("torch")
    x, m = gen.clustered_box(6000, 68, nclump=10, sigma=0.03)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(18, pg.PG_SPLIT_GAUSS, 1.5 / 18)
        a, p = c.pm_forces(x, m)
    ao, po = opm.mesh_forces(x, m, 1.0, 18, "gauss", 1.5 / 18)
    assert_mesh_parity(a, ao, "N = 18")
    assert_mesh_parity(p[:, None], po[:, None], "N = 18 phi")
    N = 32
    dev = torch.device("cuda:0")
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    with pg.Context(0) as c:
        c.set_periodic(1.0)
        c.set_pm(N, pg.PG_SPLIT_GAUSS, 1.25 / N)
        r_al = torch.empty(N ** 3, dtype=torch.float32, device=dev)
        r_mis = torch.empty(N ** 3 + 1, dtype=torch.float32, device=dev)[1:]
        assert r_mis.data_ptr() % 16 == 4
        c.pm_deposit_dev(xd, md, r_al)
        c.pm_deposit_dev(xd, md, r_mis)
        torch.cuda.synchronize()
    ra, rm = r_al.cpu().numpy(), r_mis.cpu().numpy()
    ro = opm.deposit(x, m, 1.0, N).ravel()
    # FP32 atomics in any order: each cell within a few roundings of its sum
    scale = np.abs(ro).max()
    assert np.abs(ra - ro).max() <= 1e-5 * scale and np.abs(rm - ro).max() <= 1e-5 * scale
