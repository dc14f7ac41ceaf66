"""The tree front end (the tree usage of Section 5.1) on the GPU against the
oracle's tree:

- The key order, the groups and every interaction list are identical, bit
  for bit (index work).
- Quadrupole pseudo-particles agree up to the rounding of the moments.
- Forces and potentials from those lists agree within the Newton
  tolerances (median <= 2e-6, max <= 1e-4).
- theta = 0 reproduces the direct sum.
Covered: a Plummer sphere, a King model (W0 = 9), a clustered set with dense
finest-level cells, the paper's theta = 0.75, several ncrit and nleaf,
monopole and quadrupole pseudo-particles, opening decisions at the
threshold, scaled coordinates, and the errors.
"""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def gpu_tree(pg, x, m, eps, theta, ncrit, nleaf, quadrupole=False):
    with pg.Context(0) as c:
        c.set_eps(eps)
        c.set_self(True)
        c.set_tree(theta, ncrit, nleaf, quadrupole=quadrupole)
        a, p = c.forces(x, x, m)
        t = c.get_tree()
        info = c.info()
    return a, p, t, info


def same_pseudo(t, o):
    # the same pseudo-particles up to the rounding of the moments: a spread
    # from a difference of eigenvalues that is zero in exact arithmetic (two-
    # or three-particle nodes) is sqrt(rounding) of the node's spread, so the
    # bound is relative to that spread sqrt(tr T / M), plus the coordinates'
    # own rounding
    P = o["npseudo"]
    spread = np.sqrt(np.maximum(o["nT"][:, [0, 3, 5]].sum(axis=1), 0) / o["nM"])
    tol = np.repeat(1e-6 * spread, P) + 1e-13 * np.abs(o["pseudo"][:, :3]).max()
    d = np.abs(t["pseudo"][:, :3] - o["pseudo"][:, :3]).max(axis=1)
    assert np.all(d <= tol), f"{np.count_nonzero(d > tol)} pseudo-particles differ"
    assert np.allclose(t["pseudo"][:, 3], o["pseudo"][:, 3], rtol=1e-13, atol=0)


def same_lists(t, o):
    assert np.array_equal(t["perm"], o["perm"])
    assert np.array_equal(t["g_i0"], o["g_i0"]) and np.array_equal(t["g_ni"], o["g_ni"])
    assert np.array_equal(t["j_off"], o["j_off"])
    assert np.array_equal(t["jlist"], o["jlist"])


@pytest.mark.parametrize("theta,ncrit,nleaf", [(0.75, 64, 8), (0.5, 32, 4), (1.0, 128, 16)])
def test_plummer_lists_and_forces(pg, orc, theta, ncrit, nleaf):
    x, m = gen.plummer(20000, 81)
    a, p, t, info = gpu_tree(pg, x, m, 1e-3, theta, ncrit, nleaf)
    o = orc.tree_build(x, m, theta, ncrit, nleaf)
    same_lists(t, o)
    assert t["nnodes"] == len(o["nM"]) and t["ngroups"] == len(o["g_i0"])
    assert info["pairs"] == int(np.sum(o["g_ni"] * np.diff(o["j_off"])))
    ao, po = orc.tree_forces(x, m, 1e-3, theta, ncrit, nleaf)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_clustered_set_with_dense_cells(pg, orc):
    # clumps far narrower than a finest cell: groups larger than ncrit
    x, m = gen.clustered_box(30000, 82, nclump=40, sigma=2e-4, periodic=False)
    m = m * np.random.default_rng(3).uniform(0.5, 2.0, len(m))
    a, p, t, _ = gpu_tree(pg, x, m, 1e-4, 0.75, 32, 8)
    o = orc.tree_build(x, m, 0.75, 32, 8)
    same_lists(t, o)
    assert np.max(o["g_ni"]) > 32
    ao, po = orc.tree_forces(x, m, 1e-4, 0.75, 32, 8)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_theta_zero_is_the_direct_sum(pg, orc):
    x, m = gen.plummer(6000, 83)
    a, p, _, _ = gpu_tree(pg, x, m, 0.01, 0.0, 64, 8)
    ao, po = orc.newton_allpairs(x, m, 0.01)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_eps_zero_and_repeat_runs(pg, orc):
    x, m = gen.plummer(5000, 84)
    with pg.Context(0) as c:
        c.set_eps(0.0)
        c.set_self(True)
        c.set_tree(0.75, 64, 8)
        c.set_j(x, m)
        c.set_i(x)
        c.run()
        a1, p1 = c.get_force(len(x))
        c.run()
        a2, p2 = c.get_force(len(x))
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    ao, po = orc.tree_forces(x, m, 0.0, 0.75, 64, 8)
    assert_parity(rel_vec(a1, ao), what="a")
    assert_parity(rel_scalar(p1, po), what="phi")


def test_tree_errors(pg):
    x, m = gen.plummer(100, 85)
    with pg.Context(0) as c:
        with pytest.raises(pg.PGError) as e:
            c.set_tree(0.5, 0, 8)
        assert e.value.code == pg.PG_EINVAL
        c.set_tree(0.5, 16, 4)
        c.set_j(x, m)
        c.set_i(x)
        with pytest.raises(pg.PGError) as e:      # not the self mode
            c.run()
        assert e.value.code == pg.PG_ESTATE
        c.set_self(True)
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: 1.0, 0.3, 3, 5)
        with pytest.raises(pg.PGError) as e:      # tree is Newton only
            c.run()
        assert e.value.code == pg.PG_ESTATE
        c.set_mode(pg.PG_NEWTON)
        c.set_tree(-1.0)                          # off: the all-pairs path again
        c.run()


@pytest.mark.parametrize("rel", [-1e-12, 1e-12])
def test_opening_at_the_threshold(pg, orc, rel):
    # a probe and a 4-particle cluster whose level-1 node is accepted exactly
    # when span / 2 < theta |c|; theta within 1e-12 of that value leaves the
    # FP32 pre-test undecided, so the FP64 test takes the decision
    h = 1.0 / 64.0
    c = np.array([0.75, 0.75, 0.5])
    x = np.array([[0.0, 0.0, 0.0], c + [h, h, 0], c + [-h, h, 0], c + [h, -h, 0], c + [-h, -h, 0]])
    m = np.ones(5)
    theta = (0.75 + h) / 2 / np.linalg.norm(c) * (1.0 + rel)
    _, _, t, _ = gpu_tree(pg, x, m, 0.0, theta, 1, 1)
    same_lists(t, orc.tree_build(x, m, theta, 1, 1))


@pytest.mark.parametrize("scale", [1e-9, 1e6, 1e25])
def test_scaled_sets(pg, orc, scale):
    # tiny and huge coordinates: outside the FP32 pre-test's range every
    # decision is FP64; inside it the bounds must still give the same lists
    x, m = gen.plummer(8000, 86)
    x = (x + np.array([0.3, -0.2, 0.1])) * scale
    a, p, t, _ = gpu_tree(pg, x, m, 1e-3 * scale, 0.75, 64, 8)
    same_lists(t, orc.tree_build(x, m, 0.75, 64, 8))
    if scale > 1e18:
        return          # the FP32 pair arithmetic overflows at r^2 ~ 1e50
    ao, po = orc.tree_forces(x, m, 1e-3 * scale, 0.75, 64, 8)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("theta,ncrit,nleaf", [(0.75, 64, 8), (0.5, 32, 4)])
def test_quadrupole_lists_and_forces(pg, orc, theta, ncrit, nleaf):
    x, m = gen.plummer(20000, 87)
    m = m * np.random.default_rng(7).uniform(0.5, 2.0, len(m))
    a, p, t, info = gpu_tree(pg, x, m, 1e-3, theta, ncrit, nleaf, quadrupole=True)
    o = orc.tree_build(x, m, theta, ncrit, nleaf, quadrupole=True)
    assert t["npseudo"] == 3
    same_lists(t, o)
    same_pseudo(t, o)
    assert info["pairs"] == int(np.sum(o["g_ni"] * np.diff(o["j_off"])))
    ao, po = orc.tree_forces(x, m, 1e-3, theta, ncrit, nleaf, quadrupole=True)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_quadrupole_clustered_and_direct(pg, orc):
    x, m = gen.clustered_box(30000, 88, nclump=40, sigma=2e-4, periodic=False)
    a, p, t, _ = gpu_tree(pg, x, m, 1e-4, 0.75, 32, 8, quadrupole=True)
    same_lists(t, orc.tree_build(x, m, 0.75, 32, 8, quadrupole=True))
    ao, po = orc.tree_forces(x, m, 1e-4, 0.75, 32, 8, quadrupole=True)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")
    x, m = gen.plummer(6000, 89)
    a, p, _, _ = gpu_tree(pg, x, m, 0.01, 0.0, 64, 8, quadrupole=True)
    ao, po = orc.newton_allpairs(x, m, 0.01)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("quad", [False, True])
def test_king_model(pg, orc, quad):
    # the paper's other tree workload: a King model with W0 = 9, whose core
    # packs many particles into finest-level cells
    x, m = gen.king(20000, 90, W0=9.0)
    a, p, t, _ = gpu_tree(pg, x, m, 1e-3, 0.75, 64, 8, quadrupole=quad)
    o = orc.tree_build(x, m, 0.75, 64, 8, quadrupole=quad)
    same_lists(t, o)
    if quad:
        same_pseudo(t, o)
    ao, po = orc.tree_forces(x, m, 1e-3, 0.75, 64, 8, quadrupole=quad)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("quad", [False, True])
def test_tiny_and_degenerate_sets(pg, orc, quad):
    # one particle (no force), two, all coincident (zero extent: the root
    # side falls back to 1 and one finest cell holds every particle), and a
    # huge theta (every node that may be accepted is)
    cases = [(np.array([[0.3, -0.2, 0.1]]), np.array([2.0]), 0.75),
             (np.array([[0.0, 0.0, 0.0], [0.5, 0.25, -0.5]]), np.array([1.0, 3.0]), 0.75),
             (np.tile(np.array([[0.1, 0.2, 0.3]]), (300, 1)), np.full(300, 1.0 / 300), 0.75)]
    x, m = gen.plummer(3000, 91)
    cases.append((x, m, 50.0))
    for x, m, theta in cases:
        a, p, t, _ = gpu_tree(pg, x, m, 0.01, theta, 16, 4, quadrupole=quad)
        o = orc.tree_build(x, m, theta, 16, 4, quadrupole=quad)
        same_lists(t, o)
        ao, po = orc.tree_forces(x, m, 0.01, theta, 16, 4, quadrupole=quad)
        if len(x) == 1 or np.all(x == x[0]):
            # no other particle, or every pair at distance 0: zero force.
            # Every pair term of the potential is the same FP32 value, and
            # within a j tile (512 records) a lane adds its terms in FP32, so
            # the roundings add up instead of cancelling: up to 512 * 2^-24
            # relative
            assert np.all(a == 0) and np.all(ao == 0)
            assert np.allclose(p, po, rtol=512 * 2.0 ** -24, atol=1e-9)
            continue
        assert_parity(rel_vec(a, ao), what="a")
        assert_parity(rel_scalar(p, po), what="phi")


def _sampled_list_forces(x, m, eps, o, idx):
    # FP64 sums over each sampled particle's group list, from the oracle's
    # lists and pseudo-particles (the particle's own entry left out)
    n = len(x)
    perm = o["perm"]
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    xs, ms = x[perm], m[perm]
    acc = np.zeros((len(idx), 3))
    pot = np.zeros(len(idx))
    for s, i0 in enumerate(idx):
        k = inv[i0]
        g = int(np.searchsorted(o["g_i0"], k, side="right") - 1)
        lst = o["jlist"][o["j_off"][g]:o["j_off"][g + 1]]
        lst = lst[lst != k]
        part = lst < n
        pj = np.where(part[:, None], xs[np.minimum(lst, n - 1)], o["pseudo"][np.maximum(lst - n, 0), :3])
        mj = np.where(part, ms[np.minimum(lst, n - 1)], o["pseudo"][np.maximum(lst - n, 0), 3])
        d = pj - xs[k]
        r2 = np.sum(d * d, axis=1) + eps * eps
        rinv = 1.0 / np.sqrt(r2)
        acc[s] = np.sum((mj * rinv ** 3)[:, None] * d, axis=0)
        pot[s] = -np.sum(mj * rinv)
    return acc, pot


@pytest.mark.parametrize("quad", [False, True])
def test_large_tree(pg, orc, quad):
    # 2^22 particles at the bench's settings (theta 0.75, groups of at most
    # 256): every list bit for bit, forces on a sample of particles
    x, m = gen.plummer(1 << 22, 95)
    a, p, t, _ = gpu_tree(pg, x, m, 1e-3, 0.75, 256, 8, quadrupole=quad)
    o = orc.tree_build(x, m, 0.75, 256, 8, quadrupole=quad)
    same_lists(t, o)
    idx = np.random.default_rng(96).choice(len(x), 1000, replace=False)
    ao, po = _sampled_list_forces(x, m, 1e-3, o, idx)
    assert_parity(rel_vec(a[idx], ao), what="a")
    assert_parity(rel_scalar(p[idx], po), what="phi")
