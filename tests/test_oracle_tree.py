"""Pins of the tree oracle (the grouped Barnes-Hut tree of Section 5.1,
monopole moments): against the direct sum, the mathematics of the tree, and
hand-built cases.

- theta = 0 opens every node, so the lists are all particles and the forces
  are the direct sum.
- The groups partition the particles, and each level's nodes partition them
  too.
- Node moments sum to the system's mass and first moment.
- The error against the direct sum shrinks with theta. At the paper's 0.75
  it stays at the monopole level.
- A far symmetric cluster acts as one particle at its centre of mass.
"""

import numpy as np
import pytest

import gen


def test_theta_zero_is_the_direct_sum(orc):
    x, m = gen.plummer(1500, 11)
    m = m * np.exp(np.random.default_rng(1).uniform(-1, 1, len(m)))
    a, p = orc.tree_forces(x, m, 0.01, 0.0, 40, 6)
    ad, pd = orc.newton_allpairs(x, m, 0.01)
    assert np.allclose(a, ad, rtol=1e-12, atol=1e-14 * np.abs(ad).max())
    assert np.allclose(p, pd, rtol=1e-12, atol=0)
    t = orc.tree_build(x, m, 0.0, 40, 6)
    for g in range(len(t["g_i0"])):
        lst = t["jlist"][t["j_off"][g]:t["j_off"][g + 1]]
        assert np.array_equal(np.sort(lst), np.arange(len(x)))     # every particle once


def test_groups_partition_and_moments(orc):
    x, m = gen.clustered_box(3000, 12, nclump=10, sigma=0.02, periodic=False)
    m = m * np.random.default_rng(2).uniform(0.5, 2.0, len(m))
    ncrit = 50
    t = orc.tree_build(x, m, 0.6, ncrit, 8)
    i0, ni = t["g_i0"], t["g_ni"]
    assert i0[0] == 0 and np.all(i0[1:] == i0[:-1] + ni[:-1]) and i0[-1] + ni[-1] == len(x)
    assert np.array_equal(np.sort(t["perm"]), np.arange(len(x)))
    # the root is node 0: all the mass and the system's first moment
    assert t["nM"][0] == pytest.approx(m.sum(), rel=1e-14)
    assert t["nS"][0] == pytest.approx((m[:, None] * x).sum(axis=0), rel=1e-13)
    # groups hold at most ncrit particles unless they are finest-level nodes
    big = ni > ncrit
    assert np.all(t["g_node"][big] >= 0)
    # every list holds the group's own particles (their nodes contain the box)
    for g in range(0, len(i0), 7):
        lst = t["jlist"][t["j_off"][g]:t["j_off"][g + 1]]
        own = np.arange(i0[g], i0[g] + ni[g])
        assert np.all(np.isin(own, lst))


def test_error_shrinks_with_theta(orc):
    x, m = gen.plummer(3000, 13)
    ad, pd = orc.newton_allpairs(x, m, 0.01)
    med = []
    for th in (0.3, 0.5, 0.75):
        a, p = orc.tree_forces(x, m, 0.01, th, 64, 8)
        rel = np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)
        med.append(np.median(rel))
        assert np.median(np.abs(p - pd) / np.abs(pd)) < 1e-3
    assert med[0] < med[1] < med[2]
    assert med[0] < 5e-4 and med[2] < 1e-2          # monopole accuracy at theta 0.75


def test_far_symmetric_cluster_is_one_particle(orc):
    # four unit masses at c + (+-h, +-h, 0) in one corner (total 4, centre of
    # mass c exactly) and a probe pair at the other; with a generous theta the
    # probes' group sees the far cluster as one node
    c = np.array([0.75, 0.75, 0.5])
    h = 1.0 / 64.0
    far = np.array([c + [h, h, 0], c + [-h, h, 0], c + [h, -h, 0], c + [-h, -h, 0]])
    near = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.0 / 512.0]])
    x = np.concatenate([near, far])
    m = np.array([1e-3, 1e-3, 1.0, 1.0, 1.0, 1.0])
    t = orc.tree_build(x, m, 2.0, 2, 1)
    a, p = orc.tree_forces(x, m, 0.0, 2.0, 2, 1)
    # probe 0: the other probe at d = (0, 0, 1/512) plus 4 at c
    d = c - near[0]
    r = np.linalg.norm(d)
    want = 4.0 * d / r ** 3 + 1e-3 * np.array([0, 0, 1.0]) / (1.0 / 512.0) ** 2
    assert a[0] == pytest.approx(want, rel=1e-12)
    assert p[0] == pytest.approx(-4.0 / r - 1e-3 * 512.0, rel=1e-12)
    g = int(np.flatnonzero(t["g_i0"] == 0)[0])
    lst = t["jlist"][t["j_off"][g]:t["j_off"][g + 1]]
    assert np.count_nonzero(lst >= len(x)) == 1       # one pseudo-particle


def test_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.tree_build(np.zeros((0, 3)), np.zeros(0), 0.5, 8, 4)
    with pytest.raises(ValueError):
        orc.tree_build(np.zeros((3, 3)), np.ones(3), -0.1, 8, 4)


def test_opening_decision_at_the_threshold(orc):
    # a probe at the origin and a 4-particle cluster centred at c, alone in
    # its level-1 octant of side span / 2: the level-1 node is accepted
    # exactly when span / 2 < theta |c|; just below that, its level-2 child
    # (side span / 4, the same centre) is accepted instead
    h = 1.0 / 64.0
    c = np.array([0.75, 0.75, 0.5])
    x = np.array([[0.0, 0.0, 0.0], c + [h, h, 0], c + [-h, h, 0], c + [h, -h, 0], c + [-h, -h, 0]])
    m = np.ones(5)
    span = 0.75 + h
    theta_star = (span / 2) / np.linalg.norm(c)
    for theta, level in ((theta_star * 1.02, 1), (theta_star * 0.98, 2)):
        t = orc.tree_build(x, m, theta, 1, 1)
        probe = int(np.flatnonzero(t["perm"] == 0)[0])
        g = int(np.flatnonzero(t["g_i0"] == probe)[0])
        lst = t["jlist"][t["j_off"][g]:t["j_off"][g + 1]]
        nodes = lst[lst >= len(x)] - len(x)
        assert len(nodes) == 1 and t["nlevel"][nodes[0]] == level
        assert t["nS"][nodes[0]] / t["nM"][nodes[0]] == pytest.approx(c, abs=1e-15)


def test_lists_are_breadth_first(orc):
    # every list runs level by level and in key order within a level: its
    # node entries rise in (level, index); a list holds each particle or
    # node once
    x, m = gen.plummer(4000, 14)
    n = len(x)
    t = orc.tree_build(x, m, 0.6, 48, 6)
    lev = t["nlevel"]
    for g in range(0, len(t["g_i0"]), 5):
        lst = t["jlist"][t["j_off"][g]:t["j_off"][g + 1]]
        assert len(np.unique(lst)) == len(lst)
        nodes = lst[lst >= n] - n
        assert len(np.unique(lev[nodes])) >= 2
        key = lev[nodes].astype(np.int64) * (1 << 40) + nodes
        assert np.all(np.diff(key) > 0)


def test_quadrupole_pseudo_particles_carry_the_moments(orc):
    # each node's three pseudo-particles have its mass, a zero dipole about
    # its centre of mass and second moment T - l3 I (T and its smallest
    # eigenvalue l3 computed here from the node's particles), so the same
    # trace-free quadrupole; the first lies along the principal axis of the
    # largest eigenvalue, on the side where that axis' largest component is
    # positive; a one-particle node's three sit on the particle
    x, m = gen.clustered_box(2500, 15, nclump=8, sigma=0.03, periodic=False)
    m = m * np.random.default_rng(5).uniform(0.5, 2.0, len(m))
    t = orc.tree_build(x, m, 0.7, 40, 6, quadrupole=True)
    assert t["npseudo"] == 3
    xs, ms = x[t["perm"]], m[t["perm"]]
    ps = t["pseudo"].reshape(-1, 3, 4)
    nn = len(t["nM"])
    singles = spread = 0
    for k in range(0, nn, 3):
        f, c_ = t["nfirst"][k], t["ncount"][k]
        y, w = xs[f:f + c_], ms[f:f + c_]
        M = w.sum()
        com = (w[:, None] * y).sum(axis=0) / M
        T = np.einsum("i,ia,ib->ab", w, y - com, y - com)
        scale = max(np.trace(T), 1e-300)
        assert np.allclose(t["nT"][k], T[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], rtol=1e-9,
                           atol=1e-12 * scale)
        lam, V = np.linalg.eigh(T)
        p, pm = ps[k, :, :3], ps[k, :, 3]
        # positions round to the coordinates' ulp: spreads below it are lost
        ulp = 4.0 * np.spacing(np.abs(com).max())
        assert pm.sum() == pytest.approx(M, rel=1e-14) and np.all(pm == pm[0])
        assert np.allclose((pm[:, None] * (p - com)).sum(axis=0), 0.0,
                           atol=1e-12 * np.sqrt(scale * M) + M * ulp)
        Tp = np.einsum("q,qa,qb->ab", pm, p - com, p - com)
        assert np.allclose(Tp, T - lam[0] * np.eye(3), rtol=1e-9,
                           atol=1e-10 * scale + M * ulp * (ulp + np.sqrt(scale / M)))
        alpha = np.sqrt(2.0 * max(lam[2] - lam[0], 0.0) / M)
        if lam[2] - lam[1] > 1e-6 * scale and lam[2] - lam[0] > 1e-3 * scale and alpha > 1e6 * ulp:
            spread += 1
            d0 = p[0] - com
            e1 = V[:, 2] * np.sign(V[np.argmax(np.abs(V[:, 2])), 2])
            assert np.allclose(d0 / np.linalg.norm(d0), e1, atol=1e-8)
        if c_ == 1:
            singles += 1
            assert np.allclose(p, y[0], rtol=0, atol=1e-15 * np.abs(y[0]).max())
    assert singles > 0 and spread > 100


def _far_error(pos, mass, src, msrc, d, dirs):
    pts = d * dirs
    exact = -np.sum(msrc[None, :] / np.linalg.norm(pts[:, None, :] - src[None], axis=2), axis=1)
    approx = -np.sum(mass[None, :] / np.linalg.norm(pts[:, None, :] - pos[None], axis=2), axis=1)
    return np.mean(np.abs(approx - exact))


def test_quadrupole_far_field_order(orc):
    # a lopsided cluster of size ~0.1 seen from distance d: the potential
    # error of the monopole falls as d^-3 (the quadrupole term is missing),
    # that of the four pseudo-particles as d^-4 (the octupole term)
    rng = np.random.default_rng(16)
    src = rng.normal(size=(300, 3)) * [0.05, 0.03, 0.02] + [0.02, 0.0, 0.0] * rng.random((300, 1))
    msrc = rng.uniform(0.5, 1.5, 300)
    dirs = rng.normal(size=(128, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    errs = {}
    for quad in (False, True):
        t = orc.tree_build(src, msrc, 0.5, 1000, 1000, quadrupole=quad)
        root = t["pseudo"][:t["npseudo"]]       # node 0 holds every particle
        c = (msrc[:, None] * src).sum(axis=0) / msrc.sum()
        assert np.allclose(root[:, :3].mean(axis=0), c, atol=1e-15)
        errs[quad] = [_far_error(root[:, :3] - c, root[:, 3], src - c, msrc, d, dirs)
                      for d in (4.0, 8.0)]
    mono, quad = errs[False], errs[True]
    assert 6.0 < mono[0] / mono[1] < 10.5           # 2^3
    assert 12.0 < quad[0] / quad[1] < 21.0          # 2^4
    assert quad[0] < 0.1 * mono[0]


def test_quadrupole_tree_is_more_accurate(orc):
    # against the direct sum, the quadrupole pseudo-particles cut the force
    # error of the monopole tree several fold at the same lists' nodes
    x, m = gen.plummer(3000, 17)
    ad, pd = orc.newton_allpairs(x, m, 0.01)
    for theta, gain in ((0.5, 0.35), (0.75, 0.55)):
        med = {}
        for quad in (False, True):
            a, p = orc.tree_forces(x, m, 0.01, theta, 64, 8, quadrupole=quad)
            med[quad] = np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1))
        assert med[True] < gain * med[False]
    a, p = orc.tree_forces(x, m, 0.01, 0.0, 64, 8, quadrupole=True)     # theta 0: direct
    assert np.allclose(a, ad, rtol=1e-12, atol=1e-14 * np.abs(ad).max())
