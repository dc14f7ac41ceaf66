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
