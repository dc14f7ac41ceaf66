"""Parity of the all-pairs Newton path (Eq. 1) with the FP64 oracle, through
the C ABI, on seeded inputs: the 4096-particle Plummer sphere in full, ragged
sizes that span several tiles and leave partial tiles and sub-tiles, every
launch shape, i-sets that differ from the j-set, partial j updates,
eps = 0, translation by 10^3, device pointers, CUDA-graph replay, and the
2^20-particle mixed set on a sampled subset. Tolerances: per-particle
relative error median <= 2e-6 and max <= 1e-4 for a and phi."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def run_allpairs(pg, x, m, eps, shape=None, graph=False, reps=1):
    with pg.Context(0) as c:
        c.set_eps(eps)
        c.set_self(True)
        if shape:
            c.set_shape(*shape)
        c.set_graph(graph)
        c.set_j(x, m)
        c.set_i(x)
        for _ in range(reps):
            c.run()
        return c.get_force(len(x))


def test_plummer_4096_full(pg, orc):
    x, m = gen.plummer(4096, gen.CONFIG_SEEDS[1])
    eps = 1 / 64
    a, p = run_allpairs(pg, x, m, eps)
    ao, po = orc.newton_allpairs(x, m, eps)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


@pytest.mark.parametrize("n", [1, 2, 255, 1537, 5000])
@pytest.mark.parametrize("shape", [(1, 0, 1), (2, 0, 1), (4, 0, 1), (2, 1, 1),
                                   (1, 0, 0), (2, 0, 0), (4, 0, 0)])
def test_ragged_sizes_and_shapes(pg, orc, n, shape):
    x, m = gen.plummer(n, 700 + n)
    m = m * np.exp(np.random.default_rng(n).uniform(-2, 2, n))
    eps = 0.05
    a, p = run_allpairs(pg, x, m, eps, shape=shape)
    ao, po = orc.newton_allpairs(x, m, eps)
    if n == 1:
        assert np.all(a == 0) and np.all(p == 0)
        return
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_sorted_path_mid_size(pg, orc):
    # >= 16384 i-particles: the Morton ordering of i-tiles is used
    x, m = gen.plummer_cube_mix(20000, 77)
    eps = 1e-3
    a, p = run_allpairs(pg, x, m, eps)
    idx = gen.sample_indices(len(x), 2000, 5)
    ao, po = orc.newton_subset(x, m, eps, idx)
    assert_parity(rel_vec(a[idx], ao), what="a")
    assert_parity(rel_scalar(p[idx], po), what="phi")


@pytest.mark.parametrize("ni,nj", [(700, 3001), (1, 100), (3000, 1), (513, 257)])
def test_probes_against_other_set(pg, orc, ni, nj):
    xj, mj = gen.plummer(nj, 900 + nj)
    xi = gen.plummer(ni, 901 + ni)[0] * 1.3
    eps = 0.02
    with pg.Context(0) as c:
        c.set_eps(eps)
        a, p = c.forces(xi, xj, mj)
    ao, po = orc.newton(xi, xj, mj, eps)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_partial_j_updates_and_set_n(pg, orc):
    x, m = gen.plummer(3000, 31)
    eps = 1 / 64
    with pg.Context(0) as c:
        c.set_eps(eps)
        c.set_j(x[:1000], m[:1000], adr=0)
        c.set_j(x[1000:], m[1000:], adr=1000)
        c.set_n(2500)
        a, p = c.forces(x[:50])
    ao, po = orc.newton(x[:50], x[:2500], m[:2500], eps, skip=np.arange(50))
    # without the self mode the own pair's potential -m/eps is included
    po_raw = po - m[:50] / eps
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po_raw), what="phi")


def test_eps_zero_leaves_coincident_pair_out(pg, orc):
    # unsoftened close pairs of an unordered set: the double-float
    # differences keep them at the usual tolerances
    x, m = gen.plummer(2000, 41)
    a, p = run_allpairs(pg, x, m, 0.0)
    ao, po = orc.newton_allpairs(x, m, 0.0)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_translation_by_1e3(pg, orc):
    x, m = gen.plummer(4096, gen.CONFIG_SEEDS[1])
    eps = 1 / 64
    a, p = run_allpairs(pg, x + np.array([1e3, -1e3, 5e2]), m, eps)
    ao, po = orc.newton_allpairs(x, m, eps)
    assert_parity(rel_vec(a, ao), what="a (shifted)")
    assert_parity(rel_scalar(p, po), what="phi (shifted)")


def test_device_path_matches_host_path(pg):
    torch = pytest.importorskip("torch")
    x, m = gen.plummer(3333, 51)
    a_h, p_h = run_allpairs(pg, x, m, 1 / 64)
    xd = torch.tensor(x, device="cuda")
    md = torch.tensor(m, device="cuda")
    ad = torch.empty_like(xd)
    pd = torch.empty_like(md)
    with pg.Context(0) as c:
        c.set_stream(torch.cuda.current_stream().cuda_stream)
        c.set_eps(1 / 64)
        c.set_self(True)
        c.set_j_dev(xd, md)
        c.set_i_dev(xd)
        c.run_dev(ad, pd)
        c.sync()
    assert np.array_equal(ad.cpu().numpy(), a_h) and np.array_equal(pd.cpu().numpy(), p_h)


def test_graph_replay_and_determinism(pg):
    x, m = gen.plummer(20000, 61)
    a1, p1 = run_allpairs(pg, x, m, 1 / 64)
    a2, p2 = run_allpairs(pg, x, m, 1 / 64, graph=True, reps=3)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


def test_empty_inputs(pg):
    with pg.Context(0) as c:
        c.set_eps(0.1)
        x, m = gen.plummer(10, 1)
        c.set_j(x, m)
        c.set_i(np.zeros((0, 3)))
        c.run()
        a, p = c.get_force(0)
        assert a.shape == (0, 3)
    with pg.Context(0) as c:
        c.set_eps(0.1)
        c.set_i(x)
        c.run()                      # no j: zero force
        a, p = c.get_force(10)
        assert np.all(a == 0) and np.all(p == 0)


def test_errors_are_reported(pg):
    with pg.Context(0) as c:
        with pytest.raises(pg.PGError) as e:
            c.run()
        assert e.value.code == pg.PG_ESTATE
        with pytest.raises(pg.PGError) as e:
            c.set_eps(-1.0)
        assert e.value.code == pg.PG_EINVAL
        c.set_mode(pg.PG_TABLE)
        c.set_i(np.zeros((3, 3)))
        with pytest.raises(pg.PGError) as e:
            c.run()
        assert e.value.code == pg.PG_ESTATE
        with pytest.raises(pg.PGError) as e:
            c.set_table_values(np.zeros(8, np.float32), 1.0, 9, 9)
        assert e.value.code == pg.PG_EINVAL
        c.set_mode(pg.PG_NEWTON)
        c.set_self(True)
        with pytest.raises(pg.PGError) as e:
            c.run()                  # self mode with ni > nj
        assert e.value.code == pg.PG_ESTATE


def test_mixed_2e20_sampled(pg, orc):
    """The 2^20-particle Plummer + cube set in the launch configuration the
    benchmark times, checked on a 4096-particle sample."""
    x, m = gen.plummer_cube_mix(1 << 20, gen.CONFIG_SEEDS[2])
    eps = 1e-3
    a, p = run_allpairs(pg, x, m, eps)
    idx = gen.sample_indices(len(x), 4096, gen.CONFIG_SEEDS[2] + 1)
    ao, po = orc.newton_subset(x, m, eps, idx)
    assert_parity(rel_vec(a[idx], ao), what="a")
    assert_parity(rel_scalar(p[idx], po), what="phi")


def test_pinned_host_buffers():
    # page-locked inputs and outputs go by DMA straight to and from the
    # caller's memory; the results are those of the pageable path, bit for bit
    torch = pytest.importorskip("torch")
    pg = need_cuda()
    x, m = gen.plummer(3000, 7401)
    xi = x[:1700]

    def pinned(arr):
        return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()

    with pg.Context(0) as c:
        c.set_eps(1 / 64)
        c.set_j(x, m)
        c.set_i(xi)
        c.run()
        a0, p0 = c.get_force(len(xi))
        xh, mh, xih = pinned(x), pinned(m), pinned(xi)
        ah, ph = pinned(np.zeros((len(xi), 3))), pinned(np.zeros(len(xi)))
        c.set_j(xh, mh)
        c.set_i(xih)
        xh[:] = 0.0                      # the calls copied before returning
        xih[:] = 0.0
        c.run()
        a1, p1 = c.get_force(len(xi), out=(ah, ph))
        assert a1 is ah and p1 is ph
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
