"""i-sets spread over the whole system at eps = 1e-3, on every all-pairs path
whose i-tiles are not compact: the narrow path (few i against many j), the
tiled path below the Morton threshold, and the entry point that allocates
nothing. Positions are FP64 (the inputs of Section 4.1) and the pair loop
runs in FP32; these paths form each pair difference in double-float, so the
per-particle error stays within the Newton tolerances (median 2e-6, max
1e-4 against the FP64 oracle) however far apart the i-particles that share a
tile are.

Two kinds of spread set: i drawn from the Plummer sphere itself, and i
placed at 0.5 to 2 eps from randomly chosen j-particles all over the
system, so that every i has a pair whose term dominates its force at a
distance of the order of eps. The second is the hard case for one FP32
offset per particle (its difference error is about 2^-24 of the tile's
extent): the negative control shows that the single form fails it."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu

EPS = 1e-3


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


@pytest.fixture(scope="module")
def jset():
    return gen.plummer_cube_mix(50000, 4242)


def near_j(xj, ni, seed, eps=EPS):
    """ni positions at 0.5 eps to 2 eps from distinct random j-particles."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(xj), size=ni, replace=False)
    u = rng.normal(size=(ni, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return xj[idx] + u * (eps * rng.uniform(0.5, 2.0, ni))[:, None]


def drawn(ni, seed):
    """ni positions drawn from the Plummer sphere (the whole sphere)."""
    return gen.plummer(ni, seed)[0]


def run(pg, xi, xj, mj, path, diff=None, eps=EPS):
    with pg.Context(0) as c:
        c.set_allpairs_path(path)
        if diff is not None:
            c.set_differencing(diff)
        c.set_eps(eps)
        c.set_j(xj, mj)
        c.set_i(xi)
        c.run()
        a, p = c.get_force(len(xi))
        return a, p, c.info()


@pytest.mark.parametrize("kind", ["near_j", "drawn"])
@pytest.mark.parametrize("ni", [16, 64, 512, 1000])
def test_narrow_spread_i(pg, orc, jset, ni, kind):
    xj, mj = jset
    xi = near_j(xj, ni, 700 + ni) if kind == "near_j" else drawn(ni, 700 + ni)
    a, p, info = run(pg, xi, xj, mj, pg.PG_PATH_NARROW)
    assert info["df"] == 1 and info["slots"] > 1
    ao, po = orc.newton(xi, xj, mj, EPS)
    assert_parity(rel_vec(a, ao), what=f"a narrow {kind} {ni}")
    assert_parity(rel_scalar(p, po), what=f"phi narrow {kind} {ni}")


@pytest.mark.parametrize("kind", ["near_j", "drawn"])
@pytest.mark.parametrize("ni", [5000, 16000])
def test_tiled_spread_i(pg, orc, jset, ni, kind):
    xj, mj = jset
    xi = near_j(xj, ni, 800 + ni) if kind == "near_j" else drawn(ni, 800 + ni)
    a, p, info = run(pg, xi, xj, mj, pg.PG_PATH_TILED)
    assert info["df"] == 1
    ao, po = orc.newton(xi, xj, mj, EPS)
    assert_parity(rel_vec(a, ao), what=f"a tiled {kind} {ni}")
    assert_parity(rel_scalar(p, po), what=f"phi tiled {kind} {ni}")


def test_tiled_forced_double_on_sorted_tiles(pg, orc, jset):
    # above the Morton threshold the automatic choice keeps the single form
    # for dense i-sets; the double form can be asked for and agrees
    xj, mj = jset
    xi = near_j(xj, 20000, 901)
    a, p, info = run(pg, xi, xj, mj, pg.PG_PATH_TILED, diff=pg.PG_DIFF_DOUBLE)
    assert info["df"] == 1
    ao, po = orc.newton(xi, xj, mj, EPS)
    assert_parity(rel_vec(a, ao), what="a tiled 20000 forced double")
    assert_parity(rel_scalar(p, po), what="phi tiled 20000 forced double")


@pytest.mark.parametrize("path", ["narrow", "tiled"])
def test_single_offsets_fail_the_hard_case(pg, orc, jset, path):
    # negative control: one FP32 offset per particle from a spread tile's
    # centre misses the max tolerance on the near-j set, so the sets above
    # do test the differencing
    xj, mj = jset
    ni = 512 if path == "narrow" else 5000
    xi = near_j(xj, ni, 700 + ni if path == "narrow" else 800 + ni)
    a, _, info = run(pg, xi, xj, mj, pg.PG_PATH_NARROW if path == "narrow" else pg.PG_PATH_TILED,
                     diff=pg.PG_DIFF_SINGLE)
    assert info["df"] == 0
    ao, _ = orc.newton(xi, xj, mj, EPS)
    assert rel_vec(a, ao).max() > 1e-4


def test_noalloc_spread(pg, orc):
    torch = pytest.importorskip("torch")
    # 8192 particles of the mixed set and a partner of each at 0.5 to 2 eps:
    # every particle has a close pair, and the caller's order is random
    xh, mh = gen.plummer_cube_mix(8192, 4343)
    xp = near_j(xh, 8192, 4344)
    x = np.concatenate([xh, xp])
    m = np.concatenate([mh, mh]) / 2
    perm = np.random.default_rng(4345).permutation(len(x))
    x, m = x[perm], m[perm]
    n = len(x)
    assert n == pg.PG_NOALLOC_MAX_N
    xd = torch.tensor(x, device="cuda")
    md = torch.tensor(m, device="cuda")
    a = torch.empty_like(xd)
    p = torch.empty_like(md)
    st = torch.cuda.current_stream()
    pg.pg_newton_allpairs_noalloc(xd, md, n, EPS, a, p, st.cuda_stream)
    st.synchronize()
    ao, po = orc.newton_allpairs(x, m, EPS)
    assert_parity(rel_vec(a.cpu().numpy(), ao), what="a noalloc spread")
    assert_parity(rel_scalar(p.cpu().numpy(), po), what="phi noalloc spread")
