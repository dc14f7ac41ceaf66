"""The entry point that allocates nothing (for callers whose memory pool
holds the whole GPU, or whose time-critical loop must not stall on
cudaMalloc) gives the same forces as the context path, on two calls in a
row with different inputs, matches the FP64 oracle, and refuses sizes beyond
its fixed scratch. Sizes from one particle to the largest accepted, eps = 0
(a coincident pair contributes nothing) and eps > 0, with and without the
potential output. Collected last so that a failure here does not hide the
other tests."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


def noalloc(pg, torch, x, m, eps, want_phi, stream):
    n = len(x)
    xd = torch.tensor(x, device="cuda")
    md = torch.tensor(m, device="cuda")
    a = torch.full_like(xd, float("nan"))
    p = torch.full_like(md, float("nan")) if want_phi else None
    pg.pg_newton_allpairs_noalloc(xd, md, n, eps, a, p, stream.cuda_stream)
    stream.synchronize()
    return a.cpu().numpy(), (p.cpu().numpy() if want_phi else None)


def context(pg, x, m, eps):
    with pg.Context(0) as c:
        c.set_eps(eps)
        c.set_self(True)
        c.set_j(x, m)
        c.set_i(x)
        c.run()
        return c.get_force(len(x))


def test_noalloc_matches_context_path_on_two_calls():
    pg = need_cuda()
    torch = pytest.importorskip("torch")
    st = torch.cuda.current_stream()
    for seed, n, eps in ((11, 5000, 1 / 64), (12, pg.PG_NOALLOC_MAX_N, 0.02)):
        x, m = gen.plummer(n, seed)
        a, p = noalloc(pg, torch, x, m, eps, True, st)
        a2, p2 = context(pg, x, m, eps)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
        assert_parity(rel_vec(a, a2), what=f"a (n={n})")
        assert_parity(rel_scalar(p, p2), what=f"phi (n={n})")


@pytest.mark.parametrize("want_phi", [True, False])
@pytest.mark.parametrize("eps", [0.0, 1 / 64])
@pytest.mark.parametrize("n", [1, 2, 513, 5000, 16384])
def test_noalloc_against_oracle_and_context(orc, n, eps, want_phi):
    pg = need_cuda()
    torch = pytest.importorskip("torch")
    st = torch.cuda.current_stream()
    x, m = gen.plummer(n, 3000 + n)
    a, p = noalloc(pg, torch, x, m, eps, want_phi, st)
    assert np.all(np.isfinite(a))
    if n == 1:            # no other particle: no force, no potential
        assert np.all(a == 0.0)
        if want_phi:
            assert p[0] == 0.0
        return
    ao, po = orc.newton_allpairs(x, m, eps)
    assert_parity(rel_vec(a, ao), what=f"a vs oracle (n={n}, eps={eps})")
    a2, p2 = context(pg, x, m, eps)
    assert_parity(rel_vec(a, a2), what=f"a vs context (n={n}, eps={eps})")
    if want_phi:
        if n == 2 and eps > 0:
            # each particle's own pair adds m/eps = 32 to its FP32 sum before
            # the FP64 removal, 64 times its potential: the result carries the
            # rounding of that sum, a few 2^-24 of m/eps + |phi|
            bound = 8 * 2.0 ** -24 * (m / eps + np.abs(po))
            assert np.all(np.abs(p - po) <= bound) and np.all(np.abs(p - p2) <= bound)
            return
        assert_parity(rel_scalar(p, po), what=f"phi vs oracle (n={n}, eps={eps})")
        assert_parity(rel_scalar(p, p2), what=f"phi vs context (n={n}, eps={eps})")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pg = need_cuda()
    torch = pytest.importorskip("torch")
    n = pg.PG_NOALLOC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    m = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.pg_newton_allpairs_noalloc(x, m, n, 0.1, x, None, None)
    assert e.value.code == pg.PG_EINVAL
