"""The entry point that allocates nothing (for callers whose memory pool
holds the whole GPU, or whose time-critical loop must not stall on
cudaMalloc) gives the same forces as the context path, on two calls in a
row with different inputs, and refuses sizes beyond its fixed scratch.
Collected last so that a failure here does not hide the other tests."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_path_on_two_calls():
    pg = need_cuda()
    torch = pytest.importorskip("torch")
    st = torch.cuda.current_stream()
    for seed, n, eps in ((11, 5000, 1 / 64), (12, pg.PG_NOALLOC_MAX_N, 0.02)):
        x, m = gen.plummer(n, seed)
        xd = torch.tensor(x, device="cuda")
        md = torch.tensor(m, device="cuda")
        a = torch.full_like(xd, float("nan"))
        p = torch.full_like(md, float("nan"))
        pg.pg_newton_allpairs_noalloc(xd, md, n, eps, a, p, st.cuda_stream)
        a2 = torch.empty_like(xd)
        p2 = torch.empty_like(md)
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(eps)
            c.set_self(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xd)
            c.run_dev(a2, p2)
            c.sync()
        a, p, a2, p2 = (t.cpu().numpy() for t in (a, p, a2, p2))
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
        assert_parity(rel_vec(a, a2), what=f"a (n={n})")
        assert_parity(rel_scalar(p, p2), what=f"phi (n={n})")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pg = need_cuda()
    torch = pytest.importorskip("torch")
    n = pg.PG_NOALLOC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    m = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.pg_newton_allpairs_noalloc(x, m, n, 0.1, x, None, None)
    assert e.value.code == pg.PG_EINVAL
