"""Failure detection without a GPU fault: a device-side bounded wait that
nothing completes gives up after its limit, the call reports PG_ETIMEOUT,
and the same context then computes correct forces again."""

import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


def test_bounded_wait_gives_up_and_context_recovers(pg, orc):
    x, m = gen.plummer(1024, 61)
    with pg.Context(0) as c:
        for limit_ms in (1.0, 20.0):
            with pytest.raises(pg.PGError) as e:
                c.selftest_wait(limit_ms)
            assert e.value.code == pg.PG_ETIMEOUT
        c.sync()                      # the status word was cleared
        c.set_eps(1 / 64)
        c.set_self(True)
        a, p = c.forces(x, x, m)
    ao, po = orc.newton_allpairs(x, m, 1 / 64)
    assert_parity(rel_vec(a, ao), what="a")
    assert_parity(rel_scalar(p, po), what="phi")


def test_wait_limit_range(pg):
    with pg.Context(0) as c:
        for bad in (0.0, -1.0, 2001.0):
            with pytest.raises(pg.PGError) as e:
                c.selftest_wait(bad)
            assert e.value.code == pg.PG_EINVAL
