"""The roofline microbenchmark returns plausible ceilings on the device:
FP32 FMA lane rates near 128 per SM per clock, MUFU rsqrt near 16, the
Newton pair term in registers between the MUFU and FP32 bounds, random
8-byte shared-memory gathers below the conflict-free 16 per SM per clock
(from one table or four interleaved copies), and the same gathers through
the read-only global path below the shared ones."""

import pytest

from pgtest import need_cuda

pytestmark = pytest.mark.gpu


def test_microbench_ceilings():
    pg = need_cuda()
    ffma, _ = pg.pg_microbench(0)
    ffma2, _ = pg.pg_microbench(1)
    mufu, _ = pg.pg_microbench(2)
    mix, mix_s = pg.pg_microbench(3)
    # per SM per clock at the device's maximum clock (the run may clock lower)
    assert 32 < ffma < 140 and 32 < ffma2 < 140
    assert 4 < mufu < 20
    assert 2 < mix < 11 and mix_s > 1e11
    gather, _ = pg.pg_microbench(4)
    assert 1 < gather <= 16.5
    copies, _ = pg.pg_microbench(5)
    assert 1 < copies <= 16.5
    glob, _ = pg.pg_microbench(6)
    assert 0 < glob < gather
    with pytest.raises(pg.PGError):
        pg.pg_microbench(7)
