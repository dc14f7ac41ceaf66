"""The device side of the particles-split-across-ranks path on one GPU: the
self mode with an offset (i-particle k is j-particle lo + k) against the FP64
oracle, on the tiled and narrow paths, and the sharded driver for ranks
emulated one after another on the same GPU (the all-gather done by
concatenating each emulated rank's packed records, no kernel waits on
another), which must give the single-rank all-pairs forces."""

import numpy as np
import pytest

import gen
from pgtest import assert_parity, need_cuda, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    return need_cuda()


# the tiled cases above the Morton threshold take single offsets (sorted,
# dense i-sets) at the softening of the 4096-body workload, and the
# double-float form at eps = 1e-3; the narrow path is double-float anyway
@pytest.mark.parametrize("path,n,lo,hi,eps,diff", [
    ("tiled", 30000, 10000, 30000, 1 / 64, 0),
    ("tiled", 30000, 10000, 30000, 1e-3, 2),
    ("tiled", 40000, 5000, 25000, 1 / 64, 0),
    ("tiled", 12000, 3000, 9000, 1e-3, 0),
    ("narrow", 50000, 777, 1777, 1e-3, 0)])
def test_self_offset(pg, orc, path, n, lo, hi, eps, diff):
    x, m = gen.plummer_cube_mix(n, 4545)
    with pg.Context(0) as c:
        c.set_allpairs_path(pg.PG_PATH_TILED if path == "tiled" else pg.PG_PATH_NARROW)
        c.set_differencing(diff)
        c.set_eps(eps)
        c.set_self_offset(lo)
        c.set_j(x, m)
        c.set_i(x[lo:hi])
        c.run()
        a, p = c.get_force(hi - lo)
    ao, po = orc.newton(x[lo:hi], x, m, eps, skip=np.arange(lo, hi, dtype=np.int64))
    assert_parity(rel_vec(a, ao), what=f"a {path} offset {lo}")
    assert_parity(rel_scalar(p, po), what=f"phi {path} offset {lo}")


def test_self_offset_bounds(pg):
    x, m = gen.plummer(1000, 3)
    with pg.Context(0) as c:
        c.set_j(x, m)
        c.set_i(x[:500])
        c.set_self_offset(501)           # 501 + 500 > 1000
        with pytest.raises(pg.PGError) as e:
            c.run()
        assert e.value.code == pg.PG_ESTATE
        with pytest.raises(pg.PGError) as e:
            c.set_self_offset(-1)
        assert e.value.code == pg.PG_EINVAL


@pytest.mark.parametrize("world", [1, 3])
def test_sharded_driver_emulated_ranks(pg, orc, world):
    torch = pytest.importorskip("torch")
    from paper_1203_4037_gb300.multirank import ShardedAllPairs, padded_shard, shard
    n, eps = 20001, 1e-3
    x, m = gen.plummer_cube_mix(n, 4646)
    o = gen.morton_order(x)
    x, m = x[o], m[o]
    per = padded_shard(n, world)
    # every emulated rank's packed records, concatenated in rank order: what
    # the all-gather would leave on each rank
    locals_ = []
    drivers = []
    ctxs = [pg.Context(0) for _ in range(world)]
    for r in range(world):
        lo, hi = shard(n, r, world)
        ctxs[r].set_eps(eps)
        drivers.append(ShardedAllPairs(ctxs[r], n, r, world, None, device="cuda"))
        xi = torch.tensor(x[lo:hi], device="cuda")
        mi = torch.tensor(m[lo:hi], device="cuda")
        locals_.append((xi, mi))
    from paper_1203_4037_gb300.multirank import pack_records
    gathered = torch.cat([pack_records(xi, mi, per, torch.zeros((per, 4), dtype=torch.float64,
                                                                  device="cuda"))
                          for xi, mi in locals_])

    def fake_gather(out, inp):
        out.copy_(gathered)

    a_all, p_all = [], []
    for r in range(world):
        drivers[r].gather = fake_gather
        xi, mi = locals_[r]
        acc = torch.empty((xi.shape[0], 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(xi.shape[0], dtype=torch.float64, device="cuda")
        drivers[r].forces(xi, mi, acc, pot)
        torch.cuda.synchronize()
        a_all.append(acc.cpu().numpy())
        p_all.append(pot.cpu().numpy())
    for c in ctxs:
        c.close()
    a, p = np.concatenate(a_all), np.concatenate(p_all)
    idx = gen.sample_indices(n, 3000, 47)
    ao, po = orc.newton_subset(x, m, eps, idx)
    assert_parity(rel_vec(a[idx], ao), what=f"a world {world}")
    assert_parity(rel_scalar(p[idx], po), what=f"phi world {world}")
