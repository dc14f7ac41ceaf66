"""The i-range split of the multi-GPU path, on CPU with two gloo ranks: each
rank computes its shard (the FP64 oracle stands in for the GPU call), the
gathered result equals the single-rank one, and the job time is the slowest
rank's."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1203_4037_gb300.multirank import gather_rows, max_over_ranks, shard


def test_shard_covers_range_exactly():
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            ranges = [shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import gen
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, m = gen.plummer(1001, 17)
    lo, hi = shard(len(x), rank, world)
    a, p = oracle.newton(x[lo:hi], x, m, 0.05, skip=np.arange(lo, hi), nthreads_=1)
    full = gather_rows(torch.tensor(np.concatenate([a, p[:, None]], axis=1)), len(x))
    t = max_over_ranks(1.0 + rank)
    if rank == 0:
        np.save(out, full.numpy())
        np.save(out + ".t.npy", np.array([t]))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one(tmp_path, orc):
    import gen
    out = str(tmp_path / "full.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    full = np.load(out)
    x, m = gen.plummer(1001, 17)
    a, p = orc.newton_allpairs(x, m, 0.05)
    assert np.array_equal(full[:, :3], a) and np.array_equal(full[:, 3], p)
    assert np.load(out + ".t.npy")[0] == 2.0


def _pm_worker(rank, world, port, out):
    # the particle-mesh long range with the particles split across ranks:
    # each deposits its shard, the density meshes are summed (the one real
    # exchange), each solves for its own particles; the FP64 mesh oracle
    # stands in for the GPU steps
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import gen
    from oracle import pm
    from paper_1203_4037_gb300.multirank import mesh_forces_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, m = gen.clustered_box(3001, 31, nclump=10, sigma=0.02)
    lo, hi = shard(len(x), rank, world)
    N, rs = 32, 1.25 / 32

    def deposit(xl, ml):
        return torch.from_numpy(pm.deposit(xl, ml, 1.0, N).ravel().copy())

    def solve(rho, xl):
        return pm.solve(rho.numpy().reshape(N, N, N), xl, 1.0, N, "gauss", rs)

    a, p = mesh_forces_sharded(deposit, solve, dist.all_reduce, x[lo:hi], m[lo:hi])
    full = gather_rows(torch.tensor(np.concatenate([a, p[:, None]], axis=1)), len(x))
    if rank == 0:
        np.save(out, full.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_mesh_matches_one_rank(tmp_path, world):
    import gen
    from oracle import pm
    out = str(tmp_path / "pm.npy")
    mp.spawn(_pm_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    full = np.load(out)
    x, m = gen.clustered_box(3001, 31, nclump=10, sigma=0.02)
    a, p = pm.mesh_forces(x, m, 1.0, 32, "gauss", 1.25 / 32)
    # only the order of the mesh sums differs
    assert np.allclose(full[:, :3], a, rtol=1e-10, atol=1e-12 * np.abs(a).max())
    assert np.allclose(full[:, 3], p, rtol=1e-10, atol=1e-12 * np.abs(p).max())


class OracleContext:
    """Stands in for a GPU context in the sharded all-pairs driver: keeps the
    records, the offset and the i-particles it is given and evaluates them
    with the FP64 oracle (i-particle k leaves out j record offset + k)."""

    def __init__(self, eps):
        self.eps, self.off, self.nj = eps, None, None

    def set_self_offset(self, lo):
        self.off = lo

    def set_j_rec_dev(self, rec):
        self.rec = rec.numpy().copy()

    def set_n(self, nj):
        self.nj = nj

    def set_i_dev(self, x):
        self.xi = x.numpy().copy()

    def run_dev(self, acc, pot):
        import oracle
        rec = self.rec[:self.nj]
        skip = self.off + np.arange(len(self.xi), dtype=np.int64)
        assert np.array_equal(rec[skip, :3], self.xi)       # the slice sits at the offset
        a, p = oracle.newton(self.xi, rec[:, :3], rec[:, 3], self.eps, skip=skip, nthreads_=1)
        acc.copy_(torch.from_numpy(a))
        pot.copy_(torch.from_numpy(p))


def _sharded_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import gen
    from paper_1203_4037_gb300.multirank import ShardedAllPairs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 1003                       # shards of unequal size: the short ones are padded
    x, m = gen.plummer(n, 19)
    lo, hi = shard(n, rank, world)
    drv = ShardedAllPairs(OracleContext(0.03), n, rank, world, dist.all_gather_into_tensor)
    xi, mi = torch.tensor(x[lo:hi]), torch.tensor(m[lo:hi])
    acc = torch.empty((hi - lo, 3), dtype=torch.float64)
    pot = torch.empty(hi - lo, dtype=torch.float64)
    # a second step with moved particles: the exchange carries every rank's
    # current positions
    drv.forces(xi, mi, acc, pot)
    xi2 = xi + 0.01 * (rank + 1)
    drv.forces(xi2, mi, acc, pot)
    full = gather_rows(torch.cat([acc, pot[:, None]], dim=1), n)
    if rank == 0:
        np.save(out, full.numpy())
        np.save(out + ".rec.npy", drv.all.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_allpairs_exchange_matches_one_rank(tmp_path, orc, world):
    import gen
    from paper_1203_4037_gb300.multirank import padded_shard
    out = str(tmp_path / "sh.npy")
    mp.spawn(_sharded_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    full = np.load(out)
    n = 1003
    x, m = gen.plummer(n, 19)
    # the second step's positions: rank r moved its slice by 0.01 (r + 1)
    for r in range(world):
        lo, hi = shard(n, r, world)
        x[lo:hi] += 0.01 * (r + 1)
    a, p = orc.newton_allpairs(x, m, 0.03)
    assert np.allclose(full[:, :3], a, rtol=0, atol=1e-13 * np.abs(a).max())
    assert np.allclose(full[:, 3], p, rtol=1e-13)
    # the gathered records: rank order, padded shards massless
    rec = np.load(out + ".rec.npy")
    per = padded_shard(n, world)
    assert rec.shape == (per * world, 4)
    for r in range(world):
        lo, hi = shard(n, r, world)
        assert np.array_equal(rec[r * per:r * per + hi - lo, :3], x[lo:hi])
        assert np.all(rec[r * per + hi - lo:(r + 1) * per, 3] == 0.0)


def test_padded_records_are_massless():
    from paper_1203_4037_gb300.multirank import pack_records, padded_shard
    assert padded_shard(10, 3) == 4 and padded_shard(9, 3) == 3
    x = torch.arange(9, dtype=torch.float64).reshape(3, 3)
    out = torch.full((5, 4), float("nan"), dtype=torch.float64)
    pack_records(x, torch.ones(3, dtype=torch.float64), 5, out)
    assert torch.all(out[:3, :3] == x) and torch.all(out[:3, 3] == 1)
    assert torch.all(out[3:, 3] == 0) and torch.all(torch.isfinite(out))
