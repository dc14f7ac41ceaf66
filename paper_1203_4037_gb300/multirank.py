"""Host logic of the work split across ranks (one process per GPU).

Forces on different i-particles are independent (the paper splits the
i-loop over cores with OpenMP, Section 3.5), so each rank owns a contiguous
slice of the particles and computes the forces on its slice. In a run the
positions change every step and each rank updates only its own, so every
force evaluation starts with the path's exchange: one all-gather of every
rank's packed j records (x, y, z, m), after which each rank evaluates its
slice against all of them, its own pairs left out through the self mode with
an offset (its slice starts at j record rank * per). The job's time is the
slowest rank's; results, when wanted on one rank, are gathered once at the
end.

The particle-mesh long range has one real exchange when the particles
themselves are split: every mesh point takes mass from every rank's
particles, so the ranks' density meshes are summed (one all-reduce of N^3
values) before each rank solves for its own particles.
"""

from __future__ import annotations


def shard(n: int, rank: int, world: int):
    """Contiguous i-range [lo, hi) of `rank` among `world` ranks (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return (n * rank) // world, (n * (rank + 1)) // world


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks of the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, n: int, device=None):
    """Concatenate each rank's rows (its shard of n) in rank order on every rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    world = dist.get_world_size()
    sizes = [shard(n, r, world) for r in range(world)]
    width = local.shape[1:] if local.dim() > 1 else ()
    parts = [torch.empty((hi - lo, *width), dtype=local.dtype, device=device) for lo, hi in sizes]
    pad = max(hi - lo for lo, hi in sizes)
    buf = torch.zeros((pad, *width), dtype=local.dtype, device=device)
    buf[:local.shape[0]] = local
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf)
    for r, (lo, hi) in enumerate(sizes):
        parts[r] = outs[r][:hi - lo]
    return torch.cat(parts)


def padded_shard(n: int, world: int) -> int:
    """Records per rank in the all-gathered j buffer: the largest shard. A
    rank with a shorter shard pads it with massless records, which add
    nothing to any force (m = 0 at a finite position)."""
    return max(hi - lo for lo, hi in (shard(n, r, world) for r in range(world))) if world > 0 else 0


def pack_records(x, m, per, out):
    """This rank's records into out (per, 4): x, y, z, m, then massless
    padding at the first particle's position (or the origin)."""
    k = x.shape[0]
    out[:k, :3] = x
    out[:k, 3] = m
    if k < per:
        out[k:, :3] = x[0] if k > 0 else 0.0
        out[k:, 3] = 0.0
    return out


class ShardedAllPairs:
    """All-pairs forces of this rank's slice of the particles, each call
    starting from this rank's current positions and masses: pack the slice's
    records, all-gather every rank's (NCCL on GPUs; the path's one exchange),
    load them as the j-set, and evaluate the slice with its own pairs left out.

    ctx: a pg Context on this rank's GPU; all_gather_into_tensor(out, inp):
    the collective (torch.distributed's, or a stand-in)."""

    def __init__(self, ctx, n, rank, world, all_gather_into_tensor, device=None):
        import torch
        self.ctx, self.n, self.rank, self.world = ctx, n, rank, world
        self.lo, self.hi = shard(n, rank, world)
        self.per = padded_shard(n, world)
        self.gather = all_gather_into_tensor
        self.local = torch.zeros((self.per, 4), dtype=torch.float64, device=device)
        self.all = torch.empty((self.per * world, 4), dtype=torch.float64, device=device)
        ctx.set_self_offset(rank * self.per)

    def exchange(self, x, m):
        """x (ni, 3), m (ni,): this rank's slice. After it, every rank's
        records sit in self.all, rank r's at [r per, r per + size_r)."""
        pack_records(x, m, self.per, self.local)
        self.gather(self.all, self.local)
        return self.all

    def forces(self, x, m, acc, pot=None):
        """Exchange, then this slice's acceleration (ni, 3) and potential
        (ni,) into acc, pot (device tensors)."""
        self.exchange(x, m)
        self.ctx.set_j_rec_dev(self.all)
        self.ctx.set_n(self.per * self.world)
        self.ctx.set_i_dev(x)
        self.ctx.run_dev(acc, pot)
        return acc, pot


def mesh_forces_sharded(deposit, solve, all_reduce, x, m):
    """Mesh forces of this rank's particles x, m: deposit(x, m) gives this
    rank's density mesh, all_reduce sums the meshes of all ranks in place,
    and solve(mesh, x) gives the acceleration and potential at x."""
    rho = deposit(x, m)
    all_reduce(rho)
    return solve(rho, x)
