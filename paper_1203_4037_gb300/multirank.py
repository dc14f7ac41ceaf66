"""Host logic of the work split across ranks (one process per GPU).

Forces on different i-particles are independent, so ranks take contiguous
i-ranges against the full j-set and exchange nothing on the data path. The
job's time is the slowest rank's; results, when wanted on one rank, are
gathered once at the end.

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


def mesh_forces_sharded(deposit, solve, all_reduce, x, m):
    """Mesh forces of this rank's particles x, m: deposit(x, m) gives this
    rank's density mesh, all_reduce sums the meshes of all ranks in place,
    and solve(mesh, x) gives the acceleration and potential at x."""
    rho = deposit(x, m)
    all_reduce(rho)
    return solve(rho, x)
