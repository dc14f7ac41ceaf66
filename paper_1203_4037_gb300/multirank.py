"""Host logic of the i-range split across ranks (one process per GPU).

Forces on different i-particles are independent, so ranks take contiguous
i-ranges against the full j-set and exchange nothing on the data path. The
job's time is the slowest rank's; results, when wanted on one rank, are
gathered once at the end.
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
