"""Host logic of the multi-GPU (one process per GPU) form: env shards and
the timing reduction.  Envs are independent and every random draw is keyed by
the global env index, so rank r of `world` simply owns the contiguous global
env range [r*n, (r+1)*n) (weak scaling: n envs per rank) and the data path
needs no collective.  The only exchange is the benchmark's max-over-ranks
time, done once per run."""
from __future__ import annotations


def env_base(rank: int, n_envs_per_rank: int) -> int:
    """First global env index of `rank`'s shard."""
    if rank < 0 or n_envs_per_rank < 1:
        raise ValueError("bad shard")
    return rank * n_envs_per_rank


def split_range(n_envs: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous near-equal split of a fixed batch (strong scaling form)."""
    if not 0 <= rank < world:
        raise ValueError("rank outside world")
    return rank * n_envs // world, (rank + 1) * n_envs // world


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / max_seconds
