"""Host-side helpers for runs on several GPUs of one node (one process per GPU).

Lattices are independent, so several GPUs only ever run separate lattices: a batch or
a request stream is dealt out round-robin, and a benchmark runs one replica per rank
(seed offset by rank).  There is no data-path collective; the only communication is
the end-of-run reduction of the timing (maximum over ranks) and of the work done (sum).
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(seed: int, rank: int) -> int:
    """Seed of `rank`'s replica: the rank in bits 48..63, the seed below them, so that
    distinct (seed, rank) pairs never share a random stream (seed < 2^48, rank < 2^16)."""
    seed, rank = int(seed), int(rank)
    if not (0 <= seed < (1 << 48) and 0 <= rank < (1 << 16)):
        raise ValueError("replica seeds need 0 <= seed < 2^48 and 0 <= rank < 2^16")
    return (rank << 48) | seed


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (every item goes to exactly one rank)."""
    return list(items)[rank::world]


def reduce_run(elapsed_s: float, work: float, device=None) -> tuple[float, float]:
    """(max elapsed over ranks, total work over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(work)
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
