"""Data-parallel Monte-Carlo across ranks (one process per GPU).

Codewords are independent trials (the paper's batch dimension, Sec. III-A),
so ranks draw disjoint Philox codeword ranges and exchange nothing on the
data path. The only collective work is host-side bookkeeping: the sum of
the int64 error counters of a sweep and the maximum of the per-rank step
time, both through ``torch.distributed`` (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

RANK_STRIDE_BITS = 40  # each rank owns codeword indices [rank << 40, (rank + 1) << 40)


def rank_cw_base(rank: int) -> int:
    """First codeword index of a rank's private Philox range (weak scaling: every rank runs its own batches)."""
    if rank < 0 or rank >= (1 << (64 - RANK_STRIDE_BITS)):
        raise ValueError("rank out of range")
    return rank << RANK_STRIDE_BITS


def split_range(total: int, rank: int, world: int, cw0: int = 0) -> tuple[int, int]:
    """Contiguous share [start, start + count) of `total` codewords for `rank` (strong scaling)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad split")
    lo = total * rank // world
    hi = total * (rank + 1) // world
    return cw0 + lo, hi - lo


def sum_counts(counts, group=None):
    """All-reduce (sum) int64 counters [.., 5] in place; returns them."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def max_time(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank time over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
