"""Realization sharding for one process per GPU.

Realization r of an ensemble depends only on the seed and r: the Philox
counters of its grid noise carry the pair index r/2 and those of its nugget
carry r (the noise mapping of Section 2, step 2 and 3, as implemented by the
library).  The set-up (eigenvalues, Kriging weights, the FP64 inverse of the
prediction matrix) is small and replicated on every rank.  So ranks split the
realizations into contiguous, pair-aligned ranges and never exchange data on
the hot path; the only collectives are host-side bookkeeping: the slowest
rank's time, an optional gather of the pieces, and the all-reduce of the
ensemble moments (2 M doubles) when ensemble statistics are wanted.
"""
from __future__ import annotations


def pair_aligned_shard(R_total: int, rank: int, world: int) -> tuple[int, int]:
    """(r_offset, R_local) of `rank` when R_total realizations are split over
    `world` ranks (strong scaling).  Ranks take whole realization pairs (one
    complex FFT gives two realizations), the first (pairs mod world) ranks one
    pair more, so r_offset is even as the C ABI requires; a rank may get 0."""
    if world < 1 or not 0 <= rank < world or R_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, R_total >= 0")
    pairs = (R_total + 1) // 2
    base, extra = divmod(pairs, world)
    p0 = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    r0 = 2 * p0
    return r0, max(0, min(2 * count, R_total - r0))


def weak_offset(R_per_rank: int, rank: int) -> int:
    """r_offset of `rank` when every rank draws its own R_per_rank realizations
    (weak scaling); rounded up to whole pairs so that every offset is even."""
    if R_per_rank < 0 or rank < 0:
        raise ValueError("need R_per_rank >= 0 and rank >= 0")
    return rank * (R_per_rank + R_per_rank % 2)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1 else None


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the whole job's time is the slowest
    rank's); the value itself when no process group of size > 1 is active."""
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_realizations(piece, R_total: int, device=None):
    """Concatenate every rank's (R_local x m x m) piece of a strong-scaling
    split (`pair_aligned_shard`) into the full (R_total x m x m) ensemble on
    every rank.  Pieces are padded to the largest share for the all-gather."""
    import torch
    dist = _dist()
    piece = torch.as_tensor(piece)
    if dist is None:
        return piece
    world = dist.get_world_size()
    shares = [pair_aligned_shard(R_total, k, world)[1] for k in range(world)]
    width = max(shares)
    buf = torch.zeros((width,) + tuple(piece.shape[1:]), dtype=piece.dtype, device=device)
    buf[: piece.shape[0]] = piece.to(device) if device is not None else piece
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return torch.cat([p[:s] for p, s in zip(parts, shares)], dim=0)


def allreduce_moments(sums, count: int):
    """Add every rank's ensemble moments (the (sum, sum of squares) pair of
    ce_ensemble_moments, in place) and its draw count: the one exchange the
    sharded ensemble needs, 2 M doubles.  Returns the total count."""
    import torch
    dist = _dist()
    if dist is None:
        return int(count)
    for t in sums:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    c = torch.tensor([float(count)], dtype=torch.float64, device=sums[0].device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return int(round(c.item()))
