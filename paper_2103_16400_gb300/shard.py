"""Sharding of independent NTT work across ranks (one process per GPU).

Every RNS limb of a polynomial is a separate ring Z_q[X]/(X^N+1) and every
polynomial is transformed on its own (Section 2, RNS representation; the
batched NTT of Section 3), so the hot path splits into (polynomial, limb)
units with no exchange between them.  Ranks therefore share nothing on the
data path: each takes its own units, runs them on its own GPU with its own
copy of the twiddle tables for the primes it touches, and only the timing
(max over ranks) and, where a caller wants it, a gather of outputs cross
process boundaries.

All functions here are pure host logic; `max_over_ranks` works with any
initialised torch.distributed process group (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple


def unit_range(n_units: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) slice of n_units for `rank`; sizes differ by at most one
    and the slices of ranks 0..world-1 tile [0, n_units) in order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if n_units < 0:
        raise ValueError("n_units must be non-negative")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def poly_limb_units(n_polys: int, n_limbs: int, world: int, rank: int) -> List[Tuple[int, int]]:
    """The (poly, limb) pairs `rank` owns when a [n_polys][n_limbs][N] batch is
    split into n_polys * n_limbs units in row-major order."""
    lo, hi = unit_range(n_polys * n_limbs, world, rank)
    return [divmod(u, n_limbs) for u in range(lo, hi)]


def transform_cost(N: int, n_limbs: int) -> int:
    """Butterfly count of the forward (or inverse) transform of one ragged item:
    N/2 log2 N per limb."""
    if N < 2 or N & (N - 1):
        raise ValueError(f"N={N} is not a power of two")
    return (N // 2) * (N.bit_length() - 1) * n_limbs


def assign_items(costs: Sequence[int], world: int) -> List[List[int]]:
    """Split ragged items over ranks by cost: longest item first, each to the
    rank with the least work so far (ties to the lower rank).  Deterministic;
    every item lands on exactly one rank; each rank's list is in item order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for lst in out:
        lst.sort()
    return out


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s inputs under weak scaling: each rank transforms its
    own independent batch of the same shape."""
    return base + 0x10000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
