"""Ordinate sharding of the sweep (Sec. 4: the ordinates' sweeps are independent given the
Maxwellian of the current moments; the sum over ordinates in Eq. moments is the one
coupling per Picard iteration).

- ``ordinate_shards``: contiguous ranges of whole values of the outermost velocity index,
  one per part, sizes differing by at most one index value.
- ``sum_fixed_order``: the parts' partial moments summed in part order, the same on every
  part (an allreduce whose result does not depend on the collective's internal order).

Host logic only; the partial moments and the range sweeps are ``Solver.moments_range_device``
and ``Solver.sweep_range``.
"""
from __future__ import annotations


def ordinate_shards(n_points: int, dim: int, parts: int):
    """[(j_begin, j_end)] of each part: the N outer index values split as evenly as possible,
    each carrying its N^(dim-1) ordinates (j lexicographic, last dimension fastest)."""
    if parts < 1 or parts > n_points:
        raise ValueError("parts must be in 1..N")
    inner = n_points ** (dim - 1)
    out = []
    for p in range(parts):
        a = p * n_points // parts
        b = (p + 1) * n_points // parts
        out.append((a * inner, b * inner))
    return out


def sum_fixed_order(partial, group=None):
    """Sum of every rank's tensor `partial` added in rank order 0, 1, ... on every rank
    (all_gather, then a local ordered sum): bitwise the same result on all ranks and for
    any collective algorithm.  Without a process group (one part) it returns `partial`."""
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return partial.clone()
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(bufs, partial.contiguous(), group=group)
    total = bufs[0].clone()
    for b in bufs[1:]:
        total += b
    return total
