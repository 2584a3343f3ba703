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


def moment_change(U_new, U_old, dim):
    """The Picard convergence measure of Eq. (convergence-criteria) on summed moments
    [node][d+2]: the largest of the relative l2 changes of n, n u (relative to
    max(|n u|, |n|)) and E."""
    import torch
    n = torch.linalg.vector_norm
    dU = U_new - U_old
    m0 = n(dU[:, 0]) / n(U_old[:, 0])
    m1 = n(dU[:, 1:1 + dim]) / torch.maximum(n(U_old[:, 1:1 + dim]), n(U_old[:, 0]))
    m2 = n(dU[:, -1]) / n(U_old[:, -1])
    return float(torch.max(torch.stack([m0, m1, m2])))


def picard_sharded(parts, allreduce, dim, tol, l_max):
    """One backward-Euler stage's Picard loop (Sec. 4) over ordinate shards.

    parts: the shards this process holds, each an object with
      partial(U_out)  -- its partial moments (sum over its ordinates) into U_out,
      sweep(U_in)     -- one sweep of its ordinates with the summed moments U_in,
      commit()        -- make the converged state the base of the next step.
    allreduce(U): the sum over all processes of U, the same bits on every process (e.g.
    sum_fixed_order; identity when this process holds every shard).
    Every process computes the same measure from the same summed moments, so all of them
    stop at the same iteration.  Returns the iteration count; raises RuntimeError if the
    loop does not converge within l_max."""
    def summed():
        local = None
        for p in parts:
            U = p.new_moments()
            p.partial(U)
            local = U if local is None else local + U
        return allreduce(local)
    U_old = summed()
    for it in range(1, l_max + 1):
        for p in parts:
            p.sweep(U_old)
        U_new = summed()
        meas = moment_change(U_new, U_old, dim)
        U_old = U_new
        if meas < tol:
            for p in parts:
                p.commit()
            return it
    raise RuntimeError("sharded Picard loop did not converge within l_max")


class SolverShard:
    """A shard of ordinates [j_begin, j_end) of one problem held by a Solver (the whole
    problem is set up on every device; only the shard's ordinates are swept and summed)."""

    def __init__(self, solver, j_begin, j_end):
        import torch
        self.s, self.jb, self.je = solver, int(j_begin), int(j_end)
        self.shape = (solver.nnode, solver.dim + 2)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._f = None

    def new_moments(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def partial(self, U_out):
        self.s.moments_range_device(self.jb, self.je, U_out.data_ptr())

    def sweep(self, U_in):
        # U_in may come from torch kernels (the sum of the partials) on torch's stream; the
        # library works on its own stream, so wait for them first
        import torch
        torch.cuda.current_stream().synchronize()
        self.s.sweep_range(self.jb, self.je, U_in.data_ptr())

    def commit(self):
        # f^{k+1} becomes the stage base f^k of the next step (bgk_set_f_device copies f
        # into both the state and the base)
        import torch
        import numpy as np
        if self._f is None:
            dt = torch.float64 if self.s.fdtype == np.float64 else torch.float32
            self._f = torch.empty((self.s.nv, self.s.nnode), dtype=dt, device=self.device)
        self.s.get_f_device(self._f.data_ptr(), self.s.fdtype)
        self.s.set_f_device(self._f.data_ptr(), self.s.fdtype)


def sharded_be_steps(parts, allreduce, dim, nu, dt, tau, steps, l_max=1000):
    """`steps` backward-Euler steps of a sharded problem; returns the iteration counts.
    The tolerance is the single-device one, tau / max(1, nu dt)."""
    tol = tau / max(1.0, nu * dt)
    return [picard_sharded(parts, allreduce, dim, tol, l_max) for _ in range(steps)]
