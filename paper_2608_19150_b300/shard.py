"""Ordinate sharding of implicit steps (Sec. 4: the ordinates' sweeps are independent given
the Maxwellian of the current moments; the sum over ordinates in Eq. moments is the one
coupling per Picard iteration; Sec. 3.5: the stages of a step run one after another).

- ``ordinate_shards``: contiguous ranges of whole values of the outermost velocity index,
  one per part, sizes differing by at most one index value.
- ``gather_sum``: every process's partial moments, gathered (``all_gather``: NCCL for CUDA
  tensors, gloo for host tensors) and added in rank order by the part's own fixed-order
  sum, so that every process holds the same bits.
- ``sharded_steps``: implicit steps of a problem whose ordinates are split over parts
  (several per process, or one per device): per stage, the Picard loop sweeps every part
  with the summed moments and stops on the measure of Eq. (convergence-criteria).

This module orders calls and collectives only: the stage bookkeeping, the sweeps, the
partial moments, the fixed-order sum and the measure are the parts' own operations (for
``SolverShard`` the library's bgk_shard_* / bgk_sweep_range / bgk_moments_range_device /
bgk_sum_partials_device / bgk_conv_measure_device calls).
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


def _dist_active(group):
    import torch.distributed as dist
    return group is not None or (dist.is_available() and dist.is_initialized())


def gather_sum(local, part, group=None):
    """The sum over all processes of `local` ([node][d+2]), added in rank order 0, 1, ... by
    `part.sum_partials` on the gathered stack: the same bits on every process, for any
    collective algorithm.  `local` is a CUDA tensor with an NCCL group or a host tensor
    with a gloo group.  Without a process group it returns `local`."""
    import torch
    import torch.distributed as dist
    if not _dist_active(group):
        return local
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(bufs, local.contiguous(), group=group)
    return part.sum_partials(torch.stack(bufs))


def sum_fixed_order(partial, group=None):
    """The rank-ordered sum of every process's `partial` with a plain elementwise sum (host
    tensors, tests and tools); the solver path uses gather_sum with the library's sum."""
    import torch
    import torch.distributed as dist
    if not _dist_active(group):
        return partial.clone()
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(bufs, partial.contiguous(), group=group)
    total = bufs[0].clone()
    for b in bufs[1:]:
        total += b
    return total


def _summed(parts, group):
    """Partial moments of this process's parts, summed in part order, then over processes."""
    import torch
    local = []
    for p in parts:
        U = p.new_moments()
        p.partial(U)
        local.append(U)
    U = local[0] if len(local) == 1 else parts[0].sum_partials(torch.stack(local))
    return gather_sum(U, parts[0], group)


def sharded_steps(parts, steps, group=None, l_max=1000):
    """`steps` implicit steps of a problem split over ordinate parts.

    parts: the parts this process holds (objects with step_begin() -> (stages, tol),
    stage_begin(s), stage_end(s), step_end(), new_moments(), partial(U), sweep(U),
    sum_partials(stack) -> U, measure(U_new, U_old) -> float).  group: the process group
    over which the partial moments are summed (None: this process holds every part).
    Every process computes the same measure from the same summed moments, so all stop at
    the same iteration.  Returns the Picard iterations of every stage of every step;
    raises RuntimeError when a stage does not converge within l_max."""
    out = []
    for _ in range(steps):
        shape = [p.step_begin() for p in parts]
        n_stages, tol = shape[0]
        if any(x != shape[0] for x in shape):
            raise RuntimeError("parts disagree on the step's stages")
        its = []
        for st in range(n_stages):
            for p in parts:
                p.stage_begin(st)
            U_old = _summed(parts, group)
            for it in range(1, l_max + 1):
                for p in parts:
                    p.sweep(U_old)
                U_new = _summed(parts, group)
                meas = parts[0].measure(U_new, U_old)
                U_old = U_new
                if meas < tol:
                    break
            else:
                raise RuntimeError("sharded Picard loop did not converge within l_max")
            for p in parts:
                p.stage_end(st)
            its.append(it)
        for p in parts:
            p.step_end()
        out.append(its)
    return out


class SolverShard:
    """Ordinates [j_begin, j_end) of one problem held by a Solver (the whole problem is set
    up on every device; only the part's ordinates are swept and summed).  The Solver should
    run on torch's current stream (Solver(..., stream=torch.cuda.current_stream().cuda_stream))
    so that the gathered moments and the library's work are ordered without host waits."""

    def __init__(self, solver, j_begin, j_end):
        import torch
        self.s, self.jb, self.je = solver, int(j_begin), int(j_end)
        self.shape = (solver.nnode, solver.dim + 2)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.same_stream = getattr(solver, "stream", None) == torch.cuda.current_stream().cuda_stream

    def _order(self):
        # moments made by torch or a collective on torch's stream, read by the library
        if not self.same_stream:
            import torch
            torch.cuda.current_stream().synchronize()

    def new_moments(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def step_begin(self):
        return self.s.shard_step_begin()

    def stage_begin(self, stage):
        self.s.shard_stage_begin(stage)

    def stage_end(self, stage):
        self.s.shard_stage_end(stage)

    def step_end(self):
        self.s.shard_step_end()

    def partial(self, U_out):
        self.s.moments_range_device(self.jb, self.je, U_out.data_ptr())

    def sweep(self, U_in):
        self._order()
        self.s.sweep_range(self.jb, self.je, U_in.data_ptr())

    def sum_partials(self, stack):
        self._order()
        stack = stack.contiguous()
        out = self.new_moments()
        self.s.sum_partials_device(stack.data_ptr(), stack.shape[0], out.data_ptr())
        return out

    def measure(self, U_new, U_old):
        self._order()
        return self.s.conv_measure_device(U_new.data_ptr(), U_old.data_ptr())
