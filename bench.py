"""Benchmark of the implicit sweep solver on B300: DOF-updates/s of whole implicit steps.

A step is one implicit time step of the 2D-2V shock tube (128 x 128 squares, 32,768 P2
triangles, 32 x 32 velocities, 3-stage DIRK, Knudsen 1e-3): every stage runs Picard
iterations (Maxwellian + source, transport sweep, moments, convergence test) until the
moment criterion meets 1e-8.  value = DOF x sweeps / time over the timed steps.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded sample
of the same workload.  Under torchrun every rank runs an independent replica (the solver
runs on one GPU; replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sweep DOF-updates/s; time per implicit step to 1e-8 residual vs plain FP64"
UNIT = "DOF-updates/s"
WALL_NOTE = ("; wall faces read as inflow data in the sampled sweep (the mirror rows are not in the sample; "
             "a wall read costs the same per face)")
# Sec. 4.2 wall sets for the single-problem workloads (sides without an entry: inflow)
WALL_SETS = {"none": None,
             "channel": {"y-": "reflect", "y+": "reflect"},
             "closed_reflect": {sd: "reflect" for sd in ("x-", "x+", "y-", "y+", "z-", "z+")},
             "closed_bounce_back": {sd: "bounce_back" for sd in ("x-", "x+", "y-", "y+", "z-", "z+")}}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed"])
    p.add_argument("--n-side", type=int, default=None,
                   help="cells per side (shock_tube 128, bump3d 24, learned 256)")
    p.add_argument("--n-v", type=int, default=None, help="velocity points per dimension (32; bump3d 16)")
    p.add_argument("--sweep-reps", type=int, default=5)
    p.add_argument("--workload", default="shock_tube", choices=["shock_tube", "p1_square", "bump3d", "strip", "sod", "sod2d", "batched",
                                                         "learned"])
    p.add_argument("--nu", type=float, default=1000.0, help="sod: collision frequency (the paper runs 1 and 1000)")
    p.add_argument("--integrator", default="DIRK2", choices=["BE", "DIRK2"], help="sod: DIRK-1 or DIRK-2")
    p.add_argument("--sweep-mode", default="auto", choices=["auto", "tgs", "ts"],
                   help="sweep algorithm: generation sweep (tgs), one thread per ordinate (ts), or automatic")
    p.add_argument("--walls", default="none", choices=sorted(WALL_SETS),
                   help="Sec. 4.2 walls: channel = reflecting walls at y = 0, 1 (single-problem workloads)")
    p.add_argument("--collision", default="maxwellian", choices=["maxwellian", "linear"],
                   help="linear: the simplified Maxwellian n/|V| (single-problem workloads)")
    p.add_argument("--train-runs", type=int, default=200)
    p.add_argument("--eval-runs", type=int, default=4)
    p.add_argument("--instances", type=int, default=64)
    p.add_argument("--no-guess", action="store_true", help="batched: without the learned guess")
    p.add_argument("--no-compare", action="store_true", help="batched: skip the plain FP64 batch")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cache", default="auto", choices=["auto", "on", "off"],
                   help="local-inverse cache of the sweep")
    p.add_argument("--stage-predictor", action="store_true",
                   help="start each DIRK stage after the first from moments extrapolated across the stage "
                        "abscissae (both arms; off: the previous stage's moments, the paper's iteration)")
    p.add_argument("--eager", action="store_true",
                   help="launch each step's kernels from a host loop instead of one CUDA graph (profiling)")
    a = p.parse_args()
    if a.n_side is None:
        a.n_side = {"bump3d": 24, "learned": 256, "strip": 4096, "sod": 256, "sod2d": 160,
                    "p1_square": 16}.get(a.workload, 128)
    if a.n_v is None and a.workload in ("sod2d", "p1_square"):
        a.n_v = 16
    if a.n_v is None:
        a.n_v = 16 if a.workload == "bump3d" else 32
    return a


def workload(args):
    from paper_2608_19150_b300 import synth
    if args.workload == "p1_square":
        return synth.workload_p1_square(n_side=args.n_side, seed=0, n_v=args.n_v, k_v=3, L=6.0, knudsen=1e-2,
                                        integrator="BE", cfl=10.0)
    if args.workload == "bump3d":
        return synth.workload_3d_bump(n_side=args.n_side, seed=2, n_v=args.n_v, k_v=3, L=6.0, knudsen=1e-2,
                                      integrator="BE", cfl=8.0)
    if args.workload == "sod2d":
        return synth.workload_sod_2d(n=args.n_side, n_v=args.n_v, k_v=3, L=6.0, knudsen=1.0 / args.nu,
                                     integrator=args.integrator, cfl=7.0)
    if args.workload == "sod":
        return synth.workload_sod_strip(nx=args.n_side, ny=6, n_v=args.n_v, k_v=3, L=6.0, knudsen=1.0 / args.nu,
                                        integrator=args.integrator, dt=1.76e-3, quads=True)
    if args.workload == "strip":
        return synth.workload_strip(nx=args.n_side, ny=2, seed=5, kx=1, n_v=args.n_v, k_v=3, L=6.0, knudsen=1e-2,
                                    integrator="BE", cfl=10.0)
    return synth.workload_shock_tube(n_side=args.n_side, seed=1, kx=2, n_v=args.n_v, k_v=3, L=8.0, knudsen=1e-3,
                                     integrator="DIRK3", cfl=10.0)


def elem_of(w):
    """(name of the element tables, dofs per cell, velocity dimension) of a workload."""
    if w.mesh.dim == 3:
        return "p1tet", 4, 3
    if w.mesh.cells.shape[1] == 4:
        return "q1quad", 4, 2
    return ("p2tri", 6, 2) if w.kx == 2 else ("p1tri", 3, 2)


L2_BYTES = 126 * 2 ** 20           # B300 L2


def l2_note(f_bytes):
    if f_bytes > 2 * L2_BYTES:
        return "inputs larger than L2 (f %.2f GB per array)" % (f_bytes / 1e9)
    return "L2 flushed before every timed step (a 504 MiB buffer written outside the timed region; f %.1f MB)" % (
        f_bytes / 1e6)


def l2_flusher(f_bytes):
    """A callable that evicts L2 by writing a buffer four times its size, or None when the
    step's arrays are larger than L2 themselves."""
    if f_bytes > 2 * L2_BYTES:
        return None
    import torch
    buf = torch.empty(4 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush():
        buf.fill_(1.0)
    return flush


def config(w, args, extra=None):
    _, nd, dv = elem_of(w)
    dof = int(w.mesh.n_cells * nd * args.n_v ** dv)
    if w.mesh.dim == 3:
        name = ("3D-3V Gaussian bump, %d^3 cubes (%d P1 tetrahedra), %d^3 velocities on [-6,6]^3, backward Euler, "
                "Kn 1e-2, CFL 8, tau 1e-8" % (args.n_side, w.mesh.n_cells, args.n_v))
        integ = "BE"
    elif args.workload == "p1_square":
        name = ("2D-2V smooth problem, %dx%d squares (%d P1 triangles), %dx%d velocities on [-6,6]^2, backward Euler, "
                "Kn 1e-2, CFL 10, tau 1e-8" % (args.n_side, args.n_side, w.mesh.n_cells, args.n_v, args.n_v))
        integ = "BE"
    elif args.workload == "sod2d":
        name = ("2D-2V Sod problem, X = [0,2]^2, disc of radius 0.4, %dx%d Q1 squares, %dx%d velocities on [-6,6]^2, "
                "%s, nu %g, dt 7x explicit, tau 1e-8" % (args.n_side, args.n_side, args.n_v, args.n_v, args.integrator,
                                                         args.nu))
        integ = args.integrator
    elif args.workload == "sod":
        name = ("2D-2V Sod problem in a strip [-1,1]x[-3/128,3/128], %dx6 Q1 quadrilaterals (%d cells), reflecting "
                "walls at x2 = +-3/128, %dx%d velocities on [-6,6]^2, %s, nu %g, dt 1.76e-3, tau 1e-8"
                % (args.n_side, w.mesh.n_cells, args.n_v, args.n_v, args.integrator, args.nu))
        integ = args.integrator
    elif args.workload == "strip":
        name = ("2D-2V smooth quasi-1D problem on a %dx2 strip (%d P1 triangles), %dx%d velocities on [-6,6]^2, "
                "backward Euler, Kn 1e-2, CFL 10, tau 1e-8" % (args.n_side, w.mesh.n_cells, args.n_v, args.n_v))
        integ = "BE"
    else:
        name = ("2D-2V shock tube, %dx%d squares (%d P2 triangles), %dx%d velocities on [-8,8]^2, DIRK3, "
                "Kn 1e-3, CFL 10, tau 1e-8" % (args.n_side, args.n_side, w.mesh.n_cells, args.n_v, args.n_v))
        integ = "DIRK3"
    if getattr(args, "collision", "maxwellian") == "linear":
        name += ", simplified Maxwellian n/|V|"
    if getattr(args, "walls", "none") != "none":
        name += ", walls: " + ", ".join("%s %s" % kv for kv in sorted(WALL_SETS[args.walls].items())
                                        if kv[0][0] in "xyz"[:w.mesh.dim])
    c = {"workload": name,
         "n_cells": w.mesh.n_cells, "dof_per_sweep": dof,
         "precision": {"fp64": "FP64 sweeps", "fp32": "FP32 sweeps, FP64-accurate moments",
                       "mixed": "FP32 sweeps to the FP32 floor, then FP64 sweeps; FP64 moments"}[args.precision],
         "integrator": integ,
         "l2": l2_note(dof * (4 if args.precision == "fp32" else 8)),
         "parallelism": "replicas", "launch": "eager host loop" if args.eager else
         "one CUDA graph per step, conditional while-node per stage", "sweep_mode": args.sweep_mode}
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------- flop count
def sweep_flops_per_item(cached, kind="p2tri"):
    """Floating-point operations of one local solve, counted from the generated reference
    tables (multiply and add each count one) with the average face mix of the simplex: half
    the faces outflow, half inflow.  cached: right-hand side plus one matrix-vector product
    with the stored inverse."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2608_19150_b300", "csrc"))
    import gen_tables as gt
    d, nd, nf, Mh, Dd, Eh, fn = gt.tables(kind)
    half = nf / 2.0
    fl = 0.0
    fl += nf * (2 * d - 1 + 2)                     # s_i = v . N_i, |s_i| * (1/|K|)
    if cached:
        fl += sum(2 * sum(1 for b in range(nd) if Mh[a][b] != 0) - 1 for a in range(nd))
        fl += half * sum(2 * sum(1 for k in range(len(fn[0])) if Eh[0][a][fn[0][k]] != 0) + 1
                         for a in range(nd) if any(Eh[0][a][fn[0][k]] != 0 for k in range(len(fn[0]))))
        return fl + nd * (2 * nd - 1)
    for a in range(nd):
        for b in range(nd):
            t = (Mh[a][b] != 0) + sum(Dd[i][a][b] != 0 for i in range(nf))
            fl += max(0, 2 * t - 1)
    nnzE = sum(1 for a in range(nd) for b in range(nd) if Eh[0][a][b] != 0)
    fl += half * 2 * nnzE                          # outflow face terms
    fl += sum(2 * sum(1 for b in range(nd) if Mh[a][b] != 0) - 1 for a in range(nd))
    fl += half * sum(2 * sum(1 for k in range(len(fn[0])) if Eh[0][a][fn[0][k]] != 0) + 1
                     for a in range(nd) if any(Eh[0][a][fn[0][k]] != 0 for k in range(len(fn[0]))))
    for k in range(nd):                            # LU without pivoting + substitution
        fl += 1 + (nd - k - 1) * (1 + 2 * (nd - k - 1) + 2)
    for i in range(nd):
        fl += 2 * (nd - i - 1) + 1
    return fl


# --------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- CPU oracle
def host_cpu():
    """(logical cores this process may use, CPU model name) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


def _oracle_sweep_rate(w, js, dt, omp):
    """DOF-updates/s of one oracle sweep over the ordinates js of the full mesh (the
    first-stage coefficient, f^l = M = f of the initial state), and the seconds it took."""
    from oracle.oracle import Oracle, tableau
    # the sampled sweep reads wall faces as inflow data (the mirror rows are not sampled)
    o = Oracle(w.mesh.dim, w.kx, w.mesh.xyz, w.mesh.cells, w.n_v, w.k_v, w.L, omp=omp)
    o.build_dags_for(js)
    f0 = o.maxwellian_rows(w.init, js)
    fbc = o.maxwellian_rows(w.inflow, js)
    A, _, _ = tableau(w.integrator)
    nus = w.nu + 1.0 / (dt * A[0, 0])
    t0 = time.perf_counter()
    o.sweep_rows(js, f0, f0, f0 / (dt * A[0, 0]), fbc, w.nu, nus)
    el = time.perf_counter() - t0
    return len(js) * o.nnode / el, el, o.nv, len(js) * o.nnode


def _sample_ordinates(nv, n_ord):
    n_ord = min(n_ord, nv)
    j0 = (nv - n_ord) // 2
    return np.arange(j0, j0 + n_ord, dtype=np.int32)


def cpu_baseline(w, n_ord, dt):
    """The oracle as it stands on the host: one sweep over n_ord ordinates of the full mesh
    with the loop over ordinates on all cores (the OpenMP build of the same source), and a
    quarter of that sample on one core (the sequential parity build)."""
    cores, model = host_cpu()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    nv = w.n_v ** w.mesh.dim
    js = _sample_ordinates(nv, n_ord)
    v_all, el_all, nv, dof_all = _oracle_sweep_rate(w, js, dt, omp=True)
    js1 = _sample_ordinates(nv, max(1, len(js) // 4))
    v_one, el_one, _, dof_one = _oracle_sweep_rate(w, js1, dt, omp=False)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "sample": "one sweep over %d of %d ordinates of the full mesh (%d DOF) in %.2f s, OpenMP loop over "
                      "ordinates on %d threads" % (len(js), nv, dof_all, el_all, cores),
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": "one sweep over %d ordinates (%d DOF) in %.2f s, sequential build"
                                        % (len(js1), dof_one, el_one)}}


# --------------------------------------------------------------------- runs
def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units, elapsed_max, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return sum_over_ranks(float(units), world) / elapsed_max


def run_reference(args):
    """The reference arm: the CPU oracle as it stands (the OpenMP build, all host cores),
    each step one oracle sweep over a bounded sample of the workload's ordinates (rank 0
    only)."""
    rank, world, _ = dist_init(args)
    if rank != 0:
        return
    w = workload(args)
    cores, model = host_cpu()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    from oracle.oracle import Oracle, tableau
    o = Oracle(w.mesh.dim, w.kx, w.mesh.xyz, w.mesh.cells, w.n_v, w.k_v, w.L, omp=True)   # see cpu_baseline
    js = _sample_ordinates(o.nv, 16 * cores)
    n_ord = len(js)
    o.build_dags_for(js)
    dt = w.dt if w.dt > 0 else w.cfl * o.dt_explicit()
    f0 = o.maxwellian_rows(w.init, js)
    fbc = o.maxwellian_rows(w.inflow, js)
    A, _, _ = tableau(w.integrator)
    nus = w.nu + 1.0 / (dt * A[0, 0])
    for _ in range(max(0, args.warmup)):
        o.sweep_rows(js[:cores], f0[:cores], f0[:cores], f0[:cores] / (dt * A[0, 0]), fbc[:cores], w.nu, nus)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.sweep_rows(js, f0, f0, f0 / (dt * A[0, 0]), fbc, w.nu, nus)
    el = time.perf_counter() - t0
    dof = n_ord * o.nnode * args.steps
    v = dof / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config(w, args, {"sample": "each step: one oracle sweep over %d of %d ordinates of the "
                                                 "full mesh" % (n_ord, o.nv), "precision": "FP64 CPU oracle"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
                             "sample": "%d ordinates x %d cells x %d nodes per step, OpenMP loop over ordinates "
                                       "on %d threads%s" % (
                                           n_ord, o.ncell, o.nnode // o.ncell, cores,
                                           WALL_NOTE if (args.walls != "none" or w.walls) else "")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def launches_per_step(st, guess=False, main_fp32=False, walls=False, refine=False, bdf2=False, mixed=False,
                      projected=True):
    """Kernels one step launches (graph nodes of kernel type), from its statistics.  FP32
    sweeps form their source themselves (factors, sweep, moments, test per iteration);
    FP64 iterations add the source pass; walls add their refresh to every iteration.  The
    mixed precision's FP32 phase: state reset, stage begin, moment copy, record, the
    hand-over moment pass and its fallback, plus the conversions of f and q that the
    stage-start moment pass and the stage combine do not already write (with a guess
    changing f first).  refine: the FP64 iterations after the first of a stage are
    corrections (the factors' change -- one kernel for the projected Maxwellian, a factor
    pass and a difference otherwise --, the source change, the wall refresh, FP32 sweep,
    update with moments, test).  A stage after the first reuses the moments the previous
    one left (no moment pass; the mixed precision converts f for its FP32 phase only when
    walls read it)."""
    n = 1
    per_main = (4 if main_fp32 else 5) + bool(walls)
    for k in range(st.n_stages):
        if k == 0 or guess:
            n += 2                                         # stage set-up, moments
        else:
            n += 1 + (1 if (mixed and walls) else 0)       # stage set-up, the FP32 copy of f
        n += (k > 0) + (k < st.n_stages - 1)               # stage combines
        n += 9 if guess else 0
        if st.iterations_fp32[k]:
            conv = (1 + (0 if (bdf2 or k > 0) else 1)) if guess else 0
            n += 6 + conv + (4 + bool(walls)) * st.iterations_fp32[k]   # FP32 phase
        its = st.iterations[k]
        per_corr = (5 if projected else 6) + bool(walls)
        n += (per_main + per_corr * (its - 1)) if (refine and its > 0) else per_main * its
    return n


def timed_steps(s, steps, world, local, tstream, guess=False, main_fp32=False, walls=False, restore=None,
                refine=False, mixed=False, projected=True):
    """Run `steps` steps of solver s (already warmed up; created on torch stream tstream),
    each bracketed by CUDA events on that stream; the time is the sum of the steps'
    device times (the statistics read between steps is not inside any bracket).
    restore: called before every step, outside the bracket (puts back the step's input
    state, so every timed step advances the same f^k)."""
    import torch
    s.synchronize()
    sweeps0 = s.last_stats().total_sweeps
    clocks = Clocks(local)
    barrier(world)
    clocks.start()
    torch.cuda.synchronize()
    iters, launches, el = [], 0, 0.0
    for _ in range(steps):
        if restore is not None:
            restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(tstream)
        s.step_async(1)
        e1.record(tstream)
        st = s.last_stats()
        if st.status != 0:
            raise RuntimeError("step failed with status %d" % st.status)
        e1.synchronize()
        el += e0.elapsed_time(e1) * 1e-3
        iters.append({"fp64": list(st.iterations)[:st.n_stages], "fp32": list(st.iterations_fp32)[:st.n_stages]})
        launches += launches_per_step(st, guess, main_fp32, walls, refine, mixed=mixed, projected=projected)
    s.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    sweeps = s.last_stats().total_sweeps - sweeps0
    return max_over_ranks(el, world), sweeps, iters, launches, clk


# DRAM bytes (read + write) per sweep launch at the 64x64 shock tube with 32x32 velocities,
# from the ncu captures summarised in profiles/ (the same kernels as timed here); a launch
# of the n x n workload moves (n / 64)^2 times as much (traffic grows with the cells).
PROFILED_TRAFFIC = {
    "fp64": (3.750e9, "profiles/sweep_fp64_cached_shock_tube_64_p2_v32.md"),
    "fp64_pairs_front": (3.409e9, "profiles/sweep_front_pair_fp64_shock_tube_64_p2_v32.md"),
    "fp32_front": (0.528e9, "profiles/sweep_front_fp32_shock_tube_64_p2_v32.md"),
}


def sweep_roofline(w, precision, reps, peaks, n_side=None, n_v=None, sweep_mode="auto", fp64_peak=None,
                   pairs=False):
    """Event-timed sweep kernel of the given precision on its own handle (first-stage
    coefficient, local-inverse cache as in the step) and its roofline entry.  pairs: the
    FP64-data sweep in float pairs (the FP64 phase of the mixed precision), reported
    against HBM like the FP32 sweep, with its FP64-equivalent rate beside it."""
    from paper_2608_19150_b300 import bgk
    s = bgk.Solver.from_workload(w, precision=precision, sweep_mode=sweep_mode,
                                 hp_sweep="pairs" if pairs else "fp64")
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    if sweep_mode == "auto":
        s.autotune_sweep(2)
    s.sweep(0.0, 0.0)
    s.timing(reset=True)
    for _ in range(reps):
        s.sweep(0.0, 0.0)
    ms, n = s.timing(reset=True)
    sweep_ms = ms / max(1, n)
    dof = s.nv * s.nnode
    tsz = 8 if precision == "fp64" else 4
    hbm_gbs = 2 * tsz * dof / (sweep_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    cached = s.cache_bytes > 0
    kind = elem_of(w)[0]
    ename = {"p2tri": "ElemP2Tri", "p1tri": "ElemP1Tri", "p1tet": "ElemP1Tet", "q1quad": "ElemQ1Quad"}[kind]
    kname = "k_sweep_ts" if s.sweep_mode == "ts" else "k_sweep"
    front = precision != "fp64" and kname == "k_sweep" and s.front_slots > 0
    if precision == "fp64" and pairs and cached:
        fl = sweep_flops_per_item(cached, kind)
        tf = fl * s.nv * s.ncell / (sweep_ms * 1e-3) / 1e12
        r = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
             "traffic": None,
             "kernel": ("k_sweep_ts<%s,double,cached,pairs>" % ename) if kname == "k_sweep_ts" else
                       ("k_sweep_front_pair<%s>" % ename) if (s.front_slots > 0 and s.sweep_threads <= 64)
                       else "k_sweep_pair<%s>" % ename,
             "front_slots": s.front_slots,
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
             "fp64_equivalent_tflops": tf, "fp64_peak_tflops": fp64_peak, "fp64_equivalent_frac": tf / fp64_peak,
             "flops_per_local_solve": fl}
    elif precision == "fp64":
        fl = sweep_flops_per_item(cached, kind)
        tf = fl * s.nv * s.ncell / (sweep_ms * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
             "frac": tf / fp64_peak, "traffic": None,
             "kernel": "%s<%s,double,%s>" % (kname, ename, "cached" if cached else "uncached"),
             "flops_per_local_solve": fl,
             "peak_source": "measured in this run: FP64 FMA probe (bgk_probe_fma_tflops), of measured"}
    else:
        r = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
             "traffic": None,
             "kernel": ("k_sweep_front<%s>" % ename) if front else
                       "%s<%s,float,%s>" % (kname, ename, "cached" if cached else "uncached,fused source"),
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)", "front_slots": s.front_slots}
    if pairs and precision == "fp64":
        profiled = PROFILED_TRAFFIC.get("fp64_pairs_front" if (s.front_slots > 0 and s.sweep_threads <= 64 and
                                                               kname == "k_sweep") else "fp64_pairs")
    else:
        profiled = PROFILED_TRAFFIC.get("fp32_front" if front else precision)
    if profiled and kind == "p2tri" and kname == "k_sweep" and n_side and n_v == 32 and (precision == "fp32" or cached):
        r["traffic"] = profiled[0] * (n_side / 64.0) ** 2
        r["traffic_source"] = profiled[1] + " (scaled from 64x64 by the cell count)"
    r.update({"sweep_ms": sweep_ms, "sweep_mode": s.sweep_mode, "dof_per_launch": dof,
              "algorithmic_bytes_per_dof": 2 * tsz,
              "hbm_achieved_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm_peak,
              "local_inverse_cache_gb": s.cache_bytes / 1e9})
    s.close()
    return r


def state_errors(f, U, f_ref, U_ref, d):
    """Relative differences after the same steps from the same state: f in the max norm,
    each moment (n, n u, E) in the l2 norm over nodes (momentum relative to max(|n u|, |n|))."""
    nrm = np.linalg.norm
    return {"f_max_rel": float(np.abs(f - f_ref).max() / np.abs(f_ref).max()),
            "n_l2_rel": float(nrm(U[:, 0] - U_ref[:, 0]) / nrm(U_ref[:, 0])),
            "nu_l2_rel": float(nrm(U[:, 1:1 + d] - U_ref[:, 1:1 + d]) / max(nrm(U_ref[:, 1:1 + d]), nrm(U_ref[:, 0]))),
            "E_l2_rel": float(nrm(U[:, -1] - U_ref[:, -1]) / nrm(U_ref[:, -1]))}


PRE_STEPS = 3


def pre_steps(args):
    """Steps from the initial state to the state every timed step starts from."""
    return PRE_STEPS


def run_ours(args):
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_2608_19150_b300 import bgk
    w = workload(args)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    tstream = torch.cuda.Stream()
    walls = WALL_SETS[args.walls] or w.walls
    s = bgk.Solver.from_workload(w, precision=args.precision, eager=args.eager, cache_inverse=args.cache,
                                 stream=tstream.cuda_stream, sweep_mode=args.sweep_mode, walls=walls,
                                 collision=args.collision, stage_predictor=args.stage_predictor)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    tune = s.autotune_sweep(2) if args.sweep_mode == "auto" else None   # untimed set-up
    chosen = s.sweep_mode
    dof = s.nv * s.nnode
    fdt = np.float32 if args.precision == "fp32" else np.float64
    tdt = torch.float64 if fdt == np.float64 else torch.float32
    # the input state of every step: PRE_STEPS steps from the initial state (untimed); every
    # warm-up and timed step starts from it (restored outside the timed bracket), so any
    # --steps runs the same step (the shock tube itself turns non-physical after about
    # 3.7e-3 time units, the 13th step at CFL 10, as the oracle does on coarser grids)
    pre = pre_steps(args)
    for _ in range(pre):
        s.step(1)
    f_in = torch.empty(dof, dtype=tdt, device="cuda")
    s.get_f_device(f_in.data_ptr(), fdt)
    torch.cuda.synchronize()

    flush = l2_flusher(dof * np.dtype(fdt).itemsize)

    def restore_main():
        s.set_f_device(f_in.data_ptr(), fdt)
        if flush:
            flush()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        restore_main()
        s.step(1)
    refine = s.refine_active
    el_max, sweeps, iters, launches, clk = timed_steps(s, args.steps, world, local, tstream,
                                                       main_fp32=args.precision == "fp32", walls=bool(walls),
                                                       restore=restore_main, refine=refine,
                                                       mixed=args.precision == "mixed",
                                                       projected=args.collision == "maxwellian")
    value = job_throughput(dof * sweeps, el_max, world)
    f_end, U_end = s.get_f(np.float64), s.get_moments()
    # end to end through the C ABI with host buffers: every step's f^k comes in from pinned
    # host memory (the next step's copy overlapping this step's sweeps on the handle's copy
    # stream) and its moments go out to the host
    f_host = torch.empty(dof, dtype=tdt, pin_memory=True)
    f_host.copy_(f_in.cpu())
    U = np.empty((s.nnode, s.dim + 2))
    barrier(world)
    t0 = time.perf_counter()
    e2e_sweeps = 0
    s.upload_f_async(f_host.data_ptr(), fdt)
    for k in range(args.steps):
        s.set_f_uploaded()
        if k + 1 < args.steps:
            s.upload_f_async(f_host.data_ptr(), fdt)
        st = s.step(1)
        e2e_sweeps += sum(list(st.iterations)[:st.n_stages]) + sum(list(st.iterations_fp32)[:st.n_stages])
        s.lib.bgk_get_moments(s.h, U.ctypes.data_as(bgk.C.c_void_p))
    el_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": job_throughput(dof * e2e_sweeps, el_e2e, world), "unit": UNIT,
           "h2d_bytes_per_step": int(f_host.numel() * f_host.element_size()), "d2h_bytes_per_step": int(U.nbytes),
           "copies": "bgk_upload_f_async / bgk_set_f_uploaded: each step's input copied from pinned host memory "
                     "on the handle's copy stream while the previous step runs; moments read back every step"}
    dt = s.dt
    s.close()
    del s
    # the plain FP64 path on the same steps, for the comparison the metric asks for
    plain = None
    if args.precision != "fp64":
        p = bgk.Solver.from_workload(w, precision="fp64", stream=tstream.cuda_stream, sweep_mode=args.sweep_mode,
                                     walls=walls, collision=args.collision, stage_predictor=args.stage_predictor)
        f_in64 = f_in.to(torch.float64)
        p.set_f_device(f_in64.data_ptr(), np.float64)
        p.set_inflow_maxwellian(w.inflow)
        if args.sweep_mode == "auto":
            p.autotune_sweep(2)

        def restore_plain():
            p.set_f_device(f_in64.data_ptr(), np.float64)
            if flush:
                flush()
                torch.cuda.synchronize()

        for _ in range(args.warmup):
            restore_plain()
            p.step(1)
        pe, psw, pit, _, pclk = timed_steps(p, args.steps, world, local, tstream, walls=bool(walls),
                                            restore=restore_plain)
        plain = {"ms_per_step": 1e3 * pe / args.steps, "value": job_throughput(dof * psw, pe, world), "picard_iterations": pit,
                 "clocks": pclk,
                 "error_vs_plain_fp64": state_errors(f_end, U_end, p.get_f(np.float64), p.get_moments(), p.dim)}
        p.close()
        del p
    # the sweep kernels, event-timed on their own stream; the FP64 sweep's arithmetic peak
    # is the FMA rate measured here and now
    fp64_peak = bgk.probe_fma_tflops(np.float64)
    rl = {"fp64": sweep_roofline(w, "fp64", args.sweep_reps, peaks, args.n_side, args.n_v, args.sweep_mode,
                                 fp64_peak)}
    if args.precision == "mixed":
        # the kernel of the mixed step's FP64 phase (float pairs; the plain path keeps FP64)
        rl["fp64_pairs"] = sweep_roofline(w, "fp64", args.sweep_reps, peaks, args.n_side, args.n_v,
                                          args.sweep_mode, fp64_peak, pairs=True)
    if args.precision != "fp64":
        rl["fp32"] = sweep_roofline(w, "fp32", args.sweep_reps, peaks, args.n_side, args.n_v, args.sweep_mode)
    # dominant kernel of the timed step: the sweep that used the most time
    n64 = sum(sum(i["fp64"]) for i in iters)
    n32 = sum(sum(i["fp32"]) for i in iters)
    if refine:
        # the FP64 iterations after the first of a stage are FP32 correction sweeps
        full = sum(sum(1 for x in i["fp64"] if x > 0) for i in iters)
        n32 += n64 - full
        n64 = full
    k64 = "fp64_pairs" if "fp64_pairs" in rl and rl["fp64_pairs"]["local_inverse_cache_gb"] > 0 else "fp64"
    dom = k64
    if "fp32" in rl and n32 * rl["fp32"]["sweep_ms"] > n64 * rl[k64]["sweep_ms"]:
        dom = "fp32"
    roofline = dict(rl[dom])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, 1024 if w.mesh.dim == 2 else 256, dt)
        if walls:
            cpu["sample"] += WALL_NOTE
    if rank != 0:
        return
    ms = 1e3 * el_max / args.steps
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32 sweeps then f64 (mixed)"}[args.precision],
            "data": "synthetic",
            "config": config(w, args, dict({"step_input": "the state after %d steps from the initial state, "
                                                          "restored before every step outside the timed region" % pre},
                                           **({"stage_predictor": "stages after the first start from moments "
                                                                  "extrapolated across the stage abscissae (both arms)"}
                                              if args.stage_predictor else {}))),
            "roofline": roofline, "rooflines": rl,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "picard_iterations": iters, "sweeps_timed": sweeps, "dt": dt,
            "fp64_phase": ("per stage one full float-pair sweep, then FP32 correction sweeps of the change of "
                           "the source (Picard refinement)") if refine else "full sweeps"}
    if tune:
        line["sweep_autotune_ms"] = tune
        line["sweep_chosen"] = chosen
    if plain:
        line["plain_fp64"] = plain
        line["speedup_vs_plain_fp64"] = plain["ms_per_step"] / ms
    print(json.dumps(line), flush=True)


def run_batched(args):
    """64 independent backward-Euler instances (seeded draw), one persistent sweep launch
    per Picard iteration over all of them."""
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_2608_19150_b300 import bgk, synth
    draws = synth.batched_draw(args.instances, seed=3)
    ws = [synth.workload_random_smooth(seed=d["seed"], n_side=d["n_side"], kx=d["kx"], n_v=d["n_v"],
                                       knudsen=d["knudsen"]) for d in draws]
    mlp, guess_info = None, None
    use_guess = not args.no_guess
    if use_guess:
        # guess network trained on seeded small runs drawn like the batch (other seeds)
        from paper_2608_19150_b300 import guess as G
        t0 = time.perf_counter()
        X, Y = [], []
        for d in synth.batched_draw(96, seed=11):
            w = synth.workload_random_smooth(seed=d["seed"], n_side=min(d["n_side"], 24), kx=d["kx"], n_v=16,
                                             knudsen=d["knudsen"])
            s_ = bgk.Solver.from_workload(w, l_max=3000)
            s_.set_state_maxwellian(w.init)
            s_.set_inflow_maxwellian(w.inflow)
            G.collect(s_, 4, X, Y)
            s_.close()
        X, Y = torch.cat(X), torch.cat(Y)
        mlp = bgk.MLP(X.shape[1], Y.shape[1], 128, seed=7)
        losses = G.train(mlp, X, Y, iters=2000, batch=8192, lr=2e-3, lr_final=1e-4, seed=3)
        guess_info = {"train_runs": 96, "samples": int(X.shape[0]), "train_s": time.perf_counter() - t0,
                      "loss_first": float(losses[:20].mean()), "loss_last": float(losses[-50:].mean())}
        del X, Y

    tstream = torch.cuda.Stream()

    def run(precision, use_guess):
        t0 = time.perf_counter()
        b = bgk.Batch(ws, precision=precision, cache_inverse=args.cache, l_max=3000, stream=tstream.cuda_stream)
        setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        blocks = b.autotune(reps=2)          # before any state is set: nothing to save
        tune_s = time.perf_counter() - t0
        if use_guess:
            b.set_guess(mlp)
        for s_, w in zip(b.instances, ws):
            s_.set_state_maxwellian(w.init)
            s_.set_inflow_maxwellian(w.inflow)
        dofs = np.array([s_.nv * s_.nnode for s_ in b.instances], dtype=np.float64)
        for _ in range(args.warmup):
            b.step(1)
        clocks = Clocks(local)
        barrier(world)
        clocks.start()
        torch.cuda.synchronize()
        upd, el = 0.0, 0.0
        iters = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(tstream)
            it, st = b.step(1)
            e1.record(tstream)
            e1.synchronize()
            el += e0.elapsed_time(e1) * 1e-3
            upd += float((dofs * it).sum())
            iters.append(it.tolist())
        torch.cuda.synchronize()
        clk = clocks.stop()
        return b, blocks, setup, tune_s, upd, iters, max_over_ranks(el, world), clk

    plain = None
    if not args.no_compare:
        pb, _, _, _, pupd, pit, pel, pclk = run("fp64", False)
        plain = {"ms_per_step": 1e3 * pel / args.steps, "value": job_throughput(pupd, pel, world),
                 "picard_iterations_per_instance": pit, "clocks": pclk}
        pb.close()
        del pb
    b, blocks, setup, tune_s, upd, iters, el_max, clk = run(args.precision, use_guess)
    b.timing(reset=True)
    for _ in range(args.sweep_reps):
        b.sweep()
    ms, n = b.timing(reset=True)
    sweep_ms = ms / max(1, n)
    info = b.info()
    tsz = 4 if args.precision == "fp32" else 8
    hbm_gbs = 2 * tsz * info["dof"] / (sweep_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    if rank != 0:
        return
    line = {"metric": METRIC, "value": job_throughput(upd, el_max, world), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32 sweeps then f64 (mixed)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "batched 2D-2V: %d instances, 2k-50k triangles (seeded jittered squares), P1/P2, "
                                   "16^2-48^2 velocities, Kn log-uniform 1e-4..1, backward Euler, CFL 10"
                                   % args.instances,
                       "total_dof": int(info["dof"]), "sweep_units": info["units"], "persistent_ctas": info["ctas"],
                       "precision": args.precision, "parallelism": "replicas",
                       "ordinates_per_cta_chosen": np.bincount(blocks, minlength=5)[[1, 2, 4]].tolist(),
                       "setup_s": setup, "autotune_s": tune_s,
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_gbs / hbm_peak, "traffic": None, "kernel": "k_sweep_batched",
                         "sweep_ms": sweep_ms},
            "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
            "picard_iterations_per_instance": iters}
    if guess_info:
        line["learned_guess"] = guess_info
    if plain:
        line["plain_fp64_batch"] = plain
        line["speedup_vs_plain_fp64"] = plain["ms_per_step"] / line["ms_per_step"]
    print(json.dumps(line), flush=True)


def _learned_workload(seed, n_side, dt=None):
    """Held-out / training run of the learned-guess workload: P1, 32x32 velocities, BDF2,
    Kn log-uniform in [1e-4, 1] drawn from the run's seed, random smooth initial moments."""
    from paper_2608_19150_b300 import synth
    r = synth.splitmix64_uniform(seed, 1)[0]
    kn = 10.0 ** (-4.0 + 4.0 * r)
    return synth.workload_random_smooth(seed=seed, n_side=n_side, kx=1, n_v=32, knudsen=kn, k_v=3,
                                        integrator="BDF2")


def run_learned(args):
    """Learned initial guess on the 256x256 P1 BDF2 workload: train on seeded small runs
    (dt of the full mesh), then time full-size held-out runs with and without it."""
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_2608_19150_b300 import bgk, guess
    n_full = args.n_side if args.n_side != 128 else 256
    probe = _learned_workload(2000, n_full)
    s0 = bgk.Solver.from_workload(probe, precision=args.precision, cache_inverse="off")
    dt_full = s0.dt
    s0.close()
    del s0
    # training data: seeded runs 1000.. on 32x32 meshes with the full mesh's time step
    t0 = time.perf_counter()
    X, Y, train_iters = [], [], []
    for k in range(args.train_runs):
        w = _learned_workload(1000 + k, 32)
        s = bgk.Solver.from_workload(w, dt=dt_full, l_max=2000)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        train_iters += guess.collect(s, 4, X, Y)
        s.close()
    X = torch.cat(X)
    Y = torch.cat(Y)
    gen_s = time.perf_counter() - t0
    F, O = X.shape[1], Y.shape[1]
    m = bgk.MLP(F, O, 128, seed=7)
    t0 = time.perf_counter()
    losses = guess.train(m, X, Y, iters=3000, batch=8192, lr=2e-3, lr_final=1e-4, seed=3)
    train_s = time.perf_counter() - t0
    # held-out full-size runs
    res = {"plain": [0, 0.0, 0], "learned": [0, 0.0, 0]}
    per_run = []
    clocks = Clocks(local)
    clocks.start()
    for k in range(args.eval_runs):
        w = _learned_workload(2000 + k, n_full)
        row = {"knudsen": w.knudsen}
        for name in ("plain", "learned"):
            tstream = torch.cuda.Stream()
            s = bgk.Solver.from_workload(w, precision=args.precision, l_max=2000, stream=tstream.cuda_stream)
            s.set_state_maxwellian(w.init)
            s.set_inflow_maxwellian(w.inflow)
            if name == "learned":
                s.set_guess(m)
            s.step(1)                                  # BDF2 start-up step (backward Euler), untimed
            torch.cuda.synchronize()
            its, el = 0, 0.0
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(tstream)
                s.step_async(1)
                e1.record(tstream)
                st = s.last_stats()
                if st.status != 0:
                    raise RuntimeError("step failed with status %d" % st.status)
                e1.synchronize()
                el += e0.elapsed_time(e1) * 1e-3
                its += st.iterations[0] + st.iterations_fp32[0]
            torch.cuda.synchronize()
            res[name][0] += its
            res[name][1] += el
            res[name][2] += args.steps
            row[name] = {"iterations": its, "ms_per_step": 1e3 * el / args.steps}
            dof = s.nv * s.nnode
            s.close()
        per_run.append(row)
    clk = clocks.stop()
    value = job_throughput(dof * res["learned"][0], max_over_ranks(res["learned"][1], world), world)
    if rank != 0:
        return
    ms_plain = 1e3 * res["plain"][1] / res["plain"][2]
    ms_learn = 1e3 * res["learned"][1] / res["learned"][2]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": 1, "ms_per_step": ms_learn, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32 sweeps then f64 (mixed)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "learned initial guess, 2D-2V: %dx%d squares (%d P1 triangles), 32x32 velocities, "
                                   "BDF2, CFL 10, Kn log-uniform 1e-4..1 per run; MLP 4 layers x 128 (FP32 training, "
                                   "BF16 inference)" % (n_full, n_full, 2 * n_full * n_full),
                       "train_runs": args.train_runs, "train_mesh": "32x32 squares, dt of the full mesh",
                       "train_samples": int(X.shape[0]), "eval_runs": args.eval_runs, "parallelism": "replicas",
                       "l2": "inputs larger than L2"},
            "learned_guess": {"iterations_plain": res["plain"][0], "iterations_learned": res["learned"][0],
                              "ms_per_step_plain": ms_plain, "ms_per_step_learned": ms_learn,
                              "speedup": ms_plain / ms_learn, "train_loss_first": float(losses[:20].mean()),
                              "train_loss_last": float(losses[-50:].mean()), "data_generation_s": gen_s,
                              "training_s": train_s, "per_run": per_run},
            "clocks": clk, "cpu_baseline": None, "e2e": None, "roofline": None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "batched" and args.impl == "ours":
        run_batched(args)
        return
    if args.workload == "learned" and args.impl == "ours":
        run_learned(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
