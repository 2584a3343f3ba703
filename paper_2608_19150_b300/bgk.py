"""ctypes binding of libbgk_b300.so (include/bgk.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  There is no CPU fallback:
:func:`load` raises when the library is missing or cannot be loaded.  PyTorch is used by
callers only for device memory and streams (``data_ptr()`` / ``cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbgk_b300.so")

BGK_OK, BGK_E_INVALID, BGK_E_CUDA, BGK_E_OOM, BGK_E_NOCONV, BGK_E_NONPHYSICAL, BGK_E_TIMEOUT, BGK_E_IO = range(8)
INTEGRATORS = {"BE": 0, "DIRK2": 1, "DIRK3": 2, "BSTABLE2": 3, "BDF2": 4}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}
DTYPES = {np.dtype(np.float64): 0, np.dtype(np.float32): 1}


class BgkError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s failed: %s (status %d)" % (where, _lib_status(status), status))
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("k_x", C.c_int), ("n_vertices", C.c_int), ("xyz", C.c_void_p),
                ("n_cells", C.c_int), ("cell_vertices", C.c_void_p), ("shape", C.c_int)]


def _shape(dim, cells):
    """0: simplices; 1: Q1 quadrilaterals (2D cells of four vertices)."""
    return 1 if dim == 2 and cells.shape[1] == 4 else 0


class VGrid(C.Structure):
    _fields_ = [("L", C.c_double), ("n_points", C.c_int), ("k_v", C.c_int)]


class Physics(C.Structure):
    _fields_ = [("nu", C.c_double), ("integrator", C.c_int), ("dt", C.c_double), ("cfl", C.c_double),
                ("collision", C.c_int), ("walls", C.c_int * 6)]


COLLISIONS = {"maxwellian": 0, "linear": 1, "interpolated": 2}
WALLS = {"inflow": 0, "bounce_back": 1, "reflect": 2}
SIDES = ("x-", "x+", "y-", "y+", "z-", "z+")


class Config(C.Structure):
    _fields_ = [("tau", C.c_double), ("l_max", C.c_int), ("precision", C.c_int), ("block_threads", C.c_int),
                ("stream", C.c_void_p), ("eager", C.c_int),
                ("cache_inverse", C.c_int), ("fp32_floor", C.c_double), ("prefetch", C.c_int),
                ("sweep_mode", C.c_int), ("sweep_front", C.c_int), ("hp_sweep", C.c_int),
                ("refine", C.c_int), ("stage_predictor", C.c_int)]

SWEEP_MODES = {"auto": 0, "tgs": 1, "ts": 2}
# arithmetic of FP64-data sweeps with cached local inverses (bgk_config.hp_sweep): automatic
# (float pairs in the FP64 phase of the mixed precision, FP64 otherwise), FP64, float pairs
HP_SWEEPS = {"auto": 0, "fp64": 1, "pairs": 2}


class Stats(C.Structure):
    _fields_ = [("n_stages", C.c_int), ("iterations", C.c_int * 3), ("measure", C.c_double * 3),
                ("total_sweeps", C.c_int), ("status", C.c_int), ("iterations_fp32", C.c_int * 3)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it is absent (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libbgk_b300.so not built (run paper_2608_19150_b300/build.py)")
    lib = C.CDLL(path)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, C.c_void_p
    sig = {
        "bgk_create": [C.POINTER(Mesh), C.POINTER(VGrid), C.POINTER(Physics), C.POINTER(Config), C.POINTER(P)],
        "bgk_destroy": [P],
        "bgk_sizes": [P, C.POINTER(C.c_int64)],
        "bgk_get_dt": [P, C.POINTER(D)],
        "bgk_front_slots": [P, C.POINTER(I)],
        "bgk_refine_active": [P, C.POINTER(I)],
        "bgk_set_state_maxwellian": [P, V],
        "bgk_set_inflow_maxwellian": [P, V],
        "bgk_set_inflow": [P, V],
        "bgk_set_f": [P, V, I],
        "bgk_get_f": [P, V, I],
        "bgk_set_f_device": [P, V, I],
        "bgk_upload_f_async": [P, V, I],
        "bgk_set_f_uploaded": [P],
        "bgk_get_f_device": [P, V, I],
        "bgk_get_moments": [P, V],
        "bgk_get_moments_device": [P, V],
        "bgk_get_velocity": [P, V, V],
        "bgk_get_generations": [P, I, V, C.POINTER(I)],
        "bgk_get_lagged_edges": [P, I, V, I, C.POINTER(I)],
        "bgk_save": [P, C.c_char_p],
        "bgk_load": [P, C.c_char_p],
        "bgk_get_time": [P, C.POINTER(C.c_int64), C.POINTER(D)],
        "bgk_sweep": [P, D, D],
        "bgk_sweep_range": [P, I, I, V, D, D],
        "bgk_moments_range_device": [P, I, I, V],
        "bgk_shard_step_begin": [P, C.POINTER(I), C.POINTER(D)],
        "bgk_shard_stage_begin": [P, I],
        "bgk_shard_stage_end": [P, I],
        "bgk_shard_step_end": [P],
        "bgk_sum_partials_device": [P, V, I, V],
        "bgk_conv_measure_device": [P, V, V, C.POINTER(D)],
        "bgk_step": [P, I, C.POINTER(Stats)],
        "bgk_step_async": [P, I],
        "bgk_last_stats": [P, C.POINTER(Stats)],
        "bgk_synchronize": [P],
        "bgk_timing": [P, I, C.POINTER(D), C.POINTER(C.c_int64)],
        "bgk_autotune_sweep": [P, I, V],
        "bgk_probe_fma_tflops": [I, C.POINTER(D)],
        "bgk_moments_measure_noalloc": [C.POINTER(VGrid), I, C.c_int64, V, I, V, V, V, V],
        "bgk_batch_create": [I, C.POINTER(Mesh), C.POINTER(VGrid), C.POINTER(Physics), C.POINTER(Config),
                             C.POINTER(P)],
        "bgk_batch_destroy": [P],
        "bgk_batch_instance": [P, I, C.POINTER(P)],
        "bgk_batch_autotune": [P, I, V],
        "bgk_batch_step": [P, I, V, V],
        "bgk_batch_sweep": [P],
        "bgk_batch_timing": [P, I, C.POINTER(D), C.POINTER(C.c_int64)],
        "bgk_batch_info": [P, C.POINTER(C.c_int64)],
        "bgk_batch_set_guess": [P, P],
        "bgk_mlp_create": [I, I, I, C.c_uint64, C.POINTER(P)],
        "bgk_mlp_destroy": [P],
        "bgk_mlp_num_params": [P, C.POINTER(C.c_int64)],
        "bgk_mlp_get_params": [P, V, V],
        "bgk_mlp_set_params": [P, V, V],
        "bgk_mlp_fit_norm": [P, V, V, C.c_int64],
        "bgk_mlp_loss_grad": [P, V, V, C.c_int64, C.POINTER(D), V],
        "bgk_mlp_train_step": [P, V, V, C.c_int64, C.c_float, C.POINTER(D)],
        "bgk_mlp_predict": [P, V, C.c_int64, V, I],
        "bgk_guess_dims": [P, C.POINTER(I), C.POINTER(I)],
        "bgk_guess_features": [P, V],
        "bgk_guess_targets": [P, V, V, V],
        "bgk_set_guess": [P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.bgk_status_string.argtypes = [C.c_int]
    lib.bgk_status_string.restype = C.c_char_p
    _lib = lib
    return lib


def _lib_status(s):
    try:
        return load().bgk_status_string(int(s)).decode()
    except Exception:  # noqa: BLE001
        return "status %d" % s


def _ck(rc, where):
    if rc != BGK_OK:
        raise BgkError(rc, where)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def moments_measure_noalloc(L, n_points, k_v, dim, n_nodes, f_ptr, dtype, U_old_ptr, U_new_ptr, measure_ptr,
                            stream=None):
    """bgk_moments_measure_noalloc: device pointers in, device pointers out, no allocation."""
    vg = VGrid(float(L), int(n_points), int(k_v))
    _ck(load().bgk_moments_measure_noalloc(C.byref(vg), int(dim), int(n_nodes), C.c_void_p(f_ptr),
                                            DTYPES[np.dtype(dtype)], C.c_void_p(U_old_ptr), C.c_void_p(U_new_ptr),
                                            C.c_void_p(measure_ptr), C.c_void_p(stream) if stream else None),
        "bgk_moments_measure_noalloc")


def probe_fma_tflops(dtype=np.float64):
    """bgk_probe_fma_tflops: measured FMA rate of the current device (TFLOP/s)."""
    t = C.c_double()
    _ck(load().bgk_probe_fma_tflops(DTYPES[np.dtype(dtype)], C.byref(t)), "bgk_probe_fma_tflops")
    return t.value


def _wall_kinds(walls):
    """{side: kind} (sides "x-".."z+", kinds of WALLS; unnamed sides inflow) -> int[6]."""
    walls = walls or {}
    if set(walls) - set(SIDES):
        raise KeyError("unknown side in walls: %s" % sorted(set(walls) - set(SIDES)))
    return (C.c_int * 6)(*[WALLS[walls.get(side, "inflow")] for side in SIDES])


class Solver:
    """Handle of one problem on the current CUDA device (thin wrapper of bgk_create)."""

    def __init__(self, dim, kx, xyz, cells, n_v, k_v, L, nu, integrator="BE", dt=0.0, cfl=10.0, tau=1e-8,
                 l_max=1000, precision="fp64", block_threads=0, stream=None, eager=False, cache_inverse="auto", fp32_floor=0.0, prefetch=False,
                 sweep_mode="auto", collision="maxwellian", walls=None, sweep_front=True,
                 hp_sweep="auto", refine=True, stage_predictor=False):
        self.lib = load()
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._cells = np.ascontiguousarray(cells, dtype=np.int32)
        m = Mesh(dim, kx, self._xyz.shape[0], _ptr(self._xyz), self._cells.shape[0], _ptr(self._cells),
                 _shape(dim, self._cells))
        vg = VGrid(float(L), int(n_v), int(k_v))
        ph = Physics(float(nu), INTEGRATORS[integrator], float(dt), float(cfl), COLLISIONS[collision],
                     _wall_kinds(walls))
        cf = Config(float(tau), int(l_max), PRECISIONS[precision], int(block_threads),
                    C.c_void_p(stream) if stream else None, int(bool(eager)),
                    {"auto": 0, "on": 1, "off": 2}[cache_inverse], float(fp32_floor), 1 if prefetch else 0,
                    SWEEP_MODES[sweep_mode], 0 if sweep_front else 2, HP_SWEEPS[hp_sweep],
                    0 if refine else 1, 1 if stage_predictor else 0)
        h = C.c_void_p()
        _ck(self.lib.bgk_create(C.byref(m), C.byref(vg), C.byref(ph), C.byref(cf), C.byref(h)), "bgk_create")
        self.h = h
        self.stream = stream
        sz = (C.c_int64 * 10)()
        _ck(self.lib.bgk_sizes(self.h, sz), "bgk_sizes")
        (self.nv, self.nnode, self.ndof, self.ncell, self.dim, self.gmax, self.lagged, self.cache_bytes,
         self.sweep_threads, mode) = (int(x) for x in sz)
        self.sweep_mode = {1: "tgs", 2: "ts"}[mode]
        self.precision = precision
        self.fdtype = np.float32 if precision == "fp32" else np.float64

    @classmethod
    def from_workload(cls, w, **kw):
        args = dict(integrator=w.integrator, cfl=w.cfl)
        if getattr(w, "dt", 0.0) > 0.0:
            args["dt"] = w.dt
        if getattr(w, "walls", None):
            args["walls"] = w.walls
        args.update(kw)
        return cls(w.mesh.dim, w.kx, w.mesh.xyz, w.mesh.cells, w.n_v, w.k_v, w.L, w.nu, **args)

    @classmethod
    def wrap(cls, handle, precision, owner):
        """A view of a handle owned elsewhere (an instance of a Batch)."""
        self = cls.__new__(cls)
        self.lib = load()
        self.h = handle
        self._owner = owner
        sz = (C.c_int64 * 10)()
        _ck(self.lib.bgk_sizes(self.h, sz), "bgk_sizes")
        (self.nv, self.nnode, self.ndof, self.ncell, self.dim, self.gmax, self.lagged, self.cache_bytes,
         self.sweep_threads, mode) = (int(x) for x in sz)
        self.sweep_mode = {1: "tgs", 2: "ts"}[mode]
        self.precision = precision
        self.fdtype = np.float32 if precision == "fp32" else np.float64
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self.h = None
            return
        if getattr(self, "h", None):
            self.lib.bgk_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def refine_active(self):
        """True when the FP64 phase's iterations after the first of a stage are FP32
        correction sweeps (the Picard refinement of the mixed precision)."""
        n = C.c_int()
        _ck(self.lib.bgk_refine_active(self.h, C.byref(n)), "bgk_refine_active")
        return bool(n.value)

    @property
    def front_slots(self):
        """Shared-memory front slots of the FP32 generation sweep (an FP64 handle: of its
        float-pair sweep; 0: global reads)."""
        n = C.c_int()
        _ck(self.lib.bgk_front_slots(self.h, C.byref(n)), "bgk_front_slots")
        return n.value

    @property
    def dt(self):
        d = C.c_double()
        _ck(self.lib.bgk_get_dt(self.h, C.byref(d)), "bgk_get_dt")
        return d.value

    def set_state_maxwellian(self, nut):
        nut = np.ascontiguousarray(nut, dtype=np.float64)
        _ck(self.lib.bgk_set_state_maxwellian(self.h, _ptr(nut)), "bgk_set_state_maxwellian")

    def set_inflow_maxwellian(self, nut):
        nut = np.ascontiguousarray(nut, dtype=np.float64)
        _ck(self.lib.bgk_set_inflow_maxwellian(self.h, _ptr(nut)), "bgk_set_inflow_maxwellian")

    def set_inflow(self, f):
        """Inflow data f^bc as nodal values [nv, nnode] (FP64)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        _ck(self.lib.bgk_set_inflow(self.h, _ptr(f)), "bgk_set_inflow")

    def set_f(self, f):
        f = np.ascontiguousarray(f)
        _ck(self.lib.bgk_set_f(self.h, _ptr(f), DTYPES[f.dtype]), "bgk_set_f")

    def get_f(self, dtype=np.float64):
        out = np.empty((self.nv, self.nnode), dtype=dtype)
        _ck(self.lib.bgk_get_f(self.h, _ptr(out), DTYPES[np.dtype(dtype)]), "bgk_get_f")
        return out

    def set_f_device(self, ptr, dtype=np.float64):
        _ck(self.lib.bgk_set_f_device(self.h, C.c_void_p(ptr), DTYPES[np.dtype(dtype)]), "bgk_set_f_device")

    def get_f_device(self, ptr, dtype=np.float64):
        _ck(self.lib.bgk_get_f_device(self.h, C.c_void_p(ptr), DTYPES[np.dtype(dtype)]), "bgk_get_f_device")

    def upload_f_async(self, host_ptr, dtype=np.float64):
        """Start copying the next state from (pinned) host memory to the handle's staging
        buffer on its copy stream; keep the host buffer unchanged until set_f_uploaded."""
        _ck(self.lib.bgk_upload_f_async(self.h, C.c_void_p(host_ptr), DTYPES[np.dtype(dtype)]),
            "bgk_upload_f_async")

    def set_f_uploaded(self):
        """The staged state becomes the state (ordered after its copy, no host wait)."""
        _ck(self.lib.bgk_set_f_uploaded(self.h), "bgk_set_f_uploaded")

    def get_moments(self):
        U = np.empty((self.nnode, self.dim + 2))
        _ck(self.lib.bgk_get_moments(self.h, _ptr(U)), "bgk_get_moments")
        return U

    def get_moments_device(self, ptr):
        _ck(self.lib.bgk_get_moments_device(self.h, C.c_void_p(ptr)), "bgk_get_moments_device")

    def velocity(self):
        v = np.empty((self.nv, self.dim))
        w = np.empty(self.nv)
        _ck(self.lib.bgk_get_velocity(self.h, _ptr(v), _ptr(w)), "bgk_get_velocity")
        return v, w

    def generations(self, j):
        gen = np.empty(self.ncell, dtype=np.int32)
        n = C.c_int()
        _ck(self.lib.bgk_get_generations(self.h, int(j), _ptr(gen), C.byref(n)), "bgk_get_generations")
        return gen, n.value

    def lagged_edges(self, j):
        """[(upwind cell, downwind cell)] of ordinate j's lagged (cycle-breaking) edges."""
        n = C.c_int()
        _ck(self.lib.bgk_get_lagged_edges(self.h, int(j), None, 0, C.byref(n)), "bgk_get_lagged_edges")
        e = np.empty((max(n.value, 1), 2), dtype=np.int32)
        _ck(self.lib.bgk_get_lagged_edges(self.h, int(j), _ptr(e), n.value, C.byref(n)), "bgk_get_lagged_edges")
        return e[:n.value]

    def save(self, path):
        _ck(self.lib.bgk_save(self.h, os.fsencode(path)), "bgk_save")

    def load(self, path):
        _ck(self.lib.bgk_load(self.h, os.fsencode(path)), "bgk_load")

    def time(self):
        """(steps since the state was set or loaded, the time they span)"""
        n = C.c_int64()
        t = C.c_double()
        _ck(self.lib.bgk_get_time(self.h, C.byref(n), C.byref(t)), "bgk_get_time")
        return n.value, t.value

    def sweep(self, nu_s, q_scale):
        _ck(self.lib.bgk_sweep(self.h, float(nu_s), float(q_scale)), "bgk_sweep")

    def sweep_range(self, j_begin, j_end, U_ptr, nu_s=0.0, q_scale=0.0):
        """One sweep of ordinates [j_begin, j_end) with the moments at device pointer U_ptr."""
        _ck(self.lib.bgk_sweep_range(self.h, int(j_begin), int(j_end), C.c_void_p(U_ptr), float(nu_s),
                                     float(q_scale)), "bgk_sweep_range")

    def moments_range_device(self, j_begin, j_end, U_ptr):
        """Partial moments of ordinates [j_begin, j_end) into the device buffer at U_ptr."""
        _ck(self.lib.bgk_moments_range_device(self.h, int(j_begin), int(j_end), C.c_void_p(U_ptr)),
            "bgk_moments_range_device")

    # ---- a step driven stage by stage (ordinate shards; bgk_shard_*)
    def shard_step_begin(self):
        """(stages of the step, Picard tolerance)"""
        n, tol = C.c_int(), C.c_double()
        _ck(self.lib.bgk_shard_step_begin(self.h, C.byref(n), C.byref(tol)), "bgk_shard_step_begin")
        return n.value, tol.value

    def shard_stage_begin(self, stage):
        _ck(self.lib.bgk_shard_stage_begin(self.h, int(stage)), "bgk_shard_stage_begin")

    def shard_stage_end(self, stage):
        _ck(self.lib.bgk_shard_stage_end(self.h, int(stage)), "bgk_shard_stage_end")

    def shard_step_end(self):
        _ck(self.lib.bgk_shard_step_end(self.h), "bgk_shard_step_end")

    def sum_partials_device(self, parts_ptr, n_parts, U_ptr):
        _ck(self.lib.bgk_sum_partials_device(self.h, C.c_void_p(parts_ptr), int(n_parts), C.c_void_p(U_ptr)),
            "bgk_sum_partials_device")

    def conv_measure_device(self, U_new_ptr, U_old_ptr):
        m = C.c_double()
        _ck(self.lib.bgk_conv_measure_device(self.h, C.c_void_p(U_new_ptr), C.c_void_p(U_old_ptr), C.byref(m)),
            "bgk_conv_measure_device")
        return m.value

    def step(self, nsteps=1):
        st = Stats()
        rc = self.lib.bgk_step(self.h, int(nsteps), C.byref(st))
        _ck(rc, "bgk_step")
        return st

    def step_async(self, nsteps=1):
        _ck(self.lib.bgk_step_async(self.h, int(nsteps)), "bgk_step_async")

    def last_stats(self):
        st = Stats()
        _ck(self.lib.bgk_last_stats(self.h, C.byref(st)), "bgk_last_stats")
        return st

    def synchronize(self):
        _ck(self.lib.bgk_synchronize(self.h), "bgk_synchronize")

    def autotune_sweep(self, reps=3):
        """Keep the faster of TGS and TS on the current state (bgk_autotune_sweep); returns
        the per-sweep times in ms: {"tgs", "ts"} and, with an FP32 shadow, {"tgs32", "ts32"}."""
        ms = np.zeros(4)
        _ck(self.lib.bgk_autotune_sweep(self.h, int(reps), _ptr(ms)), "bgk_autotune_sweep")
        sz = (C.c_int64 * 10)()
        _ck(self.lib.bgk_sizes(self.h, sz), "bgk_sizes")
        self.sweep_mode = {1: "tgs", 2: "ts"}[int(sz[9])]
        out = {"tgs": float(ms[0]), "ts": float(ms[1])}
        if ms[2] > 0:
            out.update(tgs32=float(ms[2]), ts32=float(ms[3]))
        return out

    def timing(self, reset=False):
        ms = C.c_double()
        n = C.c_int64()
        _ck(self.lib.bgk_timing(self.h, int(bool(reset)), C.byref(ms), C.byref(n)), "bgk_timing")
        return ms.value, n.value

    # ---- learned initial guess
    def guess_dims(self):
        f, o = C.c_int(), C.c_int()
        _ck(self.lib.bgk_guess_dims(self.h, C.byref(f), C.byref(o)), "bgk_guess_dims")
        return f.value, o.value

    def guess_features(self, d_X_ptr):
        _ck(self.lib.bgk_guess_features(self.h, C.c_void_p(d_X_ptr)), "bgk_guess_features")

    def guess_targets(self, d_Ustart_ptr, d_X_ptr, d_Y_ptr):
        _ck(self.lib.bgk_guess_targets(self.h, C.c_void_p(d_Ustart_ptr), C.c_void_p(d_X_ptr), C.c_void_p(d_Y_ptr)),
            "bgk_guess_targets")

    def set_guess(self, mlp):
        self._guess = mlp
        _ck(self.lib.bgk_set_guess(self.h, mlp.h if mlp is not None else None), "bgk_set_guess")


class Batch:
    """Many independent backward-Euler problems advanced together (bgk_batch_*)."""

    def __init__(self, workloads, precision="fp64", tau=1e-8, l_max=1000, cache_inverse="auto", dt=None, stream=None,
                 walls=None):
        self.lib = load()
        n = len(workloads)
        self._keep = []
        meshes = (Mesh * n)()
        vgrids = (VGrid * n)()
        phys = (Physics * n)()
        for i, w in enumerate(workloads):
            xyz = np.ascontiguousarray(w.mesh.xyz, dtype=np.float64)
            cells = np.ascontiguousarray(w.mesh.cells, dtype=np.int32)
            self._keep += [xyz, cells]
            meshes[i] = Mesh(w.mesh.dim, w.kx, xyz.shape[0], _ptr(xyz), cells.shape[0], _ptr(cells),
                             _shape(w.mesh.dim, cells))
            vgrids[i] = VGrid(float(w.L), int(w.n_v), int(w.k_v))
            phys[i] = Physics(float(w.nu), INTEGRATORS["BE"], float(dt[i]) if dt else 0.0, float(w.cfl), 0,
                              _wall_kinds(walls))
        cf = Config(float(tau), int(l_max), PRECISIONS[precision], 0, C.c_void_p(stream) if stream else None, 0,
                    {"auto": 0, "on": 1, "off": 2}[cache_inverse], 0.0, 0, 0)
        self.mixed = precision == "mixed"
        h = C.c_void_p()
        _ck(self.lib.bgk_batch_create(n, meshes, vgrids, phys, C.byref(cf), C.byref(h)), "bgk_batch_create")
        self.h = h
        self.n = n
        self.precision = precision
        self.instances = []
        for i in range(n):
            hi = C.c_void_p()
            _ck(self.lib.bgk_batch_instance(self.h, i, C.byref(hi)), "bgk_batch_instance")
            self.instances.append(Solver.wrap(hi, precision, self))

    def close(self):
        if getattr(self, "h", None):
            for s in self.instances:
                s.h = None
            self.lib.bgk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_guess(self, mlp):
        self._guess = mlp
        _ck(self.lib.bgk_batch_set_guess(self.h, mlp.h if mlp is not None else None), "bgk_batch_set_guess")

    def autotune(self, reps=3):
        out = np.zeros(self.n, dtype=np.int32)
        _ck(self.lib.bgk_batch_autotune(self.h, int(reps), _ptr(out)), "bgk_batch_autotune")
        return out

    def step(self, nsteps=1, check=True):
        it = np.zeros(self.n, dtype=np.int32)
        st = np.zeros(self.n, dtype=np.int32)
        rc = self.lib.bgk_batch_step(self.h, int(nsteps), _ptr(it), _ptr(st))
        if check:
            _ck(rc, "bgk_batch_step")
        return it, st

    def sweep(self):
        _ck(self.lib.bgk_batch_sweep(self.h), "bgk_batch_sweep")

    def timing(self, reset=False):
        ms = C.c_double()
        n = C.c_int64()
        _ck(self.lib.bgk_batch_timing(self.h, int(bool(reset)), C.byref(ms), C.byref(n)), "bgk_batch_timing")
        return ms.value, n.value

    def info(self):
        out = (C.c_int64 * 4)()
        _ck(self.lib.bgk_batch_info(self.h, out), "bgk_batch_info")
        return dict(instances=out[0], dof=out[1], units=out[2], ctas=out[3])


class MLP:
    """The guess network (bgk_mlp_*): FP32 training kernels, BF16 inference."""

    def __init__(self, n_in, n_out, n_hidden=128, seed=0):
        self.lib = load()
        h = C.c_void_p()
        _ck(self.lib.bgk_mlp_create(int(n_in), int(n_hidden), int(n_out), C.c_uint64(seed), C.byref(h)),
            "bgk_mlp_create")
        self.h = h
        self.F, self.H, self.O = int(n_in), int(n_hidden), int(n_out)
        n = C.c_int64()
        _ck(self.lib.bgk_mlp_num_params(self.h, C.byref(n)), "bgk_mlp_num_params")
        self.n_params = n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.bgk_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def get_params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        nrm = np.empty(2 * self.F + 2 * self.O, dtype=np.float32)
        _ck(self.lib.bgk_mlp_get_params(self.h, _ptr(p), _ptr(nrm)), "bgk_mlp_get_params")
        return p, nrm

    def set_params(self, p=None, norm=None):
        pp = None if p is None else np.ascontiguousarray(p, dtype=np.float32)
        nn = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _ck(self.lib.bgk_mlp_set_params(self.h, _ptr(pp) if pp is not None else None,
                                        _ptr(nn) if nn is not None else None), "bgk_mlp_set_params")

    def fit_norm(self, X_ptr, Y_ptr, n):
        _ck(self.lib.bgk_mlp_fit_norm(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), int(n)), "bgk_mlp_fit_norm")

    def loss_grad(self, X_ptr, Y_ptr, n):
        loss = C.c_double()
        g = np.empty(self.n_params, dtype=np.float32)
        _ck(self.lib.bgk_mlp_loss_grad(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), int(n), C.byref(loss), _ptr(g)),
            "bgk_mlp_loss_grad")
        return loss.value, g

    def train_step(self, X_ptr, Y_ptr, n, lr):
        loss = C.c_double()
        _ck(self.lib.bgk_mlp_train_step(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), int(n), C.c_float(lr),
                                        C.byref(loss)), "bgk_mlp_train_step")
        return loss.value

    def predict(self, X_ptr, n, Y_ptr, bf16=True):
        _ck(self.lib.bgk_mlp_predict(self.h, C.c_void_p(X_ptr), int(n), C.c_void_p(Y_ptr), int(bool(bf16))),
            "bgk_mlp_predict")
