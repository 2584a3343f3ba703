"""ctypes wrapper of the plain sequential FP64 CPU oracle (``oracle/bgk_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use this module; the product path never imports it.  It shares no
code with the CUDA library.

The C source follows the paper's statement step by step (its header lists the sections
and the readings taken where the paper is silent).  This wrapper only marshals arrays.

Parity status per function (pins live in ``tests/test_oracle_pins*.py``; the multi-stage
time integration in ``tests/test_oracle_pins_time.py``: the stability function of each
tableau on a transport-free relaxation, the BDF2 recurrence, the temporal order):
  velocity grid, element matrices, projection, moments, sweep graph / generations,
  one sweep, one time step (BE, DIRK2, DIRK3, B-stable DIRK2, BDF2), the simplified
  Maxwellian collision model, the interpolated Maxwellian, bounce-back and reflecting
  walls: pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libbgk_oracle.so")
# the same source with the loop over ordinates of a sweep on all host cores (OpenMP): the
# timed CPU baseline only; parity checks use the sequential build above
_LIB_OMP_PATH = os.path.join(_HERE, "_build", "libbgk_oracle_omp.so")

INTEGRATORS = {"BE": 0, "DIRK2": 1, "DIRK3": 2, "BSTABLE2": 3, "BDF2": 4}

_lib = None
_lib_omp = None


def _compile(path, extra):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math"] + extra + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add): the sequential
    parity build and the OpenMP build of the CPU baseline."""
    if force:
        for p in (_LIB_PATH, _LIB_OMP_PATH):
            if os.path.exists(p):
                os.remove(p)
    _compile(_LIB_OMP_PATH, ["-fopenmp"])
    return _compile(_LIB_PATH, [])


def _load(omp: bool = False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(C.CDLL(_LIB_OMP_PATH))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(lib):
    """ctypes signatures of the oracle's entry points."""
    P = C.c_void_p
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
    up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_int, ip, C.c_int, C.c_int, C.c_double]
    lib.orc_create_quad.restype = P
    lib.orc_create_quad.argtypes = [C.c_int, dp, C.c_int, ip, C.c_int, C.c_int, C.c_double]
    lib.orc_destroy.argtypes = [P]
    lib.orc_info.argtypes = [P, ip]
    lib.orc_velocity.argtypes = [P, dp, dp, dp, dp]
    lib.orc_cell.argtypes = [P, C.c_int, dp, dp, dp, dp, dp, dp, ip, ip]
    lib.orc_project_1d.argtypes = [P, C.c_double, C.c_double, dp]
    lib.orc_maxwellian.argtypes = [P, dp, dp]
    lib.orc_moments.argtypes = [P, dp, dp]
    lib.orc_build_dags.restype = C.c_long
    lib.orc_build_dags.argtypes = [P]
    lib.orc_build_dags_for.restype = C.c_long
    lib.orc_build_dags_for.argtypes = [P, ip, C.c_int]
    lib.orc_generations.restype = C.c_int
    lib.orc_generations.argtypes = [P, C.c_int, ip, up]
    lib.orc_face_signs.argtypes = [P, C.c_int, ip]
    lib.orc_sweep.argtypes = [P, dp, dp, dp, dp, C.c_double, C.c_double, dp]
    lib.orc_sweep_range.argtypes = [P, dp, dp, dp, dp, C.c_double, C.c_double, dp, C.c_int, C.c_int]
    lib.orc_maxwellian_rows.argtypes = [P, dp, ip, C.c_int, dp]
    lib.orc_sweep_rows.restype = C.c_int
    lib.orc_sweep_rows.argtypes = [P, ip, C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, dp]
    lib.orc_dt_explicit.restype = C.c_double
    lib.orc_dt_explicit.argtypes = [P]
    lib.orc_tableau.restype = C.c_int
    lib.orc_tableau.argtypes = [C.c_int, dp, dp, dp]
    lib.orc_conv_measure.restype = C.c_double
    lib.orc_conv_measure.argtypes = [P, dp, dp]
    lib.orc_set_physics.argtypes = [P, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int]
    lib.orc_set_collision.argtypes = [P, C.c_int]
    lib.orc_set_walls.restype = C.c_int
    lib.orc_set_walls.argtypes = [P, ip]
    lib.orc_step.restype = C.c_int
    lib.orc_step.argtypes = [P, dp, C.c_void_p, dp, ip, dp]
    return lib


def tableau(integrator: str):
    lib = _load()
    A, b, c = np.zeros(9), np.zeros(3), np.zeros(3)
    S = lib.orc_tableau(INTEGRATORS[integrator], A, b, c)
    return A.reshape(3, 3)[:S, :S].copy(), b[:S].copy(), c[:S].copy()


class Oracle:
    """One problem: mesh + spatial degree + velocity grid (+ physics for time steps)."""

    def __init__(self, dim, kx, xyz, cells, n1d, kv, L, omp=False):
        """omp: run sweeps on all host cores (the OpenMP build; CPU baseline only)."""
        self.lib = _load(omp)
        self.dim, self.kx, self.n1d, self.kv, self.L = dim, kx, n1d, kv, L
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        if dim == 2 and cells.shape[1] == 4:       # Q1 quadrilaterals
            self.h = self.lib.orc_create_quad(xyz.shape[0], xyz, cells.shape[0], cells, n1d, kv, float(L))
        else:
            self.h = self.lib.orc_create(dim, kx, xyz.shape[0], xyz, cells.shape[0], cells, n1d, kv, float(L))
        if not self.h:
            raise ValueError("oracle rejected the problem")
        info = np.zeros(5, dtype=np.int32)
        self.lib.orc_info(self.h, info)
        self.nv, self.nnode, self.ndof, self.nface, self.ncell = (int(x) for x in info)
        self._dags = False

    @classmethod
    def from_workload(cls, w, omp=False):
        o = cls(w.mesh.dim, w.kx, w.mesh.xyz, w.mesh.cells, w.n_v, w.k_v, w.L, omp=omp)
        if getattr(w, "walls", None):
            o.set_walls(w.walls)
        return o

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # --- grid and geometry -------------------------------------------------------
    def velocity(self):
        v = np.zeros(self.nv * self.dim)
        w = np.zeros(self.nv)
        x1, w1 = np.zeros(self.n1d), np.zeros(self.n1d)
        self.lib.orc_velocity(self.h, v, w, x1, w1)
        return v.reshape(self.nv, self.dim), w, x1, w1

    def cell(self, c):
        nd, nf, d = self.ndof, self.nface, self.dim
        vol = np.zeros(1)
        M, G = np.zeros(nd * nd), np.zeros(d * nd * nd)
        Fm, un, ar = np.zeros(nf * nd * nd), np.zeros(nf * d), np.zeros(nf)
        nbr, nn = np.zeros(nf, dtype=np.int32), np.zeros(nf * nd, dtype=np.int32)
        self.lib.orc_cell(self.h, int(c), vol, M, G, Fm, un, ar, nbr, nn)
        return dict(vol=vol[0], M=M.reshape(nd, nd), G=G.reshape(d, nd, nd), F=Fm.reshape(nf, nd, nd),
                    unit_n=un.reshape(nf, d), area=ar, nbr=nbr, nbr_node=nn.reshape(nf, nd))

    def dt_explicit(self):
        return self.lib.orc_dt_explicit(self.h)

    # --- Maxwellian and moments --------------------------------------------------
    def project_1d(self, u, theta):
        c = np.zeros(self.n1d)
        self.lib.orc_project_1d(self.h, float(u), float(theta), c)
        return c

    def maxwellian(self, nut):
        """nut [nnode, d+2] -> f [nv, nnode] (projected Maxwellian at every node)."""
        out = np.zeros((self.nv, self.nnode))
        self.lib.orc_maxwellian(self.h, np.ascontiguousarray(nut, dtype=np.float64), out)
        return out

    def maxwellian_rows(self, nut, js):
        """Projected Maxwellian for the ordinates js only: [len(js), nnode]."""
        js = np.ascontiguousarray(js, dtype=np.int32)
        out = np.zeros((len(js), self.nnode))
        self.lib.orc_maxwellian_rows(self.h, np.ascontiguousarray(nut, dtype=np.float64), js, len(js), out)
        return out

    def sweep_rows(self, js, fold, Mn, q, fbc, nu, nu_s):
        """One sweep of the ordinates js; every array holds only those rows."""
        if not self._dags:
            self.build_dags()
        js = np.ascontiguousarray(js, dtype=np.int32)
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(len(js), self.nnode)  # noqa: E731
        fnew = np.zeros((len(js), self.nnode))
        st = self.lib.orc_sweep_rows(self.h, js, len(js), c(fold), c(Mn), c(q), c(fbc), float(nu), float(nu_s), fnew)
        if st != 0:
            raise ValueError("sweep_rows needs the mirror rows of wall faces: not available with walls set")
        return fnew

    def moments(self, f):
        U = np.zeros((self.nnode, self.dim + 2))
        self.lib.orc_moments(self.h, np.ascontiguousarray(f, dtype=np.float64), U)
        return U

    def conv_measure(self, Unew, Uold):
        return self.lib.orc_conv_measure(self.h, np.ascontiguousarray(Unew), np.ascontiguousarray(Uold))

    # --- sweep graphs --------------------------------------------------------------
    def build_dags(self):
        n = self.lib.orc_build_dags(self.h)
        if n < 0:
            raise RuntimeError("oracle DAG construction failed")
        self._dags = True
        return int(n)

    def build_dags_for(self, js):
        """Build the sweep graphs of the ordinates js only (for sampled full-size checks)."""
        js = np.ascontiguousarray(js, dtype=np.int32)
        n = self.lib.orc_build_dags_for(self.h, js, len(js))
        if n < 0:
            raise RuntimeError("oracle DAG construction failed")
        self._dags = True
        return int(n)

    def generations(self, j):
        if not self._dags:
            self.build_dags()
        gen = np.zeros(self.ncell, dtype=np.int32)
        lag = np.zeros(self.ncell * self.nface, dtype=np.uint8)
        G = self.lib.orc_generations(self.h, int(j), gen, lag)
        return gen, lag.reshape(self.ncell, self.nface), G

    def face_signs(self, j):
        s = np.zeros(self.ncell * self.nface, dtype=np.int32)
        self.lib.orc_face_signs(self.h, int(j), s)
        return s.reshape(self.ncell, self.nface)

    # --- sweep and step ------------------------------------------------------------
    def sweep(self, fold, Mn, q, fbc, nu, nu_s):
        if not self._dags:
            self.build_dags()
        fnew = np.zeros((self.nv, self.nnode))
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(self.nv, self.nnode)  # noqa: E731
        self.lib.orc_sweep(self.h, c(fold), c(Mn), c(q), c(fbc), float(nu), float(nu_s), fnew)
        return fnew

    def sweep_range(self, fold, Mn, q, fbc, nu, nu_s, j0, j1, fnew=None):
        """One sweep restricted to ordinates j0 <= j < j1 (writes those rows of fnew)."""
        if not self._dags:
            self.build_dags()
        if fnew is None:
            fnew = np.zeros((self.nv, self.nnode))
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(self.nv, self.nnode)  # noqa: E731
        self.lib.orc_sweep_range(self.h, c(fold), c(Mn), c(q), c(fbc), float(nu), float(nu_s), fnew, int(j0), int(j1))
        return fnew

    def set_physics(self, nu, dt, integrator="BE", tau=1e-8, lmax=1000):
        self.integrator = integrator
        self.lib.orc_set_physics(self.h, float(nu), float(dt), INTEGRATORS[integrator], float(tau), int(lmax))

    def set_collision(self, kind):
        """'maxwellian' (App. B projection), 'linear' (Eq. linear-Maxwellian: n / |V|) or
        'interpolated' (the Maxwellian's values at the grid points, Sec. 5.1.1)."""
        self.lib.orc_set_collision(self.h, {"maxwellian": 0, "linear": 1, "interpolated": 2}[kind])

    def set_walls(self, walls):
        """Sec. 4.2 boundary conditions per box side: {"x-"|"x+"|"y-"|"y+"|"z-"|"z+":
        "inflow"|"bounce_back"|"reflect"}; sides not named stay inflow."""
        sides = ("x-", "x+", "y-", "y+", "z-", "z+")
        kinds = {"inflow": 0, "bounce_back": 1, "reflect": 2}
        k = np.array([kinds[walls.get(sd, "inflow")] for sd in sides], dtype=np.int32)
        st = self.lib.orc_set_walls(self.h, k)
        if st != 0:
            raise ValueError("orc_set_walls: status %d" % st)

    def step(self, f, fbc, fprev=None):
        """One time step in place on a copy; returns (f_next, iters per stage, measures, status)."""
        if not self._dags:
            self.build_dags()
        f = np.array(f, dtype=np.float64, order="C").reshape(self.nv, self.nnode)
        fbc = np.ascontiguousarray(fbc, dtype=np.float64).reshape(self.nv, self.nnode)
        iters = np.zeros(3, dtype=np.int32)
        meas = np.zeros(3)
        pp = None
        if fprev is not None:
            fprev = np.ascontiguousarray(fprev, dtype=np.float64).reshape(self.nv, self.nnode)
            pp = fprev.ctypes.data_as(C.c_void_p)
        st = self.lib.orc_step(self.h, f, pp, fbc, iters, meas)
        return f, iters, meas, st
