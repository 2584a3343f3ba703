"""Parity at the workloads' full sizes, on sampled ordinates the oracle computes one by one.

- 2D-2V shock tube, 128x128 squares (32,768 P2 triangles), 32x32 velocities: generations
  bit-exact and one FP64 sweep within 1e-12 on sampled ordinates (the launch configuration
  the benchmark times: local-inverse cache on).
- 3D-3V bump, 24^3 cubes (82,944 tetrahedra), 16^3 velocities, FP32 storage (5.4 GB):
  generations bit-exact on sampled ordinates; one FP32 sweep within 2e-5 of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_19150_b300 import bgk, synth

pytestmark = pytest.mark.gpu


def _rows_from_device(s, js, dtype):
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    buf = torch.empty((s.nv, s.nnode), dtype=td, device="cuda")
    s.get_f_device(buf.data_ptr(), dtype)
    torch.cuda.synchronize()
    return buf[torch.as_tensor(js, device="cuda")].double().cpu().numpy()


def _check(w, precision, js, tol):
    s = bgk.Solver.from_workload(w, precision=precision)
    o = Oracle.from_workload(w)
    o.build_dags_for(js)
    for j in js:
        gg, G = s.generations(j)
        go, _, Go = o.generations(j)
        assert G == Go
        np.testing.assert_array_equal(gg, go)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    s.sweep(0.0, 0.0)            # first-stage coefficient, the cached inverses
    fg = _rows_from_device(s, js, s.fdtype)
    f0 = o.maxwellian_rows(w.init, js)
    fbc = o.maxwellian_rows(w.inflow, js)
    # the Maxwellian of the initial state's moments is the initial state itself (the
    # projection reproduces the moments exactly, App. B; pinned on the oracle side)
    Mn = f0
    from oracle.oracle import tableau
    A, _, _ = tableau(w.integrator if w.integrator != "BDF2" else "BE")
    dt = s.dt
    nus = w.nu + 1.0 / (dt * A[0, 0])
    fo = o.sweep_rows(js, f0, Mn, f0 / (dt * A[0, 0]), fbc, w.nu, nus)
    err = np.abs(fg - fo).max() / np.abs(fo).max()
    assert err < tol, err
    return s


def test_shock_tube_full_size_sampled():
    w = synth.workload_shock_tube(n_side=128, seed=1, kx=2, n_v=32, knudsen=1e-3, integrator="DIRK3")
    js = [0, 77, 511, 528, 1023]
    s = _check(w, "fp64", js, 1e-12)
    assert s.cache_bytes > 0


def test_3d_bump_full_size_sampled_fp32():
    w = synth.workload_3d_bump(n_side=24, seed=2, n_v=16)
    js = [0, 1365, 2047, 2730, 4095]
    _check(w, "fp32", js, 2e-5)
