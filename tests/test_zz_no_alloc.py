"""The allocation-free moments + convergence-measure entry point.

Callers that cannot call cudaMalloc (their device memory is all handed to their own pool
allocator, or they must never synchronize the device) use bgk_moments_measure_noalloc,
whose scratch is a fixed file-scope device array.  This checks it through the C ABI
against the handle's own moment reduction (bgk_get_moments_device) and its measure
against a closed form, on two calls in a row, for FP64 and FP32 data, triangles (2D) and
tetrahedra (3D).  Collected last on purpose.
"""
import numpy as np
import pytest

from paper_2608_19150_b300 import synth

pytestmark = pytest.mark.gpu


def _tet_workload():
    m = synth.cube_mesh(3, 2, 0.15)
    x = synth.node_coords(m, 1).reshape(-1, 3)
    n = 1.0 + 0.5 * np.exp(-((x - 0.5) ** 2).sum(1) / 0.02)
    u = np.zeros_like(x)
    th = np.ones_like(n)
    init = np.concatenate([n[:, None], u, th[:, None]], axis=1)
    inflow = np.concatenate([np.ones((n.size, 1)), u, th[:, None]], axis=1)
    return synth.Workload("bump3d_small", m, 1, 8, 3, 6.0, 1e-2, "BE", 8.0, init, inflow)


CASES = {
    "p2tri_fp64": (lambda: synth.workload_shock_tube(n_side=8, seed=1, kx=2, n_v=16, knudsen=1e-3,
                                                     integrator="BE"), "fp64"),
    "p2tri_fp32": (lambda: synth.workload_shock_tube(n_side=8, seed=1, kx=2, n_v=16, knudsen=1e-3,
                                                     integrator="BE"), "fp32"),
    "p1tet_fp64": (_tet_workload, "fp64"),
    "p1tet_fp32": (_tet_workload, "fp32"),
}


# The handle sums FP32 data with compensated float pairs (about 2^-47 relative), the
# allocation-free kernel converts to FP64 and sums in FP64: both are FP64-accurate sums of
# the same values, so they agree to 1e-12 relative like the FP64 branch.
TOL = 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_moments_and_measure_match_existing_entry_point(case):
    import torch

    from paper_2608_19150_b300 import bgk

    make, precision = CASES[case]
    w = make()
    s = bgk.Solver.from_workload(w, precision=precision)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    dev = torch.device("cuda", 0)
    nm = s.dim + 2
    fdt = np.float32 if precision == "fp32" else np.float64
    f = torch.empty(s.nv * s.nnode, dtype=torch.float32 if precision == "fp32" else torch.float64, device=dev)
    U_old = torch.empty(s.nnode * nm, dtype=torch.float64, device=dev)
    U_new = torch.empty_like(U_old)
    U_ref = torch.empty_like(U_old)
    meas = torch.zeros(1, dtype=torch.float64, device=dev)
    dt = s.dt
    for call, eps in enumerate((1e-3, 2.5e-5)):
        s.sweep(w.nu + 1.0 / dt, 1.0 / dt)
        s.get_f_device(f.data_ptr(), fdt)
        s.get_moments_device(U_ref.data_ptr())
        # with U_old = (1 + eps) U every relative change is eps / (1 + eps); the momentum
        # term divides by max(|U_1|, |U_0|) and is no larger, so the measure is eps/(1+eps)
        U_old.copy_(U_ref * (1.0 + eps))
        torch.cuda.synchronize()
        bgk.moments_measure_noalloc(w.L, w.n_v, w.k_v, s.dim, s.nnode, f.data_ptr(), fdt,
                                    U_old.data_ptr(), U_new.data_ptr(), meas.data_ptr())
        torch.cuda.synchronize()
        un, ur = U_new.cpu().numpy(), U_ref.cpu().numpy()
        err = np.abs(un - ur).max() / np.abs(ur).max()
        assert err < TOL, (case, call, err)
        expect = eps / (1.0 + eps)
        assert abs(meas.item() - expect) <= 1e-9 * expect, (case, call, meas.item(), expect)
    # sizes beyond the static scratch are refused, before any work is enqueued
    with pytest.raises(bgk.BgkError):
        bgk.moments_measure_noalloc(w.L, w.n_v, w.k_v, s.dim, 2_097_153, f.data_ptr(), fdt,
                                    U_old.data_ptr(), U_new.data_ptr(), meas.data_ptr())
    s.close()
