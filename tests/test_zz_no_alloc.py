"""The allocation-free moments + convergence-measure entry point.

Callers that cannot call cudaMalloc (their device memory is all handed to their own pool
allocator, or they must never synchronize the device) use bgk_moments_measure_noalloc,
whose scratch is a fixed file-scope device array.  This checks it through the C ABI
against the handle's own moment reduction (bgk_get_moments_device) and its measure
against a closed form, on two calls in a row.  Collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_moments_and_measure_match_existing_entry_point():
    import torch

    from paper_2608_19150_b300 import bgk, synth

    w = synth.workload_shock_tube(n_side=8, seed=1, kx=2, n_v=16, knudsen=1e-3, integrator="BE")
    s = bgk.Solver.from_workload(w)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    dev = torch.device("cuda", 0)
    nm = s.dim + 2
    f = torch.empty(s.nv * s.nnode, dtype=torch.float64, device=dev)
    U_old = torch.empty(s.nnode * nm, dtype=torch.float64, device=dev)
    U_new = torch.empty_like(U_old)
    U_ref = torch.empty_like(U_old)
    meas = torch.zeros(1, dtype=torch.float64, device=dev)
    dt = s.dt
    for call, eps in enumerate((1e-3, 2.5e-5)):
        s.sweep(w.nu + 1.0 / dt, 1.0 / dt)
        s.get_f_device(f.data_ptr())
        s.get_moments_device(U_ref.data_ptr())
        # with U_old = (1 + eps) U every relative change is eps / (1 + eps); the momentum
        # term divides by max(|U_1|, |U_0|) and is no larger, so the measure is eps/(1+eps)
        U_old.copy_(U_ref * (1.0 + eps))
        torch.cuda.synchronize()
        bgk.moments_measure_noalloc(w.L, w.n_v, w.k_v, s.dim, s.nnode, f.data_ptr(), np.float64,
                                    U_old.data_ptr(), U_new.data_ptr(), meas.data_ptr())
        torch.cuda.synchronize()
        un, ur = U_new.cpu().numpy(), U_ref.cpu().numpy()
        err = np.abs(un - ur).max() / np.abs(ur).max()
        assert err < 1e-12, (call, err)
        expect = eps / (1.0 + eps)
        assert abs(meas.item() - expect) <= 1e-9 * expect, (call, meas.item(), expect)
    # sizes beyond the static scratch are refused, before any work is enqueued
    with pytest.raises(bgk.BgkError):
        bgk.moments_measure_noalloc(w.L, w.n_v, w.k_v, s.dim, 2_097_153, f.data_ptr(), np.float64,
                                    U_old.data_ptr(), U_new.data_ptr(), meas.data_ptr())
