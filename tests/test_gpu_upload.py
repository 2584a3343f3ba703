"""Overlapped input of the next state (bgk_upload_f_async / bgk_set_f_uploaded): the staged
state gives the same step as bgk_set_f of the same host data, bit for bit, also when the
next upload is queued while a step runs; misuse is refused with BGK_E_INVALID."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk

from gpu_common import small_shock_tube

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    s = bgk.Solver.from_workload(w, **kw)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    return s


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_uploaded_state_steps_like_set_f(precision):
    import torch
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3")
    s = _solver(w, precision=precision, tau=1e-6 if precision == "fp32" else 1e-8)
    s.step(1)
    dt = np.float32 if precision == "fp32" else np.float64
    f_in = s.get_f(dt)
    host = torch.from_numpy(f_in.copy()).pin_memory()
    ref = []
    for _ in range(2):
        s.set_f(f_in)
        s.step(1)
        ref.append(s.get_f(dt))
    out = []
    s.upload_f_async(host.data_ptr(), dt)
    for k in range(2):
        s.set_f_uploaded()
        if k == 0:
            s.upload_f_async(host.data_ptr(), dt)       # queued while the next step runs
        s.step(1)
        out.append(s.get_f(dt))
    for a, b in zip(ref, out):
        np.testing.assert_array_equal(a, b)


def test_upload_misuse_is_refused():
    import torch
    w = small_shock_tube(n=6, kx=1, n_v=8, integrator="BE")
    s = _solver(w)
    with pytest.raises(bgk.BgkError):
        s.set_f_uploaded()                           # nothing uploaded
    host = torch.zeros(s.nv * s.nnode, dtype=torch.float32).pin_memory()
    with pytest.raises(bgk.BgkError):
        s.upload_f_async(host.data_ptr(), np.float32)  # the handle stores FP64
