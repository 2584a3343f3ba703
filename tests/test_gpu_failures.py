"""Failure reporting without GPU faults: a non-physical state (negative density from the
caller's f) is reported as BGK_E_NONPHYSICAL by the step and the sweep, the handle stays
usable afterwards, and l_max is reported as BGK_E_NOCONV (test_gpu_parity).  The kernels
contain no device-side spin-waits (CTA barriers only), so BGK_E_TIMEOUT has no source."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_nonphysical_state_is_reported_and_the_handle_recovers(precision):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, knudsen=0.05, integrator="DIRK3")
    tau = 1e-6 if precision == "fp32" else 1e-8
    s = bgk.Solver.from_workload(w, precision=precision, tau=tau)
    s.set_inflow_maxwellian(w.inflow)
    s.set_state_maxwellian(w.init)
    good = s.get_f(np.float64)
    bad = good.copy()
    bad[:, :9] = -bad[:, :9]                 # n < 0 at the first cell's nodes
    s.set_f(bad.astype(s.fdtype))
    with pytest.raises(bgk.BgkError) as e:
        s.step(1)
    assert e.value.status == bgk.BGK_E_NONPHYSICAL
    with pytest.raises(bgk.BgkError) as e:
        s.sweep(0.0, 0.0)
    assert e.value.status == bgk.BGK_E_NONPHYSICAL
    # a valid state afterwards steps as a fresh handle does
    s.set_state_maxwellian(w.init)
    st = s.step(1)
    r = bgk.Solver.from_workload(w, precision=precision, tau=tau)
    r.set_inflow_maxwellian(w.inflow)
    r.set_state_maxwellian(w.init)
    st_r = r.step(1)
    assert list(st.iterations) == list(st_r.iterations)
    assert rel_err(s.get_f(), r.get_f()) == 0.0
