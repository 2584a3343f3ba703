"""The interpolated Maxwellian (Sec. 5.1.1: the Maxwellian of the current moments evaluated
at the grid velocities, the non-conservative alternative to the projection) on the CUDA
path against the oracle: FP64 within 1e-12 relative (max-norm) with equal Picard counts.
The CUDA side forms it as a product of 1D Gaussians per dimension (the factor array the
sweep reads); the oracle evaluates the d-dimensional formula directly."""
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu


def _pair(w, **kw):
    s, o = make_pair(w, collision="interpolated", **kw)
    o.set_collision("interpolated")
    return s, o


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("integ", ["BE", "DIRK3", "BDF2"])
def test_interpolated_steps_match_oracle(integ, cache):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    s, o = _pair(w, cache_inverse=cache)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, integ, 1e-8, 1000)
    f, fbc, fprev = o.maxwellian(w.init), o.maxwellian(w.inflow), None
    for k in range(2):
        st = s.step(1)
        f_new, it, meas, status = o.step(f, fbc, fprev=fprev)
        assert status == 0
        if integ == "BDF2":
            fprev = f
        f = f_new
        assert list(st.iterations)[:st.n_stages] == list(it)[:st.n_stages]
        assert rel_err(s.get_f(), f) < 1e-12


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet_cycles"])
def test_interpolated_p2_and_tet(name):
    w = (small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3") if name == "p2_tri"
         else twisted_workload(3, 8))
    s, o = _pair(w)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, w.integrator, 1e-8, 1000)
    st = s.step(1)
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    assert list(st.iterations)[:st.n_stages] == list(it)[:st.n_stages]
    assert rel_err(s.get_f(), f) < 1e-12


def test_interpolated_mixed_precision():
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator="DIRK3", knudsen=1e-2)
    s = bgk.Solver.from_workload(w, precision="mixed", collision="interpolated")
    from oracle.oracle import Oracle
    o = Oracle.from_workload(w)
    o.build_dags()
    o.set_collision("interpolated")
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, "DIRK3", 1e-12, 5000)
    st = s.step(1)
    assert sum(st.iterations_fp32) > 0
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    assert rel_err(s.get_f(), f) < 1e-6
