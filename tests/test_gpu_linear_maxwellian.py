"""The simplified (linear) Maxwellian, Eq. linear-Maxwellian (N_h = n / |V| at every ordinate),
on the CUDA path against the oracle, and the L2 decay of Prop. (Linear Stability), case (ii).

Tolerances as in the other parity tests: FP64 within 1e-12 relative (max-norm), with
equal Picard iteration counts.
"""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _pair(w, **kw):
    s, o = make_pair(w, collision="linear", **kw)
    o.set_collision("linear")
    return s, o


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("integ", ["BE", "DIRK3", "BSTABLE2", "BDF2"])
def test_linear_maxwellian_steps_match_oracle(integ, cache):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    s, o = _pair(w, cache_inverse=cache)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, integ, 1e-8, 1000)
    f = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    fprev = None
    for k in range(2):
        st = s.step(1)
        f_new, it, meas, status = o.step(f, fbc, fprev=fprev)
        assert status == 0
        if integ == "BDF2":
            fprev = f
        f = f_new
        nst = st.n_stages
        assert list(st.iterations)[:nst] == list(it)[:nst], (k, list(st.iterations), list(it))
        assert rel_err(s.get_f(), f) < FP64_TOL


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet_cycles"])
def test_linear_maxwellian_p2_and_tet(name):
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
    assert rel_err(s.get_f(), f) < FP64_TOL


def test_linear_maxwellian_mixed_precision_reaches_fp64_fixed_point():
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator="DIRK3", knudsen=1e-2)
    s = bgk.Solver.from_workload(w, precision="mixed", collision="linear")
    o = __import__("oracle.oracle", fromlist=["Oracle"]).Oracle.from_workload(w)
    o.build_dags()
    o.set_collision("linear")
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, "DIRK3", 1e-12, 5000)
    st = s.step(1)
    assert sum(st.iterations_fp32) > 0
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    assert rel_err(s.get_f(), f) < 1e-6


def test_constant_state_is_steady_on_gpu():
    """Constant f with the same constant inflow is a steady state of the linear model."""
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator="DIRK3")
    s = bgk.Solver.from_workload(w, collision="linear")
    f0 = np.full((s.nv, s.nnode), 0.37)
    s.set_f(f0)
    s.set_inflow(f0)
    s.step(2)
    assert np.abs(s.get_f() - 0.37).max() < 1e-13


def test_raw_inflow_matches_maxwellian_inflow():
    """bgk_set_inflow with the projected Maxwellian's nodal values gives the same step as
    bgk_set_inflow_maxwellian."""
    w = synth.workload_p1_square(n_side=6, n_v=12, integrator="BE")
    a = bgk.Solver.from_workload(w)
    b = bgk.Solver.from_workload(w)
    for s in (a, b):
        s.set_state_maxwellian(w.init)
    a.set_inflow_maxwellian(w.inflow)
    b.set_state_maxwellian(w.inflow)
    fin = b.get_f()
    b.set_state_maxwellian(w.init)
    b.set_inflow(fin)
    a.step(1)
    b.step(1)
    np.testing.assert_array_equal(a.get_f(), b.get_f())


@pytest.mark.parametrize("integ", ["BE", "BSTABLE2"])
def test_l2_norm_decays_with_zero_inflow(integ):
    """Prop. (Linear Stability), case (ii): nu = 1000, zero inflow, B-stable integrator."""
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator=integ)
    o = __import__("oracle.oracle", fromlist=["Oracle"]).Oracle.from_workload(w)
    s = bgk.Solver(w.mesh.dim, w.kx, w.mesh.xyz, w.mesh.cells, w.n_v, w.k_v, w.L, 1000.0,
                   integrator=integ, dt=0.002, collision="linear", tau=1e-12, l_max=1000)
    s.set_state_maxwellian(w.init)
    s.set_inflow(np.zeros((s.nv, s.nnode)))
    _, wt, _, _ = o.velocity()
    Ms = [o.cell(c)["M"] for c in range(o.ncell)]
    nl = Ms[0].shape[0]

    def l2(f):
        return sum(wt[j] * sum(f[j, c * nl:(c + 1) * nl] @ Ms[c] @ f[j, c * nl:(c + 1) * nl]
                               for c in range(o.ncell)) for j in range(o.nv))
    prev = l2(s.get_f())
    for _ in range(4):
        s.step(1)
        cur = l2(s.get_f())
        assert cur < prev
        prev = cur


def test_unknown_collision_is_rejected():
    w = synth.workload_p1_square(n_side=4, n_v=8)
    with pytest.raises(KeyError):
        bgk.Solver.from_workload(w, collision="bogus")
