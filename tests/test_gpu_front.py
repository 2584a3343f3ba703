"""The FP32 generation sweep with the shared-memory front (k_sweep_front) against the same
sweep reading every upwind trace from global memory, and against the oracle.

The front only changes where a cell's upwind traces are read from (a shared-memory slot
written by the upwind cell earlier in the same sweep, instead of global memory), not the
arithmetic: FP32 sweeps agree with the global-read sweep to FP32 rounding (the two kernels
are compiled separately; 2e-6 relative) and with the oracle within the FP32 sweep tolerance
(2e-5); mixed-precision steps with and without it reach the same FP64 fixed point (1e-7).  Triangles P1 and P2, Q1 quadrilaterals with reflecting walls; 2D meshes of
convex cells have acyclic sweep graphs, so no edge is lagged in 2D."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, rel_err, small_shock_tube

pytestmark = pytest.mark.gpu


def _cases():
    return {"p1_tri": synth.workload_p1_square(n_side=12, n_v=16),
            "p2_tri": small_shock_tube(n=12, kx=2, n_v=16, integrator="BE"),
            "q1_sod_walls": synth.workload_sod_strip(nx=48, ny=6, n_v=16, knudsen=1e-3, integrator="BE")}


def _oracle_sweep(o, f, f0, fbc, nu, nus, dt):
    U = o.moments(f)
    nut = U.copy()
    d = o.dim
    nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
    nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
    return o.sweep(f, o.maxwellian(nut), f0 / dt, fbc, nu, nus)


@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "q1_sod_walls"])
def test_front_sweep_matches_global_sweep_and_oracle(name):
    w = _cases()[name]
    s, o = make_pair(w, precision="fp32", sweep_mode="tgs")
    g = bgk.Solver.from_workload(w, precision="fp32", sweep_mode="tgs", sweep_front=False)
    assert s.front_slots > 0 and g.front_slots == 0
    for x in (s, g):
        x.set_state_maxwellian(w.init)
        x.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    f = f0
    for it in range(3):
        s.sweep(0.0, 0.0)
        g.sweep(0.0, 0.0)
        fs, fg = s.get_f(), g.get_f()
        assert rel_err(fs, fg) < 2e-6, (it, rel_err(fs, fg))
        f = _oracle_sweep(o, f, f0, fbc, w.nu, w.nu + 1.0 / s.dt, s.dt)
        assert rel_err(fs, f) < 2e-5, (it, rel_err(fs, f))


@pytest.mark.parametrize("name", ["p2_tri", "q1_sod_walls"])
def test_mixed_steps_with_and_without_front(name):
    w = _cases()[name]
    out = []
    for front in (True, False):
        s = bgk.Solver.from_workload(w, precision="mixed", sweep_mode="tgs", sweep_front=front)
        assert (s.front_slots > 0) == front
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        st = s.step(2)
        out.append((s.get_f(), list(st.iterations), list(st.iterations_fp32)))
    # the FP32 phases may differ in rounding; both end at the FP64 fixed point
    assert rel_err(out[0][0], out[1][0]) < 1e-7


def test_front_is_skipped_where_it_does_not_apply():
    """3D meshes, FP64 sweeps and the batched instances read from global memory."""
    m = synth.cube_mesh(3, 2, 0.15)
    x = synth.node_coords(m, 1).reshape(-1, 3)
    nut = np.concatenate([np.ones((len(x), 1)), np.zeros_like(x), np.ones((len(x), 1))], axis=1)
    w3 = synth.Workload("cube", m, 1, 8, 3, 6.0, 1e-2, "BE", 8.0, nut, nut.copy())
    assert bgk.Solver.from_workload(w3, precision="fp32").front_slots == 0
    w2 = synth.workload_p1_square(n_side=8, n_v=8)
    assert bgk.Solver.from_workload(w2, precision="fp64").front_slots == 0
