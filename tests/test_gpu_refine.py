"""Picard refinement of the mixed precision (bgk_config.refine): after the first FP64-phase
sweep of a stage, each further Picard iteration f <- f + d takes d from an FP32 sweep of the
change of the source nu M; with walls (Sec. 4.2) and lagged edges (3D cycles, Sec. 4.1) the
correction also takes the wall data and the lagged inflow from the previous change of f.

In exact arithmetic the refined iterate equals the full sweep's (the sweep is linear in its
source and the iterate just swept satisfies its equations), so the two runs take the same
Picard iterations; the correction's FP32 rounding is relative to the small change d, and so
is that of the change of the projected Maxwellian, taken from its FP32 derivative at the
midpoint of two iterates (about 1e-6 of the change).  Bar, one single-stage step (BE, the
first BDF2 step) from the same state: the same iteration counts and f within 1e-10
relative (max norm) of the full-sweep run, against differences of order tau = 1e-8 between
iterates.  A later stage or step starts its FP32 phase from the previous result rounded to
floats: differences of 1e-12 then change some FP32 roundings, the two runs follow
different FP32 iterates and both stop within the Picard tolerance of the fixed point, so
multi-stage and multi-step runs are compared with an FP64 run converged to 1e-13: within
1e-6, as the mixed precision is, and within 1.5x of the full-sweep run's error.  Results
differ from the full-sweep run (the switch takes effect)."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu


def _run(w, refine, steps=2, **kw):
    s = bgk.Solver.from_workload(w, precision="mixed", refine=refine, **kw)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    its = []
    for _ in range(steps):
        st = s.step(1)
        its.append((list(st.iterations_fp32), list(st.iterations)))
    return s.get_f(), its


@pytest.mark.parametrize("integ", ["BE", "BDF2"])
def test_refinement_reaches_the_full_sweep_iterate(integ):
    w = small_shock_tube(n=12, kx=2, n_v=16, integrator=integ)
    f0, it0 = _run(w, False, steps=1)
    f1, it1 = _run(w, True, steps=1)
    assert it0 == it1
    assert max(it1[0][1]) >= 3          # several refinement iterations in a row
    d = rel_err(f1, f0)
    assert 0.0 < d < 1e-10, d


def test_refinement_with_large_first_changes():
    """The FP32 phase stopped early (floor 1e-3): the refinement then moves the moments by
    about 1e-2, so its factor changes come from both states' FP64 factors (the FP32
    derivatives serve only after an FP32 phase that ended within 1e-6), and it takes ~48
    corrections, whose FP32 sweeps' rounding adds up to ~2e-9 against the full-sweep run
    (the same with FP64 factor differences in every correction).  Bar: equal iteration
    counts, and the step as close to an FP64 step converged to 1e-13 as the full-sweep
    run is (within 1.5x plus 1e-9)."""
    w = small_shock_tube(n=12, kx=2, n_v=16, integrator="BE")
    f0, it0 = _run(w, False, steps=1, fp32_floor=1e-3)
    f1, it1 = _run(w, True, steps=1, fp32_floor=1e-3)
    p = bgk.Solver.from_workload(w, precision="fp64", tau=1e-13)
    p.set_state_maxwellian(w.init)
    p.set_inflow_maxwellian(w.inflow)
    p.step(1)
    tight = p.get_f()
    assert it0 == it1
    assert max(it1[0][1]) >= 3
    e_full, e_ref = rel_err(f0, tight), rel_err(f1, tight)
    assert e_ref < 1.5 * e_full + 1e-9, (e_ref, e_full)
    assert 0.0 < rel_err(f1, f0) < 1e-8


def test_refinement_on_the_p1_square():
    w = synth.workload_p1_square(n_side=16, seed=0, n_v=16, k_v=3, L=6.0, knudsen=1e-2)
    f0, it0 = _run(w, False, steps=1)
    f1, it1 = _run(w, True, steps=1)
    assert it0 == it1
    assert rel_err(f1, f0) < 1e-10


@pytest.mark.parametrize("integ", ["DIRK3", "BDF2"])
def test_refined_steps_stay_at_the_fp64_fixed_point(integ):
    w = small_shock_tube(n=12, kx=2, n_v=16, integrator=integ)
    ref, _ = _run(w, False, steps=3)
    p = bgk.Solver.from_workload(w, precision="fp64", tau=1e-13)
    p.set_state_maxwellian(w.init)
    p.set_inflow_maxwellian(w.inflow)
    p.step(3)
    tight = p.get_f()
    f1, _ = _run(w, True, steps=3)
    e_full, e_ref = rel_err(ref, tight), rel_err(f1, tight)
    assert e_ref < 1e-6 and e_full < 1e-6
    assert e_ref < 1.5 * e_full + 1e-9, (e_ref, e_full)


@pytest.mark.parametrize("case", ["walls", "tets_with_cycles"])
def test_refinement_with_walls_and_lagged_edges(case):
    if case == "walls":
        w = small_shock_tube(n=10, kx=2, n_v=16, integrator="BE")
        kw = dict(walls={"y-": "reflect", "y+": "reflect"})
    else:
        w = twisted_workload(3, 8)
        kw = {}
    f0, it0 = _run(w, False, steps=1, **kw)
    f1, it1 = _run(w, True, steps=1, **kw)
    assert it0 == it1
    assert max(it1[0][1]) >= 2
    d = rel_err(f1, f0)
    assert 0.0 < d < 1e-10, d


def test_refined_step_graph_equals_eager():
    w = small_shock_tube(n=10, kx=2, n_v=16, integrator="DIRK3")
    f_graph, it_graph = _run(w, True)
    f_eager, it_eager = _run(w, True, eager=True)
    assert it_graph == it_eager
    np.testing.assert_array_equal(f_graph, f_eager)
