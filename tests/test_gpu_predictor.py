"""The stage predictor (bgk_config.stage_predictor): a stage after the first starts its
Picard iteration from moments extrapolated across the stage abscissae instead of the
previous stage's moments.  The moments move by transport only (the collision term conserves
them), so the extrapolation is a good start; it changes where the iteration starts, not
its fixed point.  Bars: after two steps both runs have stopped on the Picard criterion
(moment change below tau = 1e-8) near the same fixed point; the distance of a stopped
iterate from the fixed point is the last change times rho / (1 - rho) for the contraction
rho, in f as in the moments, so the two agree to the bar the mixed precision holds against
FP64 (1e-6 relative, max norm); the predictor takes no more iterations;
single-stage integrators (BE, BDF2) are unchanged bit for bit; graph and eager launches
agree bit for bit."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk

from gpu_common import rel_err, small_shock_tube

pytestmark = pytest.mark.gpu


def _run(w, steps, **kw):
    s = bgk.Solver.from_workload(w, **kw)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    its = 0
    for _ in range(steps):
        st = s.step(1)
        its += sum(list(st.iterations)[:st.n_stages]) + sum(list(st.iterations_fp32)[:st.n_stages])
    return s.get_f(), its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("integ", ["DIRK2", "DIRK3", "BSTABLE2"])
def test_predictor_reaches_the_same_fixed_point(integ, precision):
    w = small_shock_tube(n=12, kx=2, n_v=16, integrator=integ)
    f0, it0 = _run(w, 2, precision=precision)
    f1, it1 = _run(w, 2, precision=precision, stage_predictor=True)
    assert 0.0 < rel_err(f1, f0) < 1e-6, rel_err(f1, f0)
    assert it1 <= it0, (it1, it0)


@pytest.mark.parametrize("integ", ["BE", "BDF2"])
def test_predictor_leaves_single_stage_steps_unchanged(integ):
    w = small_shock_tube(n=10, kx=2, n_v=16, integrator=integ)
    f0, it0 = _run(w, 2, precision="mixed")
    f1, it1 = _run(w, 2, precision="mixed", stage_predictor=True)
    np.testing.assert_array_equal(f1, f0)
    assert it1 == it0


def test_predictor_graph_equals_eager():
    w = small_shock_tube(n=10, kx=2, n_v=16, integrator="DIRK3")
    fg, itg = _run(w, 2, precision="mixed", stage_predictor=True)
    fe, ite = _run(w, 2, precision="mixed", stage_predictor=True, eager=True)
    np.testing.assert_array_equal(fg, fe)
    assert itg == ite
