"""The two sweep algorithms (Sec. 4.1): TS (one thread per ordinate walks its whole
schedule) and TGS (a CTA per ordinate walks the generations, the cells of a generation in
parallel) do the same operations per cell in a valid topological order.  They agree to
rounding (the two kernels are compiled separately and may contract the local assembly's
products into FMAs differently; with the local-inverse cache the results are identical):
one sweep and two steps, FP64 with and without the cache, FP32, mixed, triangles P1/P2 and
tetrahedra with cycles.  The default is TGS, also on a strip (narrow generations), where TS
was measured 8x slower."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu


def _cases():
    return {"p2_tri": small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3"),
            "p1_strip": synth.workload_strip(nx=48, ny=2, n_v=16, integrator="BDF2"),
            "p1_tet": twisted_workload(3, 8),
            "q1_sod": synth.workload_sod_strip(nx=48, ny=6, n_v=16, knudsen=1.0, integrator="DIRK2")}


@pytest.mark.parametrize("precision,cache", [("fp64", "on"), ("fp64", "off"), ("fp32", "off"), ("mixed", "auto")])
@pytest.mark.parametrize("name", ["p2_tri", "p1_strip", "p1_tet", "q1_sod"])
def test_ts_equals_tgs(name, precision, cache):
    w = _cases()[name]
    tau = 1e-6 if precision == "fp32" else 1e-8
    out = []
    for mode in ("tgs", "ts"):
        s = bgk.Solver.from_workload(w, precision=precision, cache_inverse=cache, sweep_mode=mode, tau=tau)
        assert s.sweep_mode == mode
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        s.sweep(0.0, 0.0)
        f1 = s.get_f(s.fdtype)
        s.set_state_maxwellian(w.init)
        st = s.step(2)
        out.append((f1, s.get_f(s.fdtype), list(st.iterations), list(st.iterations_fp32)))
    if precision == "fp64" and cache == "on":
        np.testing.assert_array_equal(out[0][0], out[1][0])
        np.testing.assert_array_equal(out[0][1], out[1][1])
    tol = 2e-6 if precision == "fp32" else 1e-12
    assert rel_err(out[1][0], out[0][0].astype(np.float64)) < tol
    assert rel_err(out[1][1], out[0][1].astype(np.float64)) < tol
    if precision == "fp64":
        assert out[0][2] == out[1][2]


def test_default_is_tgs():
    strip = bgk.Solver.from_workload(synth.workload_strip(nx=256, ny=1, n_v=16))
    square = bgk.Solver.from_workload(small_shock_tube(n=16, kx=2, n_v=16))
    assert strip.sweep_mode == "tgs" and square.sweep_mode == "tgs"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_sweep_restores_state_and_steps_like_the_chosen_mode(precision):
    """bgk_autotune_sweep times TGS and TS on the current state, keeps the faster, restores
    the state and captures the step graphs again: a step afterwards equals a step of a
    solver created with the chosen algorithm (up to rounding)."""
    from paper_2608_19150_b300 import bgk, synth
    w = synth.workload_sod_strip(nx=64, ny=6, n_v=16, knudsen=1.0)
    s = bgk.Solver.from_workload(w, precision=precision)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = s.get_f()
    t = s.autotune_sweep(2)
    assert t["tgs"] > 0 and t["ts"] > 0
    assert s.sweep_mode == ("ts" if t["ts"] < t["tgs"] else "tgs")
    np.testing.assert_array_equal(s.get_f(), f0)
    st = s.step(2)
    r = bgk.Solver.from_workload(w, precision=precision, sweep_mode=s.sweep_mode)
    r.set_state_maxwellian(w.init)
    r.set_inflow_maxwellian(w.inflow)
    str_ = r.step(2)
    if precision == "fp64":
        assert list(st.iterations) == list(str_.iterations)
        assert rel_err(s.get_f(), r.get_f()) < 1e-13
    else:   # the FP32 shadow chose for itself: the same fixed point to the tolerance
        assert rel_err(s.get_f(), r.get_f()) < 1e-6


def test_autotune_needs_a_state():
    from paper_2608_19150_b300 import bgk, synth
    s = bgk.Solver.from_workload(synth.workload_p1_square(n_side=4, n_v=8))
    with pytest.raises(bgk.BgkError) as e:
        s.autotune_sweep()
    assert e.value.status == bgk.BGK_E_INVALID


def _oracle_sweep(o, f, f0, fbc, nu, nus, dt):
    """One oracle sweep from iterate f with the Maxwellian of f's moments, q = f0 / dt."""
    U = o.moments(f)
    nut = U.copy()
    d = o.dim
    nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
    nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
    return o.sweep(f, o.maxwellian(nut), f0 / dt, fbc, nu, nus)


def _oracle_cases():
    return {"p1_tri": synth.workload_p1_square(n_side=8, n_v=16),
            "p2_tri": small_shock_tube(n=8, kx=2, n_v=16, integrator="BE"),
            "p1_tet_cycles": twisted_workload(3, 8),
            "q1_sod_walls": synth.workload_sod_strip(nx=32, ny=6, n_v=16, knudsen=1e-3, integrator="BE")}


@pytest.mark.parametrize("precision,cache", [("fp64", "on"), ("fp64", "off"), ("fp32", "off")])
@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "p1_tet_cycles", "q1_sod_walls"])
def test_ts_matches_oracle(name, precision, cache):
    """TS (Sec. 4.1) against the oracle's sweep, element by element: two sweeps from the
    initial state (the second reads the first's lagged and wall values), FP64 at 1e-12
    and FP32 at 2e-5 (the generation sweep's tolerances)."""
    from gpu_common import make_pair
    w = _oracle_cases()[name]
    s, o = make_pair(w, precision=precision, cache_inverse=cache, sweep_mode="ts")
    assert s.sweep_mode == "ts"
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    dt = s.dt
    f = f0
    tol = 2e-5 if precision == "fp32" else 1e-12
    for it in range(2):
        s.sweep(0.0, 0.0)
        f = _oracle_sweep(o, f, f0, fbc, w.nu, w.nu + 1.0 / dt, dt)
        err = rel_err(s.get_f(), f)
        assert err < tol, (it, err)
