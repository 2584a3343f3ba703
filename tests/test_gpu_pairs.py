"""Float-pair sweeps (bgk_config.hp_sweep = 2; the automatic choice in the FP64 phase of the
mixed precision) against the oracle's FP64 sweep and steps.

The pair sweep forms Mh src in the source pass, the inflow terms and x = A^-1 b with the
cached inverse stored as float pairs, in compensated FP32 arithmetic (TwoProduct by fma,
TwoSum, renormalised pairs): about 2^-44 relative per operation (5.7e-14), a few dozen
operations per local solve, amplified by at most the local condition number.  The bar is
the FP64 one, 1e-12 relative (max-norm over the array), with equal Picard counts; the pair
results are not bit-identical to the FP64 sweep's (they come from other arithmetic)."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, shard, synth

from gpu_common import make_pair, rel_err, small_shock_tube, twisted_workload
from test_gpu_quad import quad_workload

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _cases():
    return {
        "p1_tri": synth.workload_p1_square(n_side=8, n_v=16),
        "p2_tri": small_shock_tube(n=8, kx=2, n_v=16, integrator="BE"),
        "p1_tet_cycles": twisted_workload(3, 8),
        "q1": quad_workload(),
    }


def _nut(o, U):
    d = o.dim
    nut = U.copy()
    nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
    nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
    return nut


@pytest.mark.parametrize("mode", ["tgs", "ts"])
@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "p1_tet_cycles", "q1"])
def test_pair_sweeps_match_the_oracle(name, mode):
    w = _cases()[name]
    s, o = make_pair(w, hp_sweep="pairs", cache_inverse="on", sweep_mode=mode)
    assert s.cache_bytes > 0 and s.sweep_mode == mode
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    nus = w.nu + 1.0 / s.dt     # backward Euler: the cached stage coefficient
    f = f0
    for it in range(2):
        s.sweep(0.0, 0.0)
        Mn = o.maxwellian(_nut(o, o.moments(f)))
        f = o.sweep(f, Mn, f0 / s.dt, fbc, w.nu, nus)
        assert rel_err(s.get_f(), f) < TOL, (it, rel_err(s.get_f(), f))


@pytest.mark.parametrize("integ", ["BE", "DIRK2", "DIRK3", "BSTABLE2", "BDF2"])
def test_pair_steps_match_the_oracle(integ):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    s, o = make_pair(w, hp_sweep="pairs", cache_inverse="on")
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
        assert rel_err(s.get_f(), f) < TOL


def test_pair_and_fp64_sweeps_differ_by_rounding_only():
    """The switch takes effect (the results differ) and the two agree to the bar."""
    w = small_shock_tube(n=12, kx=2, n_v=16, integrator="DIRK3")
    out = {}
    for hp in ("fp64", "pairs"):
        s = bgk.Solver.from_workload(w, hp_sweep=hp, cache_inverse="on")
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        s.sweep(0.0, 0.0)
        out[hp] = s.get_f()
    d = rel_err(out["pairs"], out["fp64"])
    assert 0.0 < d < TOL, d


def test_mixed_precision_runs_its_fp64_phase_in_pairs():
    """BGK_MIXED chooses pairs for its FP64 phase by default: same Picard counts as with
    FP64 arithmetic there, results apart by rounding only.  Every FP64-phase iteration a
    full sweep (no refinement), so that each iteration compares the two arithmetics."""
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3")
    res = {}
    for hp in ("auto", "fp64", "pairs"):
        s = bgk.Solver.from_workload(w, precision="mixed", hp_sweep=hp, refine=False)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        st = s.step(2)
        res[hp] = (s.get_f(), list(st.iterations), list(st.iterations_fp32))
    np.testing.assert_array_equal(res["auto"][0], res["pairs"][0])
    assert res["auto"][1:] == res["fp64"][1:]
    d = rel_err(res["auto"][0], res["fp64"][0])
    assert 0.0 < d < TOL, d


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet_cycles"])
def test_pair_range_sweeps_reproduce_the_full_sweep(name):
    import torch
    w = _cases()[name]
    s1 = bgk.Solver.from_workload(w, hp_sweep="pairs", cache_inverse="on")
    s1.set_state_maxwellian(w.init)
    s1.set_inflow_maxwellian(w.inflow)
    U = torch.empty((s1.nnode, s1.dim + 2), dtype=torch.float64, device="cuda")
    s1.get_moments_device(U.data_ptr())
    s1.sweep(0.0, 0.0)
    f_full = s1.get_f()
    s2 = bgk.Solver.from_workload(w, hp_sweep="pairs", cache_inverse="on")
    s2.set_state_maxwellian(w.init)
    s2.set_inflow_maxwellian(w.inflow)
    for a, b in shard.ordinate_shards(w.n_v, s2.dim, 3):
        s2.sweep_range(a, b, U.data_ptr())
    np.testing.assert_array_equal(s2.get_f(), f_full)


@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "q1"])
def test_pair_front_equals_global_reads(name):
    """The float-pair sweep with the shared-memory front (k_sweep_front_pair) gives the
    global-memory pair sweep's results bit for bit: the front holds the pairs the reader
    would split from the upwind cell's FP64 values."""
    w = _cases()[name]
    out = []
    for front in (True, False):
        s = bgk.Solver.from_workload(w, hp_sweep="pairs", cache_inverse="on", sweep_front=front)
        assert (s.front_slots > 0) == front
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        s.sweep(0.0, 0.0)
        s.sweep(0.0, 0.0)
        out.append(s.get_f())
    np.testing.assert_array_equal(out[0], out[1])
