"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: DAG generations bit-exact; FP64 results within 1e-12 relative (max-norm
over the array); FP32 sweep within 2e-5 relative (a handful of FP32 roundings per
local solve, amplified by at most the local condition number).
"""
import numpy as np
import pytest

from paper_2608_19150_b300 import synth

from gpu_common import make_pair, rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def workloads():
    return {
        "p1_tri": synth.workload_p1_square(n_side=8, n_v=16),
        "p2_tri": small_shock_tube(n=8, kx=2, n_v=16, integrator="BE"),
        "p1_tet_cycles": twisted_workload(3, 8),
    }


@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "p1_tet_cycles"])
def test_generations_bit_exact(name):
    w = workloads()[name]
    s, o = make_pair(w)
    lag_total = 0
    for j in range(s.nv):
        gg, G = s.generations(j)
        go, lag, Go = o.generations(j)
        lag_total += int(lag.sum())
        assert G == Go
        np.testing.assert_array_equal(gg, go)
    assert s.lagged == lag_total
    if name == "p1_tet_cycles":
        assert lag_total > 0


def test_velocity_grid_and_initial_state():
    w = synth.workload_p1_square(n_side=8, n_v=16)
    s, o = make_pair(w)
    v, wt = s.velocity()
    vo, wo, _, _ = o.velocity()
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-15)
    np.testing.assert_allclose(wt, wo, rtol=1e-15)
    s.set_state_maxwellian(w.init)
    f = s.get_f()
    fo = o.maxwellian(w.init)
    assert rel_err(f, fo) < FP64_TOL
    U = s.get_moments()
    assert rel_err(U, o.moments(fo)) < FP64_TOL


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("name", ["p1_tri", "p2_tri", "p1_tet_cycles"])
def test_one_sweep_fp64(name, cache):
    w = workloads()[name]
    s, o = make_pair(w, cache_inverse=cache)
    if cache == "on":
        assert s.cache_bytes > 0
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    dt = s.dt
    nu = w.nu
    nus = nu + 1.0 / dt     # backward Euler: the cached stage coefficient
    f = f0
    for it in range(2):
        s.sweep(0.0, 0.0)
        U = o.moments(f)
        nut = U.copy()
        d = o.dim
        nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
        nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
        Mn = o.maxwellian(nut)
        f = o.sweep(f, Mn, f0 / dt, fbc, nu, nus)
        fg = s.get_f()
        assert rel_err(fg, f) < FP64_TOL, (it, rel_err(fg, f))


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("integ", ["BE", "DIRK2", "DIRK3", "BSTABLE2", "BDF2"])
def test_time_steps_match_oracle(integ, cache):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    s, o = make_pair(w, cache_inverse=cache)
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


def test_p2_dirk3_shock_tube_step():
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3")
    s, o = make_pair(w)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, "DIRK3", 1e-8, 1000)
    st = s.step(1)
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    assert list(st.iterations) == list(it)
    assert rel_err(s.get_f(), f) < FP64_TOL
    assert rel_err(s.get_moments(), o.moments(f)) < FP64_TOL


def test_tet_step_with_cycles():
    w = twisted_workload(3, 8)
    s, o = make_pair(w)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, "BE", 1e-8, 1000)
    st = s.step(1)
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0 and st.iterations[0] == it[0]
    assert rel_err(s.get_f(), f) < FP64_TOL


def test_uniform_maxwellian_preserved_on_gpu():
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator="DIRK3")
    s, o = make_pair(w)
    nut = np.tile([0.9, 0.2, -0.1, 1.1], (s.nnode, 1))
    s.set_state_maxwellian(nut)
    s.set_inflow_maxwellian(nut)
    f0 = s.get_f()
    s.step(2)
    assert rel_err(s.get_f(), f0) < 1e-13


def test_noconv_status_is_reported():
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2)
    from paper_2608_19150_b300 import bgk
    s = bgk.Solver.from_workload(w, l_max=1)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    with pytest.raises(bgk.BgkError) as e:
        s.step(1)
    assert e.value.status == bgk.BGK_E_NOCONV


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("name", ["p2_tri", "p1_tri", "p1_tet_cycles"])
def test_fp32_sweep_against_oracle(name, cache):
    w = workloads()[name] if name != "p2_tri" else small_shock_tube(n=8, kx=2, n_v=16, integrator="BE")
    s, o = make_pair(w, precision="fp32", cache_inverse=cache)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    dt = s.dt
    nus = w.nu + 1.0 / dt
    s.sweep(0.0, 0.0)
    U = o.moments(f0)
    nut = U.copy()
    d = o.dim
    nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
    nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
    f = o.sweep(f0, o.maxwellian(nut), f0 / dt, fbc, w.nu, nus)
    assert rel_err(s.get_f(), f) < 2e-5


def test_eager_mode_matches_graph_mode_bitwise():
    from paper_2608_19150_b300 import bgk
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3")
    out = []
    for eager in (False, True):
        s = bgk.Solver.from_workload(w, eager=eager)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        st = s.step(2)
        out.append((s.get_f(), list(st.iterations)))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_fp32_storage_moments_are_fp64_accurate():
    """The compensated FP32 reduction must equal the FP64 sum of the same FP32 data
    (a seeded FP32 distribution: a Maxwellian-like profile times a random factor)."""
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="BE")
    s, o = make_pair(w, precision="fp32")
    f0 = o.maxwellian(w.init)
    r = synth.splitmix64_uniform(77, f0.size).reshape(f0.shape)
    f32 = (f0 * (0.5 + r)).astype(np.float32)
    s.set_f(f32)
    U = s.get_moments()
    Uo = o.moments(f32.astype(np.float64))
    assert rel_err(U, Uo) < 1e-13


@pytest.mark.parametrize("integ", ["BE", "DIRK3", "BDF2"])
def test_mixed_precision_reaches_the_fp64_fixed_point(integ):
    """BGK_MIXED: FP32 sweeps to the FP32 floor, then FP64 sweeps to the criterion.  The
    result matches the oracle's FP64 step to the Picard tolerance (both stop when the
    moment change is below tau, from different iterates)."""
    from paper_2608_19150_b300 import bgk
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator=integ, knudsen=1e-2)
    s = bgk.Solver.from_workload(w, precision="mixed")
    o = __import__("oracle.oracle", fromlist=["Oracle"]).Oracle.from_workload(w)
    o.build_dags()
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, integ, 1e-12, 5000)       # the oracle converged far below tau
    f = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    fprev = None
    for k in range(2):
        st = s.step(1)
        assert sum(st.iterations_fp32) > 0
        f_new, it, meas, status = o.step(f, fbc, fprev=fprev)
        assert status == 0
        if integ == "BDF2":
            fprev = f
        f = f_new
    # tau' = 1e-8 / max(1, nu dt) on the moment change; allow 1e-6 on f and on each moment
    # (n, n u, E), each relative to its own l2 norm (momentum: to max(|n u|, |n|))
    e_f = rel_err(s.get_f(), f)
    Us, Uo = s.get_moments(), o.moments(f)
    d = Us.shape[1] - 2
    e_n = np.linalg.norm(Us[:, 0] - Uo[:, 0]) / np.linalg.norm(Uo[:, 0])
    e_m = np.linalg.norm(Us[:, 1:1 + d] - Uo[:, 1:1 + d]) / max(np.linalg.norm(Uo[:, 1:1 + d]),
                                                             np.linalg.norm(Uo[:, 0]))
    e_E = np.linalg.norm(Us[:, -1] - Uo[:, -1]) / np.linalg.norm(Uo[:, -1])
    print("mixed vs FP64 oracle (%s): f %.2e  n %.2e  nu %.2e  E %.2e" % (integ, e_f, e_n, e_m, e_E))
    assert e_f < 1e-6
    assert max(e_n, e_m, e_E) < 1e-6
    # a pure FP32 run of the same problem is visibly less accurate
    s32 = bgk.Solver.from_workload(w, precision="fp32", tau=1e-6)
    s32.set_state_maxwellian(w.init)
    s32.set_inflow_maxwellian(w.inflow)
    s32.step(2)
    assert rel_err(s32.get_f(), f) > rel_err(s.get_f(), f)


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet_cycles"])
def test_fp32_fused_source_equals_source_pass(name):
    """FP32 sweeps without a cache form src = nu M + q scale inside the sweep; the result
    matches the separate source pass to FP32 rounding (the two kernels are compiled
    separately and may contract the local solve's products into FMAs differently)."""
    from paper_2608_19150_b300 import bgk
    w = workloads()[name]
    out = []
    for prefetch in (False, True):   # prefetch=True keeps the separate source pass
        s = bgk.Solver.from_workload(w, precision="fp32", cache_inverse="off", prefetch=prefetch, tau=1e-6)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        s.sweep(0.0, 0.0)
        f1 = s.get_f(np.float32)
        st = s.step(1)
        out.append((f1, s.get_f(np.float32), list(st.iterations)))
    assert rel_err(out[0][0], out[1][0].astype(np.float64)) < 2e-6
    assert rel_err(out[0][1], out[1][1].astype(np.float64)) < 2e-5


def test_fp64_storage_moments_split_sums():
    """FP64 data are summed as float pairs with compensated FP32 arithmetic; the moments
    must match the oracle's FP64 sums of the same data (seeded, signs and magnitudes
    spread over 1e-30 .. 1e3) to 1e-13."""
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="BE")
    s, o = make_pair(w)
    f0 = o.maxwellian(w.init)
    r = synth.splitmix64_uniform(91, 2 * f0.size).reshape((2,) + f0.shape)
    f = f0 * (0.5 + r[0]) * 10.0 ** np.floor(4 * r[1] - 1)
    f[:, ::97] *= -1.0
    f[3, :50] = 10.0 ** np.linspace(-30, -20, 50)
    s.set_f(f)
    U = s.get_moments()
    Uo = o.moments(f)
    assert rel_err(U, Uo) < 1e-13
    for m in range(U.shape[1]):
        assert np.abs(U[:, m] - Uo[:, m]).max() <= 1e-13 * np.abs(Uo[:, m]).max() + 1e-300


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k_v,n_v", [(1, 12), (2, 12), (4, 15)])
def test_every_velocity_degree(k_v, n_v, precision):
    """The projection is specialised per velocity degree k_v (1..4): the projected
    Maxwellian, its moments and one BE step against the oracle for each degree."""
    w = synth.workload_p1_square(n_side=6, n_v=n_v, k_v=k_v, knudsen=0.05, integrator="BE")
    s, o = make_pair(w, precision=precision, tau=1e-8 if precision == "fp64" else 1e-6)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0 = o.maxwellian(w.init)
    tol = FP64_TOL if precision == "fp64" else 2e-6
    assert rel_err(s.get_f(), f0) < tol
    assert rel_err(s.get_moments(), o.moments(f0)) < (FP64_TOL if precision == "fp64" else 1e-6)
    if precision == "fp64":
        o.set_physics(w.nu, s.dt, "BE", 1e-8, 1000)
        st = s.step(1)
        f1, it, meas, status = o.step(f0, o.maxwellian(w.inflow))
        assert status == 0 and st.iterations[0] == it[0]
        assert rel_err(s.get_f(), f1) < FP64_TOL
