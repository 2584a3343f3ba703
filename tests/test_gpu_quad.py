"""Q1 quadrilaterals (parallelograms) on the CUDA path against the oracle.  The CUDA side
combines exact reference tables with the face normals (ElemQ1Quad); the oracle integrates
the bilinear map with tensor Gauss points.  Generations bit-exact; FP64 within 1e-12
relative (max-norm) with equal Picard counts; FP32 sweep within 2e-5."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, rel_err

pytestmark = pytest.mark.gpu


def quad_workload(nx=8, ny=6, shear=0.3, n_v=16, k_v=3, integrator="BE", knudsen=0.05):
    m = synth.rect_quad_mesh(nx, ny, shear=shear)
    x = synth.node_coords(m, 1).reshape(-1, 2)
    n = 1.0 + 0.2 * np.sin(2 * np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1])
    u = np.stack([0.1 * np.cos(np.pi * x[:, 1]), 0.05 * np.sin(np.pi * x[:, 0])], 1)
    th = 1.0 + 0.1 * np.cos(2 * np.pi * x[:, 0])
    init = np.concatenate([n[:, None], u, th[:, None]], 1)
    inflow = np.concatenate([np.ones((n.size, 1)), 0 * u, np.ones((n.size, 1))], 1)
    return synth.Workload("quad", m, 1, n_v, k_v, 6.0, knudsen, integrator, 10.0, init, inflow)


def _nut(o, U):
    d = o.dim
    nut = U.copy()
    nut[:, 1:1 + d] = U[:, 1:1 + d] / U[:, :1]
    nut[:, 1 + d] = (2 * U[:, 1 + d] / U[:, 0] - (nut[:, 1:1 + d] ** 2).sum(1)) / d
    return nut


@pytest.mark.parametrize("shear", [0.0, 0.3])
def test_quad_generations_bit_exact(shear):
    w = quad_workload(shear=shear)
    s, o = make_pair(w)
    for j in range(s.nv):
        gg, G = s.generations(j)
        go, lag, Go = o.generations(j)
        assert G == Go
        np.testing.assert_array_equal(gg, go)


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_quad_sweep_against_oracle(precision, cache):
    w = quad_workload()
    s, o = make_pair(w, precision=precision, cache_inverse=cache)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    f0, fbc = o.maxwellian(w.init), o.maxwellian(w.inflow)
    dt = s.dt
    nus = w.nu + 1.0 / dt
    s.sweep(0.0, 0.0)
    f = o.sweep(f0, o.maxwellian(_nut(o, o.moments(f0))), f0 / dt, fbc, w.nu, nus)
    assert rel_err(s.get_f(), f) < (1e-12 if precision == "fp64" else 2e-5)


@pytest.mark.parametrize("integ", ["BE", "DIRK3", "BDF2"])
def test_quad_steps_match_oracle(integ):
    w = quad_workload(integrator=integ)
    s, o = make_pair(w)
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


def test_quad_walls_and_mixed_precision():
    w = quad_workload(nx=6, ny=6, shear=0.0, integrator="DIRK3", knudsen=1e-2)
    walls = {"x+": "bounce_back", "y-": "reflect", "y+": "reflect"}
    s, o = make_pair(w, walls=walls)
    o.set_walls(walls)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, "DIRK3", 1e-8, 1000)
    st = s.step(1)
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    assert list(st.iterations)[:st.n_stages] == list(it)[:st.n_stages]
    assert rel_err(s.get_f(), f) < 1e-12
    sm = bgk.Solver.from_workload(w, walls=walls, precision="mixed")
    sm.set_state_maxwellian(w.init)
    sm.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, sm.dt, "DIRK3", 1e-12, 5000)
    f, *_ = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    stm = sm.step(1)
    assert sum(stm.iterations_fp32) > 0
    assert rel_err(sm.get_f(), f) < 1e-6


def test_quad_batch_matches_single():
    ws = [quad_workload(nx=6, ny=4), quad_workload(nx=5, ny=5, shear=0.2, n_v=12, k_v=2)]
    b = bgk.Batch(ws)
    for s, w in zip(b.instances, ws):
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
    its, sts = b.step(2)
    assert np.all(sts == 0)
    for i, w in enumerate(ws):
        s = bgk.Solver.from_workload(w)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        st = s.step(2)
        assert st.iterations[0] == its[i]
        assert rel_err(b.instances[i].get_f(), s.get_f()) < 1e-13
