"""Bounce-back and reflecting walls (Sec. 4.2) on the CUDA path against the oracle.

The CUDA side finds a wall's mirror ordinate by index arithmetic on the symmetric grid;
the oracle finds it by searching the grid for the transformed velocity.  FP64 within
1e-12 relative (max-norm) with equal Picard iteration counts, as the other parity tests.
"""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SIDES = ("x-", "x+", "y-", "y+", "z-", "z+")
WALLS = {
    "reflect": {s: "reflect" for s in SIDES},
    "bounce_back": {s: "bounce_back" for s in SIDES},
    "mixed": {"x-": "inflow", "x+": "bounce_back", "y-": "reflect", "y+": "reflect"},
}


def _pair(w, walls, **kw):
    s, o = make_pair(w, walls=walls, **kw)
    o.set_walls(walls)
    return s, o


def _run(s, o, w, integ, steps=2, tau=1e-8):
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, s.dt, integ, tau, 1000)
    f = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    fprev = None
    for k in range(steps):
        st = s.step(1)
        f_new, it, meas, status = o.step(f, fbc, fprev=fprev)
        assert status == 0
        if integ == "BDF2":
            fprev = f
        f = f_new
        nst = st.n_stages
        assert list(st.iterations)[:nst] == list(it)[:nst], (k, list(st.iterations), list(it))
        assert rel_err(s.get_f(), f) < FP64_TOL
    return f


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("integ", ["BE", "DIRK3", "BDF2"])
@pytest.mark.parametrize("kind", ["reflect", "bounce_back", "mixed"])
def test_walls_p1_triangles_match_oracle(kind, integ, cache):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    s, o = _pair(w, WALLS[kind], cache_inverse=cache)
    _run(s, o, w, integ)


def test_walls_p2_shock_tube_channel():
    """The shock tube in a channel: reflecting walls at y = 0, 1; inflow at x = 0, 1."""
    w = small_shock_tube(n=8, kx=2, n_v=16, integrator="DIRK3")
    walls = {"y-": "reflect", "y+": "reflect"}
    s, o = _pair(w, walls)
    _run(s, o, w, "DIRK3", steps=1)


@pytest.mark.parametrize("kind", ["reflect", "bounce_back"])
def test_walls_tetrahedra_match_oracle(kind):
    m = synth.cube_mesh(2, 1)
    x = synth.node_coords(m, 1).reshape(-1, 3)
    n = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(np.pi * x[:, 2])
    u = 0.2 * np.stack([np.cos(np.pi * x[:, 1]), np.sin(np.pi * x[:, 2]), np.sin(np.pi * x[:, 0])], axis=1)
    th = 1.0 + 0.2 * x[:, 0] * x[:, 1]
    init = np.concatenate([n[:, None], u, th[:, None]], axis=1)
    w = synth.Workload("cube", m, 1, 6, 2, 6.0, 1e-2, "BE", 8.0, init, init.copy())
    s, o = _pair(w, WALLS[kind])
    _run(s, o, w, "BE")


def test_walls_only_on_axis_aligned_faces_of_a_twisted_mesh():
    """The twisted cube's side faces are not axis-aligned: they stay inflow on both sides;
    its z faces are walls."""
    w = twisted_workload(3, 8)
    s, o = _pair(w, {"x-": "reflect", "x+": "reflect", "z-": "bounce_back", "z+": "reflect"})
    _run(s, o, w, "BE", steps=1)


def test_closed_box_conserves_mass_on_gpu():
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator="BE", knudsen=0.05)
    s = bgk.Solver.from_workload(w, walls=WALLS["reflect"], tau=1e-12)
    s.set_state_maxwellian(w.init)
    m0 = s.get_moments()
    s.step(3)
    m1 = s.get_moments()
    # nodal DG: the integral of n is sum over cells of (column sums of M) . n_nodes; with the
    # same mesh before and after, compare the nodal sums weighted by the oracle's masses
    from oracle.oracle import Oracle
    o = Oracle.from_workload(w)
    wts = np.concatenate([o.cell(c)["M"].sum(axis=0) for c in range(o.ncell)])
    mass0, mass1 = wts @ m0[:, 0], wts @ m1[:, 0]
    e0, e1 = wts @ m0[:, -1], wts @ m1[:, -1]
    assert abs(mass1 - mass0) < 1e-10 * mass0
    assert abs(e1 - e0) < 1e-10 * e0


@pytest.mark.parametrize("integ", ["BE", "DIRK3"])
def test_walls_fp32_and_mixed(integ):
    w = synth.workload_p1_square(n_side=8, n_v=16, integrator=integ, knudsen=1e-2)
    walls = WALLS["mixed"]
    from oracle.oracle import Oracle
    o = Oracle.from_workload(w)
    o.build_dags()
    o.set_walls(walls)
    sm = bgk.Solver.from_workload(w, precision="mixed", walls=walls)
    s32 = bgk.Solver.from_workload(w, precision="fp32", walls=walls, tau=1e-6)
    for s in (sm, s32):
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
    o.set_physics(w.nu, sm.dt, integ, 1e-12, 5000)
    f, it, meas, status = o.step(o.maxwellian(w.init), o.maxwellian(w.inflow))
    assert status == 0
    st = sm.step(1)
    assert sum(st.iterations_fp32) > 0
    s32.step(1)
    e_m, e_32 = rel_err(sm.get_f(), f), rel_err(s32.get_f(), f)
    print("walls: mixed %.2e  fp32 %.2e" % (e_m, e_32))
    assert e_m < 1e-6
    assert e_32 < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_walls_ts_equals_tgs(precision):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator="BE", knudsen=0.05)
    out = {}
    for mode in ("tgs", "ts"):
        s = bgk.Solver.from_workload(w, walls=WALLS["mixed"], sweep_mode=mode, precision=precision,
                                     tau=1e-8 if precision == "fp64" else 1e-6)
        assert s.sweep_mode == mode
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        s.step(1)
        out[mode] = s.get_f()
    assert rel_err(out["ts"], out["tgs"]) < (1e-13 if precision == "fp64" else 1e-5)


def test_sweep_range_refuses_walls():
    w = synth.workload_p1_square(n_side=4, n_v=8, k_v=3)
    s = bgk.Solver.from_workload(w, walls=WALLS["reflect"])
    s.set_state_maxwellian(w.init)
    import torch
    U = torch.zeros((s.nnode, 4), dtype=torch.float64, device="cuda")
    s.get_moments_device(U.data_ptr())
    with pytest.raises(bgk.BgkError) as e:
        s.sweep_range(0, s.nv, U.data_ptr())
    assert e.value.status == bgk.BGK_E_INVALID
