"""Pins of the oracle's wall boundary conditions (Sec. 4.2: bounce-back f^bc(x, v) = f(x, -v),
reflection f^bc(x, v) = f(x, R_n v)), against facts the paper and the mathematics fix:

  - a Maxwellian at rest, uniform in space, is an exact steady state of a closed box with
    either kind of wall (it is even in every velocity component);
  - a uniform flow tangential to reflecting walls is an exact steady state, and is not one
    for bounce-back walls (the Prop. after the boundary conditions: bounce-back forces
    u = 0 at the wall, reflection only n.u = 0);
  - in a closed box with either kind of wall the number and energy fluxes through the walls
    vanish, so a converged step conserves mass and energy (Eq. discrete-cons with the wall
    traces), for non-uniform states, P1 and P2 triangles and tetrahedra.

A wrong mirror (the wrong axis flipped, bounce-back and reflection swapped, another node's
trace) breaks one of them.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_19150_b300 import synth

ALL_REFLECT = {s: "reflect" for s in ("x-", "x+", "y-", "y+", "z-", "z+")}
ALL_BOUNCE = {s: "bounce_back" for s in ("x-", "x+", "y-", "y+", "z-", "z+")}


def _oracle(mesh, kx=1, n1d=8, kv=3, L=6.0):
    o = Oracle(mesh.dim, kx, mesh.xyz, mesh.cells, n1d, kv, L)
    o.build_dags()
    return o


def _totals(o, f):
    """Integrals of (1, v, |v|^2/2) f over X x V (nodal DG: int phi_b = column sums of M)."""
    v, wt, _, _ = o.velocity()
    E = np.concatenate([np.ones((o.nv, 1)), v, 0.5 * (v * v).sum(1, keepdims=True)], axis=1)
    nd = o.ndof if hasattr(o, "ndof") else f.shape[1] // o.ncell
    tot = np.zeros(E.shape[1])
    for c in range(o.ncell):
        cell = o.cell(c)
        r = slice(c * nd, (c + 1) * nd)
        tot += E.T @ (wt[:, None] * f[:, r]) @ cell["M"].sum(axis=0)
    return tot


@pytest.mark.parametrize("walls", [ALL_REFLECT, ALL_BOUNCE], ids=["reflect", "bounce_back"])
@pytest.mark.parametrize("integ", ["BE", "DIRK3"])
def test_rest_maxwellian_is_steady_in_closed_box(walls, integ):
    m = synth.square_mesh(4, 0)
    o = _oracle(m)
    o.set_walls(walls)
    nut = np.tile([0.9, 0.0, 0.0, 1.1], (o.nnode, 1))
    f0 = o.maxwellian(nut)
    o.set_physics(20.0, 0.02, integ, tau=1e-13, lmax=400)
    f1, it, meas, st = o.step(f0, np.zeros_like(f0))
    assert st == 0
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-13 * np.abs(f0).max())


def test_rest_maxwellian_is_steady_in_closed_cube():
    m = synth.cube_mesh(2, 0)
    o = _oracle(m, n1d=6, kv=2)
    o.set_walls(ALL_REFLECT)
    nut = np.tile([1.2, 0.0, 0.0, 0.0, 0.8], (o.nnode, 1))
    f0 = o.maxwellian(nut)
    o.set_physics(5.0, 0.02, "BE", tau=1e-13, lmax=400)
    f1, it, meas, st = o.step(f0, np.zeros_like(f0))
    assert st == 0
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-13 * np.abs(f0).max())


def test_tangential_flow_is_steady_between_reflecting_walls_only():
    m = synth.square_mesh(4, 0)
    nut = np.tile([0.9, 0.4, 0.0, 1.1], ((m.cells.shape[0]) * 3, 1))
    results = {}
    for kind in ("reflect", "bounce_back"):
        o = _oracle(m)
        o.set_walls({"y-": kind, "y+": kind})
        f0 = o.maxwellian(nut)
        o.set_physics(20.0, 0.02, "BE", tau=1e-13, lmax=400)
        f1, it, meas, st = o.step(f0, f0.copy())    # x sides: inflow of the same flow
        assert st == 0
        results[kind] = np.abs(f1 - f0).max() / np.abs(f0).max()
    assert results["reflect"] < 1e-13
    assert results["bounce_back"] > 1e-4
    # a reflection across x instead of y would also disturb the flow: x walls are hit head-on
    o = _oracle(m)
    o.set_walls({"x-": "reflect", "x+": "reflect", "y-": "reflect", "y+": "reflect"})
    f0 = o.maxwellian(nut)
    o.set_physics(20.0, 0.02, "BE", tau=1e-13, lmax=400)
    f1, *_ = o.step(f0, f0.copy())
    assert np.abs(f1 - f0).max() / np.abs(f0).max() > 1e-4


@pytest.mark.parametrize("walls", [ALL_REFLECT, ALL_BOUNCE], ids=["reflect", "bounce_back"])
@pytest.mark.parametrize("case", ["p1_tri", "p2_tri", "p1_tet"])
def test_closed_box_conserves_mass_and_energy(walls, case):
    if case == "p1_tet":
        m, kx, n1d, kv = synth.cube_mesh(2, 1), 1, 6, 2
    else:
        m, kx, n1d, kv = synth.square_mesh(3, 1), (2 if case == "p2_tri" else 1), 8, 3
    o = _oracle(m, kx=kx, n1d=n1d, kv=kv)
    o.set_walls(walls)
    x = synth.node_coords(m, kx).reshape(-1, m.dim)
    d = m.dim
    n = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1])
    u = 0.2 * np.stack([np.cos(np.pi * x[:, 1])] + [np.sin(np.pi * x[:, a]) for a in range(1, d)], axis=1)
    th = 1.0 + 0.2 * x[:, 0] * x[:, 1]
    f0 = o.maxwellian(np.concatenate([n[:, None], u, th[:, None]], axis=1))
    o.set_physics(10.0, 0.01, "BE", tau=1e-13, lmax=1000)
    f1, it, meas, st = o.step(f0, np.zeros_like(f0))
    assert st == 0
    t0, t1 = _totals(o, f0), _totals(o, f1)
    assert abs(t1[0] - t0[0]) < 1e-10 * t0[0]          # mass
    assert abs(t1[-1] - t0[-1]) < 1e-10 * t0[-1]        # energy
    # the state did move (the pin is not vacuous)
    assert np.abs(f1 - f0).max() > 1e-4 * np.abs(f0).max()


def test_inflow_box_does_not_conserve_mass():
    """Control for the pin above: the same step with zero inflow loses mass."""
    m = synth.square_mesh(3, 1)
    o = _oracle(m)
    nut = np.tile([1.0, 0.0, 0.0, 1.0], (o.nnode, 1))
    f0 = o.maxwellian(nut)
    o.set_physics(10.0, 0.01, "BE", tau=1e-13, lmax=1000)
    f1, *_ = o.step(f0, np.zeros_like(f0))
    assert _totals(o, f1)[0] < (1 - 1e-3) * _totals(o, f0)[0]


@pytest.mark.parametrize("integ", ["BE", "BSTABLE2"])
@pytest.mark.parametrize("model", ["linear", "streaming"])
def test_l2_decays_in_reflecting_box(model, integ):
    """Prop. (Linear Stability) with reflecting walls: the wall terms of the L2 estimate
    balance exactly (the inflow data are the mirror's outflow trace and |v.n| is the same),
    so with the simplified Maxwellian or nu = 0 a B-stable integrator does not let
    ||f||_{L2(X x V)} grow (the paper's L2-stability experiment)."""
    m = synth.square_mesh(4, 0)
    o = _oracle(m)
    o.set_walls(ALL_REFLECT)
    x = synth.node_coords(m, 1).reshape(-1, 2)
    n = np.where(x[:, 0] < 0.5, 1.0, 0.125)
    th = np.where(x[:, 0] < 0.5, 1.0, 0.8)
    f = o.maxwellian(np.stack([n, 0 * n, 0 * n, th], axis=1))
    _, wt, _, _ = o.velocity()
    Ms = [o.cell(c)["M"] for c in range(o.ncell)]

    def l2(f):
        return sum(wt[j] * sum(f[j, c * 3:(c + 1) * 3] @ Ms[c] @ f[j, c * 3:(c + 1) * 3] for c in range(o.ncell))
                   for j in range(o.nv))
    if model == "linear":
        o.set_collision("linear")
        o.set_physics(1000.0, 0.002, integ, tau=1e-13, lmax=1000)
    else:
        o.set_physics(0.0, 0.01, integ, tau=1e-13, lmax=1000)
    prev = l2(f)
    for _ in range(3):
        f, it, meas, st = o.step(f, np.zeros_like(f))
        assert st == 0
        cur = l2(f)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def _gauss_at_grid(v, n, u, th):
    d = v.shape[1]
    return n * (2 * np.pi * th) ** (-d / 2) * np.exp(-((v - u) ** 2).sum(1) / (2 * th))


@pytest.mark.parametrize("n1d,kv", [(8, 3), (12, 2)])
def test_interpolated_maxwellian_relaxation_in_closed_box(n1d, kv):
    """Sec. 5.1.1's interpolated Maxwellian: in a closed reflecting box a uniform state
    with even velocity dependence has no transport, so a converged backward-Euler step is
    the pure relaxation f1 = (f0 + dt nu M[f1]) / (1 + dt nu), M[f1] the Maxwellian of f1's
    discrete moments evaluated at the grid points (written out here with numpy)."""
    m = synth.square_mesh(3, 0)
    o = _oracle(m, n1d=n1d, kv=kv)
    o.set_walls(ALL_REFLECT)
    o.set_collision("interpolated")
    v, wt, _, _ = o.velocity()
    # f0: a uniform, even, non-Maxwellian distribution (two bumps)
    g = np.exp(-((np.abs(v) - 1.0) ** 2).sum(1))
    f0 = np.repeat(g[:, None], o.nnode, axis=1)
    dt, nu = 0.05, 10.0
    o.set_physics(nu, dt, "BE", tau=1e-14, lmax=500)
    f1, it, meas, st = o.step(f0, np.zeros_like(f0))
    assert st == 0
    col = f1[:, 0]
    assert np.abs(f1 - col[:, None]).max() < 1e-13 * col.max()     # stays uniform
    n = wt @ col
    E = wt @ (0.5 * (v * v).sum(1) * col)
    th = 2 * E / n / v.shape[1]
    M = _gauss_at_grid(v, n, np.zeros(v.shape[1]), th)
    np.testing.assert_allclose(col, (g + dt * nu * M) / (1 + dt * nu), rtol=0, atol=1e-11 * col.max())


def test_interpolation_is_not_conservative_and_projection_is():
    """The reason the paper projects (App. B): on a coarse grid the interpolated Maxwellian
    changes the mass of a closed box in a relaxation step, the projection does not; on a
    finer grid the interpolation's defect shrinks."""
    m = synth.square_mesh(3, 0)
    defect = {}
    for n1d, kv in ((8, 1), (16, 1)):
        for kind in ("interpolated", "maxwellian"):
            o = _oracle(m, n1d=n1d, kv=kv)
            o.set_walls(ALL_REFLECT)
            o.set_collision(kind)
            v, wt, _, _ = o.velocity()
            g = np.exp(-((np.abs(v) - 1.0) ** 2).sum(1))
            f0 = np.repeat(g[:, None], o.nnode, axis=1)
            o.set_physics(10.0, 0.05, "BE", tau=1e-14, lmax=500)
            f1, it, meas, st = o.step(f0, np.zeros_like(f0))
            assert st == 0
            defect[(n1d, kind)] = abs(wt @ f1[:, 0] - wt @ g) / (wt @ g)
    assert defect[(8, "maxwellian")] < 1e-12 and defect[(16, "maxwellian")] < 1e-12
    assert defect[(8, "interpolated")] > 1e-4
    assert defect[(16, "interpolated")] < 0.5 * defect[(8, "interpolated")]


def test_row_sweep_refuses_walls():
    """A sweep of selected ordinates has no mirror rows for wall faces: the oracle refuses
    it instead of reading rows it was not given."""
    m = synth.square_mesh(3, 0)
    o = _oracle(m)
    o.set_walls(ALL_REFLECT)
    js = np.arange(4, dtype=np.int32)
    f = np.ones((4, o.nnode))
    with pytest.raises(ValueError):
        o.sweep_rows(js, f, f, f, f, 1.0, 2.0)
