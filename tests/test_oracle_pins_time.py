"""Pins of the oracle's time integration (Sec. 3.5: stage source Eq. q-stages, recursive
stage derivative Eq. dirk-recursive-def, final combination Eq. dirk-n; App. A tableaus;
BDF2 as read in the design notes: (3 f^{n+1} - 4 f^n + f^{n-1}) / (2 dt) = F(f^{n+1}),
first step backward Euler).

1. Transport-free relaxation.  A spatially uniform, velocity-even distribution in a closed
   box with reflecting walls has no transport (no jumps at interior faces; a wall returns
   the even f unchanged), and the collision term conserves its moments, so its Maxwellian
   M stays fixed and every node obeys df/dt = nu (M - f).  One step of a Runge-Kutta method
   (A, b) then gives f^1 - M = R(-nu dt) (f^0 - M) with the stability function
   R(z) = 1 + z b^T (I - z A)^{-1} 1, and BDF2 gives e^{n+1} = (4 e^n - e^{n-1}) /
   (3 + 2 nu dt), e = f - M (e^1 = e^0 / (1 + nu dt) from its backward-Euler start).
   The tableaus are the printed ones of App. A (the DIRK3 constant from its cubic).
2. Temporal order.  Free streaming (nu = 0) with time-independent inflow data on a fixed
   mesh: the error against a fine-step reference falls like dt^p with p the method's order
   (1, 2, 3, 3, 2 for BE, DIRK2, DIRK3, the B-stable DIRK, BDF2).
A wrong coupling coefficient, weight or BDF coefficient in the oracle's step fails (1); a
method whose weights do not sum to one fails (2)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_19150_b300 import synth


def _tableau(name):
    """(A, b) as printed in App. A (DIRK3: gamma the root of 6x^3 - 18x^2 + 9x - 1 near
    0.4358665, b_1 = -3 gamma^2 / 2 + 4 gamma - 1/4, b_2 = 3 gamma^2 / 2 - 5 gamma + 5/4,
    b_3 = gamma, stiffly accurate)."""
    if name == "BE":
        return np.array([[1.0]]), np.array([1.0])
    if name == "DIRK2":
        g = 1.0 - np.sqrt(2.0) / 2.0
        return np.array([[g, 0.0], [1.0 - g, g]]), np.array([1.0 - g, g])
    if name == "DIRK3":
        roots = np.roots([6.0, -18.0, 9.0, -1.0])
        g = float(next(r.real for r in roots if abs(r.imag) < 1e-12 and 0.43 < r.real < 0.44))
        b1 = -1.5 * g * g + 4.0 * g - 0.25
        b2 = 1.5 * g * g - 5.0 * g + 1.25
        return np.array([[g, 0, 0], [(1.0 - g) / 2.0, g, 0], [b1, b2, g]]), np.array([b1, b2, g])
    if name == "BSTABLE2":
        g = (3.0 + np.sqrt(3.0)) / 6.0
        return np.array([[g, 0.0], [1.0 - 2.0 * g, g]]), np.array([0.5, 0.5])
    raise KeyError(name)


def _stability(A, b, z):
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


def _relaxation_box(nu, dt, integ):
    """Oracle on a closed reflecting box (2x2 squares, P1), 8x8 velocities on [-4, 4]^2;
    f^0 uniform in space, even in each velocity component, not a Maxwellian."""
    m = synth.square_mesh(2, 3, 0.0)
    o = Oracle(2, 1, m.xyz, m.cells, 8, 3, 4.0)
    o.set_walls({side: "reflect" for side in ("x-", "x+", "y-", "y+")})
    v, _, _, _ = o.velocity()
    g = np.exp(-v[:, 0] ** 2 / 1.4 - v[:, 1] ** 2 / 2.8) + 0.2 * np.exp(-(v ** 2).sum(1) / 0.6)
    f0 = np.repeat(g[:, None], o.nnode, axis=1)
    U = o.moments(f0)
    nut = U.copy()
    nut[:, 1:3] = U[:, 1:3] / U[:, :1]
    nut[:, 3] = (2.0 * U[:, 3] / U[:, 0] - (nut[:, 1:3] ** 2).sum(1)) / 2.0
    M = o.maxwellian(nut)
    o.set_physics(nu, dt, integ, 1e-14, 1000)
    return o, f0, M


@pytest.mark.parametrize("nu,dt", [(5.0, 0.1), (40.0, 0.05)])
@pytest.mark.parametrize("integ", ["BE", "DIRK2", "DIRK3", "BSTABLE2"])
def test_relaxation_step_equals_stability_function(integ, nu, dt):
    o, f0, M = _relaxation_box(nu, dt, integ)
    assert np.abs(f0 - M).max() > 0.1            # far from equilibrium: R(z) is visible
    f1, _, _, status = o.step(f0, f0)
    assert status == 0
    A, b = _tableau(integ)
    expect = M + _stability(A, b, -nu * dt) * (f0 - M)
    err = np.abs(f1 - expect).max() / np.abs(expect).max()
    assert err < 1e-12, err


@pytest.mark.parametrize("nu,dt", [(5.0, 0.1), (40.0, 0.05)])
def test_bdf2_relaxation_recurrence(nu, dt):
    o, f0, M = _relaxation_box(nu, dt, "BDF2")
    f1, _, _, st1 = o.step(f0, f0)                 # start-up: backward Euler
    f2, _, _, st2 = o.step(f1, f0, fprev=f0)
    f3, _, _, st3 = o.step(f2, f0, fprev=f1)
    assert st1 == st2 == st3 == 0
    e = [f0 - M]
    e.append(e[0] / (1.0 + nu * dt))
    for _ in range(2):
        e.append((4.0 * e[-1] - e[-2]) / (3.0 + 2.0 * nu * dt))
    scale = np.abs(f0).max()
    for k, f in enumerate((f1, f2, f3), start=1):
        err = np.abs(f - (M + e[k])).max() / scale
        assert err < 1e-12, (k, err)


def _free_stream(integ, n_steps, T=0.4):
    w = synth.workload_p1_square(n_side=4, seed=0, n_v=4, k_v=3, L=2.0, knudsen=1.0)
    o = Oracle.from_workload(w)
    f = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    o.set_physics(0.0, T / n_steps, integ, 1e-13, 100)
    fprev = None
    for _ in range(n_steps):
        fn, _, _, status = o.step(f, fbc, fprev=fprev)
        assert status == 0
        if integ == "BDF2":
            fprev = f
        f = fn
    return f


@pytest.mark.parametrize("integ,order", [("BE", 1), ("DIRK2", 2), ("DIRK3", 3), ("BSTABLE2", 3), ("BDF2", 2)])
def test_free_streaming_temporal_order(integ, order):
    ref = _free_stream("DIRK3", 1024)
    errs = [np.abs(_free_stream(integ, n) - ref).max() for n in (32, 64, 128)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert order - 0.2 < rates[-1] < order + 0.3, (errs, rates)
    assert rates[0] > order - 0.35, (errs, rates)
