"""Pins of the radial Euler reference solver: planar (alpha = 0) it converges to the exact
Riemann solution; cylindrical it conserves mass, keeps a uniform state uniform (the
pressure source balances the flux through the growing faces) and converges under mesh
refinement."""
import numpy as np

from euler_exact import sample
from euler_radial import solve


def _sod(r0, x0=0.0):
    return (lambda r: np.where(r < r0, 1.0, 0.125), lambda r: 0.0 * r, lambda r: np.where(r < r0, 1.0, 0.1))


def test_planar_limit_matches_the_exact_riemann_solution():
    rho0, u0, p0 = _sod(0.5)
    for n, tol in ((400, 0.02), (1600, 0.006)):
        rc, W = solve(rho0, u0, p0, 1.0, 0.15, n=n, alpha=0)
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 2.0, (rc - 0.5) / 0.15)
        e = np.mean(np.abs(W[0] - ex[:, 0]))
        assert e < tol, (n, e)


def test_cylindrical_conserves_mass_and_keeps_a_uniform_state():
    rho0, u0, p0 = _sod(0.4)
    rc, W = solve(rho0, u0, p0, 1.0, 0.15, n=800, alpha=1)
    r_f = np.linspace(0, 1.0, 801)
    V = (r_f[1:] ** 2 - r_f[:-1] ** 2) / 2
    m0 = np.sum(V * rho0(rc))
    assert abs(np.sum(V * W[0]) - m0) < 1e-12 * m0
    rc, W = solve(lambda r: 0 * r + 0.7, lambda r: 0 * r, lambda r: 0 * r + 0.3, 1.0, 0.1, n=200, alpha=1)
    np.testing.assert_allclose(W[0], 0.7, rtol=1e-13)
    np.testing.assert_allclose(W[1], 0.0, atol=1e-13)
    np.testing.assert_allclose(W[2], 0.3, rtol=1e-13)


def test_cylindrical_converges_under_refinement():
    rho0, u0, p0 = _sod(0.4)
    res = {n: solve(rho0, u0, p0, 1.0, 0.15, n=n, alpha=1) for n in (500, 1000, 2000, 4000)}
    ref_r, ref = res[4000]
    diffs = [np.mean(np.abs(np.interp(ref_r, *[res[n][0], res[n][1][0]]) - ref[0])) for n in (500, 1000, 2000)]
    assert diffs[0] > diffs[1] > diffs[2]
    assert diffs[2] < 5e-3
