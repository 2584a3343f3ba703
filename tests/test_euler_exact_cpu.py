"""Pins of the exact Riemann solver used as the fluid-limit reference of the Sod strip,
against the conservation laws it must satisfy (no stored values): the Rankine-Hugoniot
conditions across the shock, the isentropic relation and the Riemann invariant through the
rarefaction, continuity of pressure and velocity across the contact, the mirror symmetry of
the problem, and a constant state."""
import numpy as np
import pytest

from euler_exact import sample, star_state

SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))


def _cons(w, g):
    rho, u, p = w
    E = p / (g - 1) + 0.5 * rho * u * u
    return np.array([rho, rho * u, E]), np.array([rho * u, rho * u * u + p, u * (E + p)])


@pytest.mark.parametrize("g", [2.0, 1.4, 5.0 / 3.0])
def test_shock_satisfies_rankine_hugoniot(g):
    xi = np.linspace(-3, 3, 60001)
    w = sample(*SOD, g, xi)
    ps, us = star_state(*SOD, g)
    jumps = np.abs(np.diff(w[:, 0]))
    right = xi[:-1] > us + 1e-3
    k = np.argmax(np.where(right, jumps, 0.0))
    pre, post = w[k + 1], w[k]
    Upre, Fpre = _cons(pre, g)
    Upost, Fpost = _cons(post, g)
    s = (Fpost[0] - Fpre[0]) / (Upost[0] - Upre[0])       # from the mass jump
    assert abs(s - xi[k]) < 1e-3                           # the jump sits where the speed says
    np.testing.assert_allclose(Fpost - Fpre, s * (Upost - Upre), rtol=1e-12, atol=1e-12)
    assert post[2] == pytest.approx(ps, rel=1e-14) and post[1] == pytest.approx(us, rel=1e-14)


@pytest.mark.parametrize("g", [2.0, 1.4])
def test_rarefaction_isentropic_with_constant_riemann_invariant(g):
    (rl, ul, pl), _ = SOD
    al = np.sqrt(g * pl / rl)
    ps, us = star_state(*SOD, g)
    rs = rl * (ps / pl) ** (1 / g)
    xi = np.linspace(ul - al, us - np.sqrt(g * ps / rs), 101)[1:-1]
    w = sample(*SOD, g, xi)
    rho, u, p = w[:, 0], w[:, 1], w[:, 2]
    a = np.sqrt(g * p / rho)
    np.testing.assert_allclose(p / rho ** g, pl / rl ** g, rtol=1e-12)
    np.testing.assert_allclose(u + 2 * a / (g - 1), ul + 2 * al / (g - 1), rtol=1e-12)
    np.testing.assert_allclose(u - xi, a, rtol=1e-12)      # a C- characteristic fan: u - a = xi


def test_contact_continuity_and_star_equation():
    g = 2.0
    ps, us = star_state(*SOD, g)
    w = sample(*SOD, g, np.array([us - 1e-9, us + 1e-9]))
    assert w[0, 2] == pytest.approx(w[1, 2], rel=1e-14) and w[0, 1] == pytest.approx(w[1, 1], rel=1e-14)
    assert w[0, 0] > w[1, 0]                                # the density jumps at the contact
    # the star pressure makes the two wave curves meet: u*_L(p*) = u*_R(p*)
    (rl, ul, pl), (rr, ur, pr) = SOD
    al = np.sqrt(g * pl / rl)
    uL = ul - 2 * al / (g - 1) * ((ps / pl) ** ((g - 1) / (2 * g)) - 1)
    A, B = 2 / ((g + 1) * rr), (g - 1) / (g + 1) * pr
    uR = ur + (ps - pr) * np.sqrt(A / (ps + B))
    assert uL == pytest.approx(uR, abs=1e-14) and us == pytest.approx(uL, abs=1e-14)


def test_mirror_symmetry_and_constant_state():
    g = 2.0
    xi = np.linspace(-2, 2, 401)
    w = sample(*SOD, g, xi)
    (rl, ul, pl), (rr, ur, pr) = SOD
    m = sample((rr, -ur, pr), (rl, -ul, pl), g, -xi)
    np.testing.assert_allclose(m[:, 0], w[:, 0], rtol=1e-13)
    np.testing.assert_allclose(m[:, 1], -w[:, 1], atol=1e-13)
    np.testing.assert_allclose(m[:, 2], w[:, 2], rtol=1e-13)
    c = sample((0.7, 0.3, 0.5), (0.7, 0.3, 0.5), g, xi)
    np.testing.assert_allclose(c, np.tile([0.7, 0.3, 0.5], (xi.size, 1)), rtol=1e-13)
