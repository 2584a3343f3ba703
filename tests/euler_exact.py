"""Exact solution of the Riemann problem for the 1D Euler equations of an ideal gas (the
fluid limit of the BGK model: gamma = (d + 2) / d, 2 for d = 2), used as the reference
of the Sod strip in the fluid limit (Sec. 5.1.1).  Test infrastructure only.

Method (Godunov's exact solver as set out in Toro's textbook, Riemann Solvers and Numerical
Methods for Fluid Dynamics, ch. 4): the star-region pressure p* is the root of
f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the velocity jump across the left/right wave
(a shock when p > p_K: Rankine-Hugoniot; a rarefaction otherwise: isentropic, with the
Riemann invariant u +- 2a/(gamma - 1)); u* follows from f_R - f_L; the solution at
xi = x / t is read off the wave pattern.
"""
import numpy as np


def _f(p, rho, pk, g):
    """Velocity change across the K wave and its derivative in p."""
    a = np.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * a / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * a)


def star_state(left, right, g):
    """(p*, u*) for primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _f(p, rl, pl, g)
        fr, dr = _f(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p_new = max(1e-14, p - dp)
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f(p, rl, pl, g)
    fr, _ = _f(p, rr, pr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, g, xi):
    """Primitive (rho, u, p) at the similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.empty(xi.shape + (3,))
    for idx, x in np.ndenumerate(xi):
        if x <= us:   # left of the contact
            if ps > pl:   # left shock
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                sl = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[idx] = (rl, ul, pl) if x < sl else (rs, us, ps)
            else:         # left rarefaction
                rs = rl * (ps / pl) ** (1 / g)
                head, tail = ul - al, us - np.sqrt(g * ps / rs)
                if x < head:
                    out[idx] = (rl, ul, pl)
                elif x > tail:
                    out[idx] = (rs, us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - x)
                    out[idx] = (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + x),
                                pl * c ** (2 * g / (g - 1)))
        else:         # right of the contact
            if ps > pr:   # right shock
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                sr = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[idx] = (rr, ur, pr) if x > sr else (rs, us, ps)
            else:         # right rarefaction
                rs = rr * (ps / pr) ** (1 / g)
                head, tail = ur + ar, us + np.sqrt(g * ps / rs)
                if x > head:
                    out[idx] = (rr, ur, pr)
                elif x < tail:
                    out[idx] = (rs, us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - x)
                    out[idx] = (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + x),
                                pr * c ** (2 * g / (g - 1)))
    return out
