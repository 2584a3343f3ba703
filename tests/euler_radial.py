"""Radially symmetric Euler equations of an ideal gas (the fluid-limit reference of the
multi-dimensional Sod problem, Sec. 5.1.2: cylindrical for d = 2, gamma = 2), solved by a
second-order finite-volume method of my own: cells on [0, R], face areas r^alpha (alpha = 1
cylindrical, 2 spherical, 0 planar), HLL fluxes of minmod-limited primitive states, the
geometric pressure source p dA/dr, two-stage SSP Runge-Kutta in time.  Test infrastructure.
"""
import numpy as np


def _prim(U, g):
    rho = U[0]
    u = U[1] / rho
    p = (g - 1.0) * (U[2] - 0.5 * rho * u * u)
    return rho, u, p


def _flux(rho, u, p, g):
    E = p / (g - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)]), np.array([rho, rho * u, E])


def _minmod(a, b):
    return np.where(a * b > 0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def _rhs(U, r_f, V, dA, g):
    rho, u, p = _prim(U, g)
    W = np.stack([rho, u, p])
    # ghost cells: reflection at r = 0, zero gradient at r = R
    Wg = np.concatenate([W[:, :1] * np.array([[1], [-1], [1]]), W, W[:, -1:]], axis=1)
    s = _minmod(Wg[:, 1:-1] - Wg[:, :-2], Wg[:, 2:] - Wg[:, 1:-1])
    WL = W + 0.5 * s                # state at the right face of each cell
    WR = W - 0.5 * s                # state at the left face
    # face k between cells k-1 and k (k = 1..n-1); faces 0 and n from the boundary rules
    L = np.concatenate([WR[:, :1] * np.array([[1], [-1], [1]]), WL], axis=1)
    Rt = np.concatenate([WR, WL[:, -1:]], axis=1)
    FL, UL = _flux(L[0], L[1], L[2], g)
    FR, UR = _flux(Rt[0], Rt[1], Rt[2], g)
    cL = np.sqrt(g * L[2] / L[0])
    cR = np.sqrt(g * Rt[2] / Rt[0])
    sL = np.minimum(L[1] - cL, Rt[1] - cR)
    sR = np.maximum(L[1] + cL, Rt[1] + cR)
    F = np.where(sL >= 0, FL, np.where(sR <= 0, FR, (sR * FL - sL * FR + sL * sR * (UR - UL)) / (sR - sL)))
    AF = F * r_f
    dU = -(AF[:, 1:] - AF[:, :-1]) / V
    dU[1] += p * dA / V
    return dU, np.max(np.maximum(np.abs(sL), np.abs(sR)))


def solve(rho0, u0, p0, R, t_end, n=2000, alpha=1, g=2.0, cfl=0.4):
    """Cell centres and primitive (rho, u, p) at t_end, from initial primitive functions of r."""
    r_f = np.linspace(0.0, R, n + 1)
    rc = 0.5 * (r_f[1:] + r_f[:-1])
    A = r_f ** alpha if alpha else np.ones_like(r_f)
    V = (r_f[1:] ** (alpha + 1) - r_f[:-1] ** (alpha + 1)) / (alpha + 1)
    dA = A[1:] - A[:-1]
    rho, u, p = rho0(rc), u0(rc), p0(rc)
    U = np.stack([rho, rho * u, p / (g - 1.0) + 0.5 * rho * u * u])
    t = 0.0
    dr = R / n
    while t < t_end:
        k1, smax = _rhs(U, A, V, dA, g)
        dt = min(cfl * dr / smax, t_end - t)
        U1 = U + dt * k1
        k2, _ = _rhs(U1, A, V, dA, g)
        U = 0.5 * (U + U1 + dt * k2)
        t += dt
    return rc, np.stack(_prim(U, g))
