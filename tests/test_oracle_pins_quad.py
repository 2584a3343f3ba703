"""Pins of the oracle's Q1 quadrilaterals (Sec. 3.1's bilinear element), against facts fixed
independently of its reference-square Gauss route:

  - parallelograms: M, G and the edge matrices from exact rational integration (sympy) of
    the bilinear basis, mapped with the constant Jacobian;
  - a general (non-parallelogram) quadrilateral: a brute-force physical-space quadrature
    (a fine grid of points, the basis found by inverting the bilinear map);
  - integration by parts, G_al + G_al^T = sum_f n_al F_f, on a general quadrilateral;
  - the upwind DG method reproduces the exact backward-Euler stage of linear free
    streaming (linear functions lie in the Q1 space);
  - mass and energy conserved by a converged step in a closed reflecting box.
"""
import numpy as np
import pytest
import sympy as sp

from oracle.oracle import Oracle
from paper_2608_19150_b300 import synth


def _exact_ref():
    s, t = sp.symbols("s t")
    phi = [(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t]
    M = [[sp.integrate(phi[a] * phi[b], (s, 0, 1), (t, 0, 1)) for b in range(4)] for a in range(4)]
    Gs = [[sp.integrate(phi[b] * sp.diff(phi[a], s), (s, 0, 1), (t, 0, 1)) for b in range(4)] for a in range(4)]
    Gt = [[sp.integrate(phi[b] * sp.diff(phi[a], t), (s, 0, 1), (t, 0, 1)) for b in range(4)] for a in range(4)]
    f = lambda A: np.array([[float(x) for x in r] for r in A])  # noqa: E731
    return f(M), f(Gs), f(Gt)


def _one_cell(xyz):
    xyz = np.asarray(xyz, dtype=np.float64)
    return Oracle(2, 1, xyz, np.array([[0, 1, 2, 3]], dtype=np.int32), 4, 1, 6.0)


def test_parallelogram_matrices_exact():
    x0, e1, e2 = np.array([0.3, -0.2]), np.array([0.7, 0.1]), np.array([0.25, 0.5])
    o = _one_cell([x0, x0 + e1, x0 + e1 + e2, x0 + e2])
    c = o.cell(0)
    J = np.stack([e1, e2], axis=1)
    det = np.linalg.det(J)
    Ji = np.linalg.inv(J)
    M, Gs, Gt = _exact_ref()
    np.testing.assert_allclose(c["vol"], det, rtol=1e-14)
    np.testing.assert_allclose(c["M"], det * M, rtol=0, atol=1e-15)
    # grad phi = J^-T grad_ref phi: G_al = det (Ji[0, al] Gs + Ji[1, al] Gt)
    for al in range(2):
        np.testing.assert_allclose(c["G"][al], det * (Ji[0, al] * Gs + Ji[1, al] * Gt), rtol=0, atol=1e-14)
    for f in range(4):
        a, b = f, (f + 1) % 4
        L = np.linalg.norm(o.cell(0)["area"][f])
        F = np.zeros((4, 4))
        F[a, a] = F[b, b] = L / 3
        F[a, b] = F[b, a] = L / 6
        np.testing.assert_allclose(c["F"][f], F, rtol=0, atol=1e-15)


def test_general_quadrilateral_against_brute_force():
    X = np.array([[0.0, 0.0], [1.2, 0.1], [1.0, 0.9], [-0.1, 1.1]])
    o = _one_cell(X)
    c = o.cell(0)
    # physical-space midpoint rule on a fine grid; basis values by inverting the bilinear map
    n = 500
    lo, hi = X.min(0), X.max(0)
    gx = lo[0] + (np.arange(n) + 0.5) * (hi[0] - lo[0]) / n
    gy = lo[1] + (np.arange(n) + 0.5) * (hi[1] - lo[1]) / n
    P = np.stack(np.meshgrid(gx, gy, indexing="ij"), -1).reshape(-1, 2)
    dA = (hi[0] - lo[0]) * (hi[1] - lo[1]) / n ** 2
    st = np.full((P.shape[0], 2), 0.5)
    for _ in range(30):     # Newton on x(s, t) = P
        s, t = st[:, 0], st[:, 1]
        ph = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], 1)
        ds = np.stack([-(1 - t), 1 - t, t, -t], 1)
        dt_ = np.stack([-(1 - s), -s, s, 1 - s], 1)
        r = ph @ X - P
        Jm = np.stack([ds @ X, dt_ @ X], -1)      # [n, 2(x), 2(s,t)]
        st -= np.linalg.solve(Jm, r[..., None])[..., 0]
    s, t = st[:, 0], st[:, 1]
    inside = (s >= 0) & (s <= 1) & (t >= 0) & (t <= 1)
    ph = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], 1)[inside]
    ds = np.stack([-(1 - t), 1 - t, t, -t], 1)[inside]
    dt_ = np.stack([-(1 - s), -s, s, 1 - s], 1)[inside]
    Jm = np.stack([ds @ X, dt_ @ X], -1)
    Jinv = np.linalg.inv(Jm)                       # [n, (s,t), (x,y)]
    grad = np.einsum("nar,nrk->nak", np.stack([ds, dt_], -1), Jinv)   # d phi_a / d x_k
    M = dA * ph.T @ ph
    G = np.stack([dA * np.einsum("nb,na->ab", ph, grad[:, :, k]) for k in range(2)])
    vol = dA * inside.sum()
    assert abs(c["vol"] - vol) < 5e-3 * vol
    np.testing.assert_allclose(c["M"], M, rtol=0, atol=5e-3 * np.abs(M).max())
    np.testing.assert_allclose(c["G"], G, rtol=0, atol=5e-3 * np.abs(G).max())


def test_integration_by_parts_on_a_general_quadrilateral():
    o = _one_cell([[0.0, 0.0], [1.2, 0.1], [1.0, 0.9], [-0.1, 1.1]])
    c = o.cell(0)
    for al in range(2):
        rhs = sum(c["unit_n"][f, al] * c["F"][f] for f in range(4))
        np.testing.assert_allclose(c["G"][al] + c["G"][al].T, rhs, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shear", [0.0, 0.3])
def test_linear_free_streaming_reproduced(shear):
    m = synth.rect_quad_mesh(4, 3, shear=shear)
    o = Oracle(2, 1, m.xyz, m.cells, 8, 3, 6.0)
    o.build_dags()
    v, _, _, _ = o.velocity()
    X = synth.node_coords(m, 1).reshape(-1, 2)
    dt = 0.05
    a, bx, by = 0.7, 0.3, -0.2
    fk = np.zeros((o.nv, o.nnode))
    fex = np.zeros_like(fk)
    for j in range(o.nv):
        p = a + bx * X[:, 0] + by * X[:, 1]
        fk[j] = p
        fex[j] = p - dt * (v[j, 0] * bx + v[j, 1] * by)
    fnew = o.sweep(fk, np.zeros_like(fk), fk / dt, fex, 0.0, 1.0 / dt)
    np.testing.assert_allclose(fnew, fex, rtol=0, atol=1e-12)


def test_closed_box_of_quads_conserves_mass_and_energy():
    m = synth.rect_quad_mesh(4, 4)
    o = Oracle(2, 1, m.xyz, m.cells, 8, 3, 6.0)
    o.build_dags()
    o.set_walls({s: "reflect" for s in ("x-", "x+", "y-", "y+")})
    X = synth.node_coords(m, 1).reshape(-1, 2)
    n = 1.0 + 0.3 * np.sin(2 * np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    u = 0.2 * np.stack([np.cos(np.pi * X[:, 1]), np.sin(np.pi * X[:, 0])], 1)
    th = 1.0 + 0.2 * X[:, 0] * X[:, 1]
    f0 = o.maxwellian(np.concatenate([n[:, None], u, th[:, None]], 1))
    o.set_physics(10.0, 0.01, "BE", tau=1e-13, lmax=1000)
    f1, it, meas, st = o.step(f0, np.zeros_like(f0))
    assert st == 0
    v, wt, _, _ = o.velocity()
    wx = np.concatenate([o.cell(c)["M"].sum(0) for c in range(o.ncell)])
    for e in (np.ones(o.nv), 0.5 * (v * v).sum(1)):
        t0, t1 = (e * wt) @ f0 @ wx, (e * wt) @ f1 @ wx
        assert abs(t1 - t0) < 1e-10 * abs(t0)
    assert np.abs(f1 - f0).max() > 1e-4 * np.abs(f0).max()
