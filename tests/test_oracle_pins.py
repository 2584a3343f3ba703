"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's own formula:
they compare with library routines (numpy Gauss-Legendre, mpmath quadrature, networkx
graph algorithms, dense numpy solves), closed forms, and invariants the paper states.
"""
import itertools
import math
import os

import mpmath
import networkx as nx
import numpy as np
import pytest

from oracle.oracle import Oracle, tableau
from paper_2608_19150_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def small_square(n=4, seed=0, kx=1, n1d=8, kv=3, L=6.0):
    m = synth.square_mesh(n, seed, 0.2)
    return m, Oracle(2, kx, m.xyz, m.cells, n1d, kv, L)


def small_cube(n=2, seed=2, n1d=8, kv=3, L=6.0):
    m = synth.cube_mesh(n, seed, 0.15)
    return m, Oracle(3, 1, m.xyz, m.cells, n1d, kv, L)


# ------------------------------------------------------------------ velocity grid (Sec. 3.2)
@pytest.mark.parametrize("kv", [1, 2, 3, 4])
def test_velocity_grid_matches_numpy_gauss_legendre(kv):
    n1d = 3 * (kv + 1)
    _, o = small_square(2, n1d=n1d, kv=kv)
    v, w, x1, w1 = o.velocity()
    xg, wg = np.polynomial.legendre.leggauss(kv + 1)
    h = 12.0 / 3
    exp_x = np.concatenate([-6.0 + (c + 0.5) * h + 0.5 * h * xg for c in range(3)])
    exp_w = np.concatenate([0.5 * h * wg for _ in range(3)])
    np.testing.assert_allclose(x1, exp_x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w1, exp_w, rtol=1e-14)
    # tensor product, last dimension fastest
    assert np.allclose(v[1], [x1[0], x1[1]]) and np.allclose(v[n1d], [x1[1], x1[0]])
    assert abs(w.sum() - 144.0) < 1e-12


# ------------------------------------------------------- element matrices (Sec. 3.1, Table 1)
def _cross2(a, b):
    return a[0] * b[1] - a[1] * b[0]


def _tri_quadrature(p, order=12):
    """Collapsed (Duffy) Gauss rule on the triangle p[0..2]; exact for high degree."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    s, ws = 0.5 * (xg + 1), 0.5 * wg
    pts, wts = [], []
    for a, wa in zip(s, ws):
        for b, wb in zip(s, ws):
            xi, eta = a, b * (1 - a)
            pts.append(p[0] + xi * (p[1] - p[0]) + eta * (p[2] - p[0]))
            wts.append(wa * wb * (1 - a))
    J = abs(_cross2(p[1] - p[0], p[2] - p[0]))
    return np.array(pts), np.array(wts) * J


def _nodal_basis_2d(nodes, kx):
    """Lagrange basis on the given nodes via the monomial Vandermonde matrix."""
    if kx == 1:
        mono = lambda x, y: np.stack([np.ones_like(x), x, y], -1)  # noqa: E731
        dmono = lambda x, y: (np.stack([0 * x, 1 + 0 * x, 0 * x], -1), np.stack([0 * x, 0 * x, 1 + 0 * x], -1))  # noqa
    else:
        mono = lambda x, y: np.stack([np.ones_like(x), x, y, x * x, x * y, y * y], -1)  # noqa: E731
        dmono = lambda x, y: (np.stack([0 * x, 1 + 0 * x, 0 * x, 2 * x, y, 0 * x], -1),  # noqa: E731
                              np.stack([0 * x, 0 * x, 1 + 0 * x, 0 * x, x, 2 * y], -1))
    V = mono(nodes[:, 0], nodes[:, 1])
    Ci = np.linalg.inv(V)               # phi = mono @ Ci
    phi = lambda x, y: mono(x, y) @ Ci  # noqa: E731
    dphi = lambda x, y: tuple(d @ Ci for d in dmono(x, y))  # noqa: E731
    return phi, dphi


@pytest.mark.parametrize("kx", [1, 2])
def test_triangle_matrices_against_brute_force_quadrature(kx):
    m, o = small_square(3, seed=7, kx=kx)
    nodes_all = synth.node_coords(m, kx)
    for c in [0, 5, 11]:
        cell = o.cell(c)
        p = m.xyz[m.cells[c]]
        phi, dphi = _nodal_basis_2d(nodes_all[c], kx)
        X, W = _tri_quadrature(p)
        P = phi(X[:, 0], X[:, 1])
        Dx, Dy = dphi(X[:, 0], X[:, 1])
        M = np.einsum("q,qa,qb->ab", W, P, P)
        Gx = np.einsum("q,qb,qa->ab", W, P, Dx)   # int phi_b d_x phi_a
        Gy = np.einsum("q,qb,qa->ab", W, P, Dy)
        np.testing.assert_allclose(cell["M"], M, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(cell["G"][0], Gx, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(cell["G"][1], Gy, rtol=1e-11, atol=1e-13)
        assert abs(cell["vol"] - 0.5 * abs(_cross2(p[1] - p[0], p[2] - p[0]))) < 1e-15
        # face mass on each edge via 1D Gauss; face f is opposite vertex f
        xg, wg = np.polynomial.legendre.leggauss(8)
        for f in range(3):
            a, b = p[(f + 1) % 3], p[(f + 2) % 3]
            t = 0.5 * (xg + 1)
            Q = a[None] + t[:, None] * (b - a)[None]
            Wq = 0.5 * wg * np.linalg.norm(b - a)
            Pe = phi(Q[:, 0], Q[:, 1])
            Fe = np.einsum("q,qa,qb->ab", Wq, Pe, Pe)
            np.testing.assert_allclose(cell["F"][f], Fe, rtol=1e-12, atol=1e-14)
            # unit outward normal: perpendicular to the edge, pointing away from vertex f
            n = cell["unit_n"][f]
            assert abs(np.dot(n, b - a)) < 1e-14 and np.dot(n, p[f] - a) < 0
            assert abs(np.linalg.norm(n) - 1) < 1e-14


def test_closed_form_p1_matrices():
    """P1 simplex closed forms: M = |K|(1+delta)/((d+1)(d+2)); face mass |F|(1+delta)/(d(d+1))."""
    for (m, o), d in [(small_square(3), 2), (small_cube(2), 3)]:
        for c in [0, 3, 7]:
            cell = o.cell(c)
            K = cell["vol"]
            ref = K * (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
            np.testing.assert_allclose(cell["M"], ref, rtol=1e-13)
            for f in range(d + 1):
                idx = [a for a in range(d + 1) if a != f]
                F = cell["F"][f]
                ref_f = cell["area"][f] * (np.ones((d, d)) + np.eye(d)) / (d * (d + 1))
                np.testing.assert_allclose(F[np.ix_(idx, idx)], ref_f, rtol=1e-13)
                assert np.all(F[f, :] == 0) and np.all(F[:, f] == 0)


@pytest.mark.parametrize("which", ["p1", "p2", "tet"])
def test_integration_by_parts_identity(which):
    """int d_a(phi_i phi_j) = sum_e n_e,a int_e phi_i phi_j : G + G^T = sum_e n_e F_e."""
    if which == "tet":
        m, o = small_cube(2)
        d = 3
    else:
        m, o = small_square(3, kx=1 if which == "p1" else 2)
        d = 2
    for c in range(0, o.ncell, 5):
        cell = o.cell(c)
        for al in range(d):
            lhs = cell["G"][al] + cell["G"][al].T
            rhs = np.einsum("f,fab->ab", cell["unit_n"][:, al], cell["F"])
            np.testing.assert_allclose(lhs, rhs, atol=1e-14)
        # partition of unity: sum_a d phi_a = 0
        np.testing.assert_allclose(cell["G"].sum(axis=1), 0.0, atol=1e-14)


def test_neighbours_and_node_matching():
    for kx in (1, 2):
        m, o = small_square(4, kx=kx)
        xn = synth.node_coords(m, kx)
        for c in range(o.ncell):
            cell = o.cell(c)
            for f in range(3):
                nb = cell["nbr"][f]
                if nb < 0:
                    continue
                for a in range(o.ndof):
                    b = cell["nbr_node"][f, a]
                    if b >= 0:
                        assert np.allclose(xn[c, a], xn[nb, b], atol=1e-15)


# --------------------------------------------------- Maxwellian projection (App. B)
def test_projection_factors_against_mpmath_quadrature():
    _, o = small_square(2, n1d=16, kv=3, L=6.0)
    _, _, x1, w1 = o.velocity()
    mpmath.mp.dps = 30
    np_, ncl, h = 4, 4, 3.0
    for (u, th) in [(0.0, 1.0), (0.7, 0.4), (-2.5, 2.0)]:
        c = o.project_1d(u, th)
        for m in range(16):
            cl, k = divmod(m, np_)
            nodes = [mpmath.mpf(x1[cl * np_ + i]) for i in range(np_)]
            ell = lambda v: mpmath.fprod([(v - nodes[i]) / (nodes[k] - nodes[i]) for i in range(np_) if i != k])  # noqa
            g = lambda v: mpmath.exp(-(v - u) ** 2 / (2 * th)) / mpmath.sqrt(2 * mpmath.pi * th)  # noqa
            lo = -mpmath.inf if cl == 0 else mpmath.mpf(-6 + cl * h)
            hi = mpmath.inf if cl == ncl - 1 else mpmath.mpf(-6 + (cl + 1) * h)
            ref = mpmath.quad(lambda v: g(v) * ell(v), [lo, mpmath.mpf(-6 + cl * h) if cl == 0 else lo, hi]
                              if cl == 0 else [lo, hi]) / mpmath.mpf(w1[m])
            assert abs(c[m] - float(ref)) <= 1e-13 * max(1.0, abs(float(ref))), (u, th, m, c[m], ref)
        # partition of unity: sum_m w_m c_m = int g = 1
        assert abs(np.dot(w1, c) - 1.0) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_projection_reproduces_moments_exactly(d):
    """App. B eq. (cons_projection_exactness): sum_j w_j e_j (P M)_j = U_M for any n,u,theta."""
    o = small_square(2, n1d=16)[1] if d == 2 else small_cube(1, n1d=8)[1]
    v, w, _, _ = o.velocity()
    rng = np.random.default_rng(5)
    for _ in range(5):
        n = rng.uniform(0.1, 3)
        u = rng.uniform(-1.5, 1.5, d)
        th = rng.uniform(0.3, 2.0)
        nut = np.tile(np.concatenate([[n], u, [th]]), (o.nnode, 1))
        f = o.maxwellian(nut)
        U = o.moments(f)[0]
        exact = np.concatenate([[n], n * u, [0.5 * n * u @ u + 0.5 * d * n * th]])
        np.testing.assert_allclose(U, exact, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------- sweep graphs (Sec. 4.1)
def _graph(o, j):
    s = o.face_signs(j)
    G = nx.DiGraph()
    G.add_nodes_from(range(o.ncell))
    edges = {}
    for c in range(o.ncell):
        cell = o.cell(c)
        for f in range(o.nface):
            nb = cell["nbr"][f]
            if nb >= 0 and s[c, f] > 0:
                G.add_edge(c, int(nb))
                edges[(c, int(nb))] = f
    return G, s


@pytest.mark.parametrize("mesh", ["tri", "tet"])
def test_generations_are_longest_paths_of_an_acyclic_graph(mesh):
    m, o = small_square(5, n1d=8) if mesh == "tri" else _find_cyclic_cube()
    total_lagged = o.build_dags()
    checked_cycle = False
    for j in range(o.nv):
        G, s = _graph(o, j)
        gen, lag, ngen = o.generations(j)
        # signs are antisymmetric across every interior face
        for c in range(o.ncell):
            cell = o.cell(c)
            for f in range(o.nface):
                nb = cell["nbr"][f]
                if nb >= 0:
                    fb = list(o.cell(nb)["nbr"]).index(c)
                    assert s[c, f] == -s[nb, fb]
        kept = G.copy()
        lagged_edges = []
        for c in range(o.ncell):
            cell = o.cell(c)
            for f in range(o.nface):
                if lag[c, f]:
                    a = int(cell["nbr"][f])
                    assert kept.has_edge(a, c)
                    kept.remove_edge(a, c)
                    lagged_edges.append((a, c))
        assert nx.is_directed_acyclic_graph(kept)
        if lagged_edges:
            checked_cycle = True
            sccs = {v: i for i, comp in enumerate(nx.strongly_connected_components(G)) for v in comp}
            for a, b in lagged_edges:
                assert sccs[a] == sccs[b]              # only edges inside cycles are lagged
                assert gen[a] > gen[b]                 # lagged upwind value is still f^l
        else:
            assert nx.is_directed_acyclic_graph(G)
        # gen = longest path from a source (brute force over the kept DAG)
        ref = {}
        for v in nx.topological_sort(kept):
            preds = list(kept.predecessors(v))
            ref[v] = 0 if not preds else 1 + max(ref[p] for p in preds)
        assert all(gen[v] == ref[v] for v in range(o.ncell))
        assert ngen == max(ref.values()) + 1
    if mesh == "tri":
        assert total_lagged == 0      # straight-sided triangulations have acyclic sweep graphs
    else:
        assert checked_cycle == (total_lagged > 0)


def _find_cyclic_cube():
    m = synth.twisted_cube_mesh(3, 0, 0.25, 2.0)
    o = Oracle(3, 1, m.xyz, m.cells, 8, 3, 6.0)
    if o.build_dags() > 0:
        return m, o
    return None, None


def test_cycles_occur_on_jittered_tets_and_are_broken():
    m, o = _find_cyclic_cube()
    assert o is not None, "no cyclic sweep graph found among the seeded tetrahedral meshes"
    for j in range(o.nv):
        G, _ = _graph(o, j)
        gen, lag, _ = o.generations(j)
        if lag.any():
            assert not nx.is_directed_acyclic_graph(G)
            return
    pytest.fail("lagged edges reported but none found")


# -------------------------------------------------------------- sweep (Sec. 4, Eq. bgk-ss-picard)
def _global_solve(o, j, Mn, q, fbc, nu, nu_s):
    """Assemble the block system of one ordinate for the whole mesh and solve it directly."""
    v, _, _, _ = o.velocity()
    vj = v[j]
    s = o.face_signs(j)
    nd, N = o.ndof, o.ncell * o.ndof
    A = np.zeros((N, N))
    b = np.zeros(N)
    for c in range(o.ncell):
        cell = o.cell(c)
        r = slice(c * nd, (c + 1) * nd)
        A[r, r] += -np.einsum("a,aij->ij", vj, cell["G"]) + nu_s * cell["M"]
        b[r] += cell["M"] @ (nu * Mn[j, r] + q[j, r])
        for f in range(o.nface):
            vn = vj @ cell["unit_n"][f]
            F = cell["F"][f]
            if s[c, f] > 0:
                A[r, r] += vn * F
            elif s[c, f] < 0:
                nb = cell["nbr"][f]
                if nb < 0:
                    b[r] -= vn * F @ fbc[j, r]
                else:
                    for a in range(nd):
                        bb = cell["nbr_node"][f, a]
                        if bb >= 0:
                            A[r, nb * nd + bb] += vn * F[:, a]
    return np.linalg.solve(A, b)


def _random_fields(o, seed):
    rng = np.random.default_rng(seed)
    sh = (o.nv, o.nnode)
    return rng.uniform(0.1, 1, sh), rng.uniform(0.1, 1, sh), rng.uniform(0.1, 1, sh), rng.uniform(0.1, 1, sh)


@pytest.mark.parametrize("kx", [1, 2])
def test_sweep_equals_global_direct_solve_on_acyclic_graphs(kx):
    m, o = small_square(3, kx=kx, n1d=8)
    fold, Mn, q, fbc = _random_fields(o, 1)
    nu, nu_s = 3.0, 40.0
    fnew = o.sweep(fold, Mn, q, fbc, nu, nu_s)
    for j in [0, 9, 27, 63]:
        x = _global_solve(o, j, Mn, q, fbc, nu, nu_s)
        np.testing.assert_allclose(fnew[j], x, rtol=1e-12, atol=1e-14)


def test_lagged_sweeps_converge_to_global_solve_with_cycles():
    m, o = _find_cyclic_cube()
    fold, Mn, q, fbc = _random_fields(o, 2)
    nu, nu_s = 1.0, 30.0
    cyc = [j for j in range(o.nv) if o.generations(j)[1].any()]
    assert cyc
    f = fold
    for _ in range(60):              # block Gauss-Seidel in the lagged edges
        f = o.sweep(f, Mn, q, fbc, nu, nu_s)
    for j in cyc[:3]:
        x = _global_solve(o, j, Mn, q, fbc, nu, nu_s)
        np.testing.assert_allclose(f[j], x, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("kx", [1, 2])
def test_polynomial_reproduction_free_streaming(kx):
    """nu = 0, backward Euler: f = f^k - dt v.grad f^k (+ dt^2 (v.grad)^2 f^k for P2) is the
    exact stage solution, it lies in the DG space, and the upwind DG method reproduces it."""
    m, o = small_square(4, kx=kx, n1d=8)
    v, _, _, _ = o.velocity()
    X = synth.node_coords(m, kx).reshape(-1, 2)
    dt = 0.05
    a, bx, by, cxx, cxy, cyy = 0.7, 0.3, -0.2, (0.0 if kx == 1 else 0.25), (0.0 if kx == 1 else -0.1), (0.0 if kx == 1 else 0.15)
    fk = np.zeros((o.nv, o.nnode))
    fex = np.zeros_like(fk)
    for j in range(o.nv):
        vx, vy = v[j]
        x, y = X[:, 0], X[:, 1]
        p = a + bx * x + by * y + cxx * x * x + cxy * x * y + cyy * y * y
        vg = vx * (bx + 2 * cxx * x + cxy * y) + vy * (by + cxy * x + 2 * cyy * y)
        vvg = vx * vx * 2 * cxx + 2 * vx * vy * cxy + vy * vy * 2 * cyy
        fk[j] = p
        fex[j] = p - dt * vg + dt * dt * vvg
    fnew = o.sweep(fk, np.zeros_like(fk), fk / dt, fex, 0.0, 1.0 / dt)
    np.testing.assert_allclose(fnew, fex, rtol=0, atol=1e-12)


@pytest.mark.parametrize("integ", ["BE", "DIRK2", "DIRK3", "BSTABLE2", "BDF2"])
def test_uniform_maxwellian_is_a_fixed_point(integ):
    m, o = small_square(4, n1d=12, kv=2)
    nut = np.tile([0.8, 0.3, -0.2, 1.2], (o.nnode, 1))
    f0 = o.maxwellian(nut)
    o.set_physics(50.0, 0.02, integ)
    f1, it, meas, st = o.step(f0, f0, fprev=f0 if integ == "BDF2" else None)
    assert st == 0
    np.testing.assert_allclose(f1, f0, rtol=0, atol=2e-14 * np.abs(f0).max())


def test_l2_stability_free_streaming_zero_inflow():
    """Prop. (Linear Stability), case nu = 0 with zero inflow: ||f||_{L2} does not grow."""
    m, o = small_square(4, n1d=8)
    w = synth.workload_p1_square(n_side=4, n_v=8)
    f = o.maxwellian(w.init)
    _, wt, _, _ = o.velocity()
    Ms = [o.cell(c)["M"] for c in range(o.ncell)]

    def l2(f):
        return sum(wt[j] * sum(f[j, c * 3:(c + 1) * 3] @ Ms[c] @ f[j, c * 3:(c + 1) * 3] for c in range(o.ncell))
                   for j in range(o.nv))
    o.set_physics(0.0, 0.05, "BE")
    prev = l2(f)
    for _ in range(3):
        f, it, meas, st = o.step(f, np.zeros_like(f))
        cur = l2(f)
        assert cur <= prev * (1 + 1e-14)
        prev = cur


@pytest.mark.parametrize("integ", ["BE", "BSTABLE2", "DIRK3"])
def test_linear_maxwellian_constant_state_is_steady(integ):
    """Eq. linear-Maxwellian: N_h = n / |V| with |V| = (2L)^d.  A state constant in x and v
    with the same constant as inflow is an exact steady state (transport vanishes and
    N_h equals the state); a wrong |V| or moment breaks it."""
    m, o = small_square(4, n1d=8)
    c = 0.37
    f = np.full((o.nv, o.nnode), c)
    o.set_collision("linear")
    o.set_physics(1000.0, 0.05, integ, tau=1e-13, lmax=200)
    f1, it, meas, st = o.step(f, f.copy())
    assert st == 0
    np.testing.assert_allclose(f1, c, rtol=0, atol=1e-14)


@pytest.mark.parametrize("integ", ["BE", "BSTABLE2"])
def test_l2_stability_linear_maxwellian_zero_inflow(integ):
    """Prop. (Linear Stability), case (ii): with the simplified Maxwellian, nu = 1000 and
    zero inflow, B-stable integrators do not let ||f||_{L2(X x V)} grow."""
    m, o = small_square(4, n1d=8)
    w = synth.workload_p1_square(n_side=4, n_v=8)
    f = o.maxwellian(w.init)
    _, wt, _, _ = o.velocity()
    Ms = [o.cell(c)["M"] for c in range(o.ncell)]

    def l2(f):
        return sum(wt[j] * sum(f[j, c * 3:(c + 1) * 3] @ Ms[c] @ f[j, c * 3:(c + 1) * 3] for c in range(o.ncell))
                   for j in range(o.nv))
    o.set_collision("linear")
    o.set_physics(1000.0, 0.002, integ, tau=1e-13, lmax=1000)
    prev = l2(f)
    for _ in range(3):
        f, it, meas, st = o.step(f, np.zeros_like(f))
        assert st == 0
        cur = l2(f)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_linear_maxwellian_collision_conserves_mass_only():
    """The simplified collision term sum_j w_j (N_h - f_j) has zero density moment (the
    quadrature integrates 1 exactly: sum_j w_j = |V|) but not zero momentum or energy."""
    m, o = small_square(3, n1d=8)
    w = synth.workload_p1_square(n_side=3, n_v=8)
    nut = w.init.copy()
    nut[:, 1] = 0.3
    f = o.maxwellian(nut)
    v, wt, _, _ = o.velocity()
    U = o.moments(f)
    N = U[:, 0] / (2 * o.L) ** 2
    coll = N[None, :] - f
    E = np.concatenate([np.ones((o.nv, 1)), v, 0.5 * (v * v).sum(1, keepdims=True)], axis=1)
    dU = E.T @ (wt[:, None] * coll)
    assert np.abs(dU[0]).max() < 1e-14 * np.abs(U[:, 0]).max()
    assert np.abs(dU[1]).max() > 1e-3


def test_discrete_conservation_law_backward_euler():
    """Eq. (discrete-cons): after a converged BE step the change of int U equals minus dt
    times the net boundary flux sum_j w_j e_j (v_j.n) f_hat over dX (interior faces cancel)."""
    m, o = small_square(4, n1d=12, kv=2)
    w = synth.workload_p1_square(n_side=4, n_v=12, k_v=2)
    f0 = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    dt, nu = 0.01, 10.0
    o.set_physics(nu, dt, "BE", tau=1e-13, lmax=200)
    f1, it, meas, st = o.step(f0, fbc)
    assert st == 0
    v, wt, _, _ = o.velocity()
    E = np.concatenate([np.ones((o.nv, 1)), v, 0.5 * (v * v).sum(1, keepdims=True)], axis=1)
    dU = np.zeros(4)
    flux = np.zeros(4)
    for c in range(o.ncell):
        cell = o.cell(c)
        r = slice(c * 3, (c + 1) * 3)
        one_M = cell["M"].sum(axis=0)                 # int phi_b
        dU += E.T @ (wt[:, None] * (f1[:, r] - f0[:, r])) @ one_M
        for f in range(3):
            if cell["nbr"][f] >= 0:
                continue
            vn = v @ cell["unit_n"][f]
            Fsum = cell["F"][f].sum(axis=0)            # int_e phi_b
            trace = np.where((vn > 0)[:, None], f1[:, r], fbc[:, r]) @ Fsum
            flux += E.T @ (wt * vn * trace)
    np.testing.assert_allclose(dU / dt, -flux, rtol=0, atol=1e-9 * np.abs(flux).max())


# -------------------------------------------------------------- DIRK tableaus (App. A)
def test_tableaus_match_printed_digits_and_order_conditions():
    A, b, c = tableau("DIRK3")
    rows = [ln.split("|") for ln in open(os.path.join(GOLDEN, "dirk3_tableau_printed.txt"))
            if ln.strip() and not ln.startswith("#")]
    c_pr = [float(r[0]) for r in rows[:3]]
    A_pr = [[float(x) for x in r[1].split()] for r in rows[:3]]
    b_pr = [float(x) for x in rows[3][1].split()]
    np.testing.assert_allclose(A, A_pr, atol=5e-7)
    np.testing.assert_allclose(c, c_pr, atol=5e-7)
    np.testing.assert_allclose(b, b_pr, atol=5e-7)
    np.testing.assert_allclose(b, A[-1], atol=1e-15)
    assert abs(b.sum() - 1) < 1e-14 and abs(b @ c - 0.5) < 1e-14
    assert abs(b @ c ** 2 - 1 / 3) < 1e-14 and abs(b @ A @ c - 1 / 6) < 1e-14
    np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-14)
    A2, b2, c2 = tableau("DIRK2")
    g = 1 - math.sqrt(2) / 2
    np.testing.assert_allclose(A2, [[g, 0], [math.sqrt(2) / 2, g]], atol=1e-15)
    assert abs(b2.sum() - 1) < 1e-15 and abs(b2 @ c2 - 0.5) < 1e-15
    Ab, bb, cb = tableau("BSTABLE2")
    # the values printed in closed form in Eq. (B-RK): gamma = (3 + sqrt 3)/6,
    # A = [[gamma, 0], [1 - (3 + sqrt 3)/3, gamma]], c = (gamma, 1 - gamma), b = (1/2, 1/2)
    gb = (3 + math.sqrt(3)) / 6
    np.testing.assert_allclose(Ab, [[gb, 0], [1 - (3 + math.sqrt(3)) / 3, gb]], atol=1e-15)
    np.testing.assert_allclose(cb, [gb, 1 - gb], atol=1e-15)
    np.testing.assert_allclose(bb, [0.5, 0.5], atol=1e-15)
    B = np.diag(bb)
    Mb = B @ Ab + Ab.T @ B - np.outer(bb, bb)     # algebraic stability (App. A)
    assert np.linalg.eigvalsh(Mb).min() > -1e-14
    assert abs(bb @ cb - 0.5) < 1e-15 and abs(bb @ cb ** 2 - 1 / 3) < 1e-15


def test_explicit_time_step_bound():
    """Sec. 5: dt_e = (1/d) (1/(2k+1)) h_min / max_j |v_j| with h_min = (min vol)^(1/d)."""
    m, o = small_square(4, n1d=8)
    v, _, _, _ = o.velocity()
    vols = [o.cell(c)["vol"] for c in range(o.ncell)]
    ref = 0.5 * (1 / 3) * math.sqrt(min(vols)) / np.linalg.norm(v, axis=1).max()
    assert abs(o.dt_explicit() - ref) < 1e-15
