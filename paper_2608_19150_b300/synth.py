"""Seeded synthetic inputs: meshes, spatial node positions and primitive states.

This module holds no arithmetic of the solver itself.  It only draws the seeded
triangulations / tetrahedralisations and evaluates the initial and inflow states
(density n, bulk velocity u, temperature theta) that the workloads prescribe, at the
nodal points of the spatial DG basis.  Both the CUDA path and the CPU oracle receive
the same arrays from here.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), evaluated in closed
form on a counter, so every draw is reproducible on any machine.

Node ordering of a cell (the interface convention shared by every consumer):
  triangle P1: vertices 0,1,2;  triangle P2: vertices 0,1,2 then the midpoints of the
  edges (0,1), (1,2), (2,0);  tetrahedron P1: vertices 0,1,2,3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): outputs offset..offset+count-1 of splitmix64(seed)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray          # [n_vertices, dim] float64
    cells: np.ndarray        # [n_cells, dim+1] int32, positively oriented
    n_side: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.xyz.shape[0])


def square_mesh(n: int, seed: int, jitter: float = 0.2) -> Mesh:
    """Unit square: n x n squares, each cut into two triangles along a seeded diagonal.

    Interior vertices move by independent uniform offsets in [-jitter*h, jitter*h] per
    coordinate (h = 1/n); boundary vertices stay put.  Triangles are counter-clockwise.
    """
    h = 1.0 / n
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    vid = lambda i, j: i * (n + 1) + j  # noqa: E731
    r = splitmix64_uniform(seed, 2 * (n + 1) ** 2 + n * n)
    jit = (2.0 * r[: 2 * (n + 1) ** 2].reshape(-1, 2) - 1.0) * (jitter * h)
    interior = ((ii.ravel() > 0) & (ii.ravel() < n) & (jj.ravel() > 0) & (jj.ravel() < n))
    xyz[interior] += jit[interior]
    diag = r[2 * (n + 1) ** 2:] < 0.5
    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    k = 0
    for i in range(n):
        for j in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if diag[i * n + j]:       # diagonal a-c
                cells[k] = (a, b, c)
                cells[k + 1] = (a, c, d)
            else:                     # diagonal b-d
                cells[k] = (a, b, d)
                cells[k + 1] = (b, c, d)
            k += 2
    return Mesh(2, xyz, cells, n_side=n, seed=seed)


def rect_mesh(nx: int, ny: int, seed: int, jitter: float = 0.2) -> Mesh:
    """[0, 1] x [0, ny/nx]: nx x ny squares of side h = 1/nx, each cut into two triangles
    along a seeded diagonal, interior vertices jittered as in square_mesh (a strip when
    ny << nx)."""
    h = 1.0 / nx
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    vid = lambda i, j: i * (ny + 1) + j  # noqa: E731
    nvert = (nx + 1) * (ny + 1)
    r = splitmix64_uniform(seed, 2 * nvert + nx * ny)
    jit = (2.0 * r[: 2 * nvert].reshape(-1, 2) - 1.0) * (jitter * h)
    interior = (ii.ravel() > 0) & (ii.ravel() < nx) & (jj.ravel() > 0) & (jj.ravel() < ny)
    xyz[interior] += jit[interior]
    diag = r[2 * nvert:] < 0.5
    cells = np.empty((2 * nx * ny, 3), dtype=np.int32)
    k = 0
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if diag[i * ny + j]:
                cells[k] = (a, b, c)
                cells[k + 1] = (a, c, d)
            else:
                cells[k] = (a, b, d)
                cells[k + 1] = (b, c, d)
            k += 2
    return Mesh(2, xyz, cells, n_side=nx, seed=seed, meta={"ny": ny})


def rect_quad_mesh(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=None, shear=0.0) -> Mesh:
    """[x0, x1] x [y0, y1] as an nx x ny grid of Q1 quadrilaterals (vertices counter-
    clockwise from the lower left); y1 defaults to a square-celled strip.  shear > 0 slants
    every cell into a parallelogram: x += shear * (y - y0)."""
    h = (x1 - x0) / nx
    if y1 is None:
        y1 = y0 + ny * h
    xs, ys = np.linspace(x0, x1, nx + 1), np.linspace(y0, y1, ny + 1)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    xyz = np.stack([xs[ii.ravel()], ys[jj.ravel()]], axis=1).astype(np.float64)
    xyz[:, 0] += shear * (xyz[:, 1] - y0)
    vid = lambda i, j: i * (ny + 1) + j  # noqa: E731
    cells = np.array([[vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)]
                      for i in range(nx) for j in range(ny)], dtype=np.int32)
    return Mesh(2, xyz, cells, n_side=nx, meta={"ny": ny, "quad": True})


# Kuhn (Freudenthal) split of the unit cube into 6 tetrahedra sharing the main
# diagonal from corner 0 to corner 7; corners are indexed by bits (x, y, z).
_KUHN = [(0, 1, 3, 7), (0, 3, 2, 7), (0, 2, 6, 7), (0, 6, 4, 7), (0, 4, 5, 7), (0, 5, 1, 7)]


def cube_mesh(n: int, seed: int, jitter: float = 0.15) -> Mesh:
    """Unit cube: n^3 cubes, 6 tetrahedra each (conforming Kuhn split), interior jitter."""
    h = 1.0 / n
    g = np.arange(n + 1)
    ii, jj, kk = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h, kk.ravel() * h], axis=1).astype(np.float64)
    nv = (n + 1) ** 3
    r = splitmix64_uniform(seed, 3 * nv)
    jit = (2.0 * r.reshape(-1, 3) - 1.0) * (jitter * h)
    interior = np.ones(nv, dtype=bool)
    for a in (ii, jj, kk):
        interior &= (a.ravel() > 0) & (a.ravel() < n)
    xyz[interior] += jit[interior]
    base = (ii[:n, :n, :n].ravel() * (n + 1) + jj[:n, :n, :n].ravel()) * (n + 1) + kk[:n, :n, :n].ravel()
    corner = [((c >> 0) & 1) * (n + 1) * (n + 1) + ((c >> 1) & 1) * (n + 1) + ((c >> 2) & 1) for c in range(8)]
    cells = np.empty((6 * n ** 3, 4), dtype=np.int64)
    for t, tet in enumerate(_KUHN):
        for q in range(4):
            cells[t::6, q] = base + corner[tet[q]]
    # orient positively
    p = xyz[cells]
    det = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    neg = det < 0
    cells[neg, 1], cells[neg, 2] = cells[neg, 2].copy(), cells[neg, 1].copy()
    return Mesh(3, xyz, cells.astype(np.int32), n_side=n, seed=seed)


def twisted_cube_mesh(n: int, seed: int, jitter: float = 0.25, alpha: float = 2.0) -> Mesh:
    """Jittered Kuhn mesh of the unit cube, twisted about the axis x = y = 1/2 by the
    angle alpha * z.  Straight-sided tetrahedral meshes this twisted have cyclic sweep
    graphs for some ordinates (jittered Kuhn and Delaunay meshes do not), so this mesh
    exercises the lagging of cycle edges.  Raises if any tetrahedron would invert."""
    m = cube_mesh(n, seed, jitter)
    x = m.xyz.copy()
    c, s = np.cos(alpha * x[:, 2]), np.sin(alpha * x[:, 2])
    X, Y = x[:, 0] - 0.5, x[:, 1] - 0.5
    x[:, 0] = 0.5 + c * X - s * Y
    x[:, 1] = 0.5 + s * X + c * Y
    p = x[m.cells]
    det = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    if not np.all(det > 0):
        raise ValueError("twist too strong: inverted tetrahedra")
    return Mesh(3, x, m.cells.copy(), n_side=n, seed=seed, meta=dict(alpha=alpha))


def node_coords(mesh: Mesh, kx: int) -> np.ndarray:
    """Positions of the spatial DG nodes, [n_cells, n_nodes, dim], in the cell node order."""
    p = mesh.xyz[mesh.cells]
    if kx == 1:
        return p.copy()          # P1 simplices and Q1 quadrilaterals: the vertices
    if kx == 2 and mesh.dim == 2:
        mids = [(p[:, 0] + p[:, 1]) * 0.5, (p[:, 1] + p[:, 2]) * 0.5, (p[:, 2] + p[:, 0]) * 0.5]
        return np.concatenate([p, np.stack(mids, axis=1)], axis=1)
    raise ValueError("supported spatial elements: P1 triangles, P2 triangles, P1 tetrahedra")


@dataclass
class Workload:
    """One workload: mesh, DG order, velocity grid, physics and nodal states."""
    name: str
    mesh: Mesh
    kx: int
    n_v: int                 # velocity points per dimension
    k_v: int                 # velocity polynomial degree (k_v + 1 Gauss points per cell)
    L: float
    knudsen: float
    integrator: str          # "BE", "DIRK2", "DIRK3", "BSTABLE2", "BDF2"
    cfl: float
    init: np.ndarray         # [n_cells*n_nodes, dim+2]: n, u_1..u_d, theta per node
    inflow: np.ndarray       # same layout; used at nodes on inflow boundary faces
    dt: float = 0.0          # time step; 0: from the CFL number
    walls: dict = None       # Sec. 4.2 wall kinds per box side ({"y-": "reflect", ...}); None: inflow

    @property
    def nu(self) -> float:
        return 1.0 / self.knudsen


def _pack(n, u, th):
    return np.concatenate([n[:, None], u, th[:, None]], axis=1).astype(np.float64)


def workload_p1_square(n_side=16, seed=0, n_v=16, k_v=3, L=6.0, knudsen=1e-2,
                       integrator="BE", cfl=10.0) -> Workload:
    """2D-2V smooth problem: n = 1 + 0.2 sin(2 pi x) sin(2 pi y), u = 0,
    theta = 1 + 0.1 cos(2 pi x); inflow Maxwellian (1, 0, 1) on every boundary."""
    mesh = square_mesh(n_side, seed, 0.2)
    x = node_coords(mesh, 1).reshape(-1, 2)
    n = 1.0 + 0.2 * np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1])
    th = 1.0 + 0.1 * np.cos(2 * np.pi * x[:, 0])
    u = np.zeros_like(x)
    init = _pack(n, u, th)
    inflow = _pack(np.ones_like(n), u, np.ones_like(n))
    return Workload("2d2v_p1_smooth_%dx%d_v%d" % (n_side, n_side, n_v), mesh, 1, n_v, k_v, L,
                    knudsen, integrator, cfl, init, inflow)


def workload_strip(nx=1024, ny=2, seed=5, kx=1, n_v=32, k_v=3, L=6.0, knudsen=1e-2,
                   integrator="BE", cfl=10.0) -> Workload:
    """Quasi-1D smooth problem on a strip of nx x ny squares (narrow sweep generations):
    n = 1 + 0.2 sin(2 pi x), u = 0, theta = 1 + 0.1 cos(2 pi x); inflow Maxwellian (1, 0, 1)."""
    mesh = rect_mesh(nx, ny, seed, 0.2)
    x = node_coords(mesh, kx).reshape(-1, 2)
    n = 1.0 + 0.2 * np.sin(2 * np.pi * x[:, 0])
    th = 1.0 + 0.1 * np.cos(2 * np.pi * x[:, 0])
    u = np.zeros_like(x)
    init = _pack(n, u, th)
    inflow = _pack(np.ones_like(n), u, np.ones_like(n))
    return Workload("2d2v_strip_p%d_%dx%d_v%d" % (kx, nx, ny, n_v), mesh, kx, n_v, k_v, L, knudsen,
                    integrator, cfl, init, inflow)


def workload_shock_tube(n_side=128, seed=1, kx=2, n_v=32, k_v=3, L=8.0, knudsen=1e-3,
                        integrator="DIRK3", cfl=10.0) -> Workload:
    """2D-2V shock tube: left (n=1, theta=1), right (n=0.125, theta=0.8), u = 0, split at
    x = 0.5 by cell centroid; the inflow state at a boundary node is its initial state."""
    mesh = square_mesh(n_side, seed, 0.2)
    xn = node_coords(mesh, kx)
    cent = mesh.xyz[mesh.cells].mean(axis=1)[:, 0]
    left = np.repeat((cent < 0.5)[:, None], xn.shape[1], axis=1).ravel()
    n = np.where(left, 1.0, 0.125)
    th = np.where(left, 1.0, 0.8)
    u = np.zeros((n.size, 2))
    init = _pack(n, u, th)
    return Workload("2d2v_shock_tube_p%d_%dx%d_v%d" % (kx, n_side, n_side, n_v), mesh, kx, n_v,
                    k_v, L, knudsen, integrator, cfl, init, init.copy())


SOD_STEPS = 85            # Sec. 5.1.1: 85 steps of 1.76e-3 to t = 0.15 (0.14960)


def workload_sod_strip(nx=256, ny=6, kx=2, n_v=32, k_v=3, L=6.0, knudsen=1e-3, integrator="BE",
                       dt=1.76e-3, quads=True) -> Workload:
    """The 1D Sod problem in a 2D strip (Sec. 5.1.1): X = [-1, 1] x [-3/128, 3/128], an
    nx x ny uniform grid of Q1 quadrilaterals as in the paper (quads=False: each square cut
    into two triangles along a seeded diagonal, P_kx), left half (n, u, theta) = (1, 0, 1),
    right half (0.125, 0, 0.8) (pressures 1 and 0.1), reflecting walls at x_2 = +-3/128,
    the initial states as inflow data at x_1 = -1 and 1, dt = 1.76e-3.  On triangles use
    P2: with P1 triangles at this dt the density undershoots one cell downwind of the
    initial jump and the temperature there turns negative within two steps (Q1 and P2
    stay physical)."""
    if quads:
        mesh = rect_quad_mesh(nx, ny, -1.0, 1.0, -ny / nx, ny / nx)
        kx = 1
    else:
        m = rect_mesh(nx, ny, 7, jitter=0.0)
        xyz = m.xyz.copy()
        xyz[:, 0] = 2.0 * xyz[:, 0] - 1.0
        xyz[:, 1] = 2.0 * xyz[:, 1] - ny / nx          # square cells of side 2/nx, centred on x_2 = 0
        mesh = Mesh(2, xyz, m.cells, n_side=nx, seed=7, meta={"ny": ny})
    xn = node_coords(mesh, kx)
    cent = mesh.xyz[mesh.cells].mean(axis=1)[:, 0]
    left = np.repeat((cent < 0.0)[:, None], xn.shape[1], axis=1).ravel()
    n = np.where(left, 1.0, 0.125)
    th = np.where(left, 1.0, 0.8)
    u = np.zeros((n.size, 2))
    init = _pack(n, u, th)
    return Workload("2d2v_sod_strip_%s%d_%dx%d_v%d" % ("q" if quads else "p", kx, nx, ny, n_v), mesh, kx, n_v, k_v,
                    L, knudsen,
                    integrator, 0.0, init, init.copy(), dt=dt, walls={"y-": "reflect", "y+": "reflect"})


def workload_sod_2d(n=160, n_v=16, k_v=3, L=6.0, knudsen=1e-4, integrator="BE", cfl=7.0, dt=0.0) -> Workload:
    """The 2D Sod problem (Sec. 5.1.2): X = [0, 2]^2, inside the disc of radius 0.4 about
    (1, 1) the state (n, u, theta) = (1, 0, 1), outside (0.125, 0, 0.8) (split by cell
    centroid), the outer state as inflow data, to t = 0.15.  An n x n grid of Q1 squares
    (n = 160: 25,600 cells; the paper's quadrilateral grid has 25,545).  The time step is 7x
    the explicit one as in the paper (its dt = 3.7e-4 is 7x the explicit step of its locally
    finer grid; on this uniform grid that is 1.78e-3 at 16x16 velocities)."""
    mesh = rect_quad_mesh(n, n, 0.0, 2.0, 0.0, 2.0)
    xn = node_coords(mesh, 1)
    cent = mesh.xyz[mesh.cells].mean(axis=1)
    inside = np.repeat((((cent - 1.0) ** 2).sum(1) < 0.16)[:, None], xn.shape[1], axis=1).ravel()
    nn = np.where(inside, 1.0, 0.125)
    th = np.where(inside, 1.0, 0.8)
    init = _pack(nn, np.zeros((nn.size, 2)), th)
    return Workload("2d2v_sod_disc_q1_%dx%d_v%d" % (n, n, n_v), mesh, 1, n_v, k_v, L, knudsen, integrator, cfl,
                    init, init.copy(), dt=dt)


SOD_2D_T = 0.15


def workload_3d_bump(n_side=24, seed=2, n_v=16, k_v=3, L=6.0, knudsen=1e-2,
                     integrator="BE", cfl=8.0) -> Workload:
    """3D-3V Gaussian density bump n = 1 + 0.5 exp(-|x-0.5|^2/0.02), theta = 1, u = 0;
    inflow Maxwellian (1, 0, 1)."""
    mesh = cube_mesh(n_side, seed, 0.15)
    x = node_coords(mesh, 1).reshape(-1, 3)
    r2 = ((x - 0.5) ** 2).sum(axis=1)
    n = 1.0 + 0.5 * np.exp(-r2 / 0.02)
    u = np.zeros_like(x)
    th = np.ones_like(n)
    init = _pack(n, u, th)
    inflow = _pack(np.ones_like(n), u, np.ones_like(n))
    return Workload("3d3v_bump_%d^3_v%d" % (n_side, n_v), mesh, 1, n_v, k_v, L, knudsen,
                    integrator, cfl, init, inflow)


def workload_random_smooth(seed: int, n_side: int, kx: int, n_v: int, knudsen: float,
                           k_v=3, L=6.0, integrator="BE", cfl=10.0) -> Workload:
    """Random smooth sinusoidal initial moments (one instance of a batched run)."""
    mesh = square_mesh(n_side, seed, 0.2)
    x = node_coords(mesh, kx).reshape(-1, 2)
    r = splitmix64_uniform(seed ^ 0x5DEECE66D, 12)
    a, b, c = 0.2 * r[0], 0.2 * r[1], 0.3 * r[2]
    k1, k2, k3 = 1 + int(3 * r[3]), 1 + int(3 * r[4]), 1 + int(3 * r[5])
    p1, p2, p3 = 2 * np.pi * r[6], 2 * np.pi * r[7], 2 * np.pi * r[8]
    n = 1.0 + a * np.sin(2 * np.pi * k1 * x[:, 0] + p1) * np.sin(2 * np.pi * k2 * x[:, 1] + p2)
    th = 1.0 + b * np.cos(2 * np.pi * k3 * x[:, 0] + p3)
    u = c * np.stack([np.sin(2 * np.pi * x[:, 1] + p1), np.cos(2 * np.pi * x[:, 0] + p2)], axis=1)
    init = _pack(n, u, th)
    inflow = _pack(np.ones(n.size), np.zeros_like(u), np.ones(n.size))
    return Workload("2d2v_random_s%d" % seed, mesh, kx, n_v, k_v, L, knudsen, integrator,
                    cfl, init, inflow)


def batched_draw(count: int = 64, seed: int = 3):
    """Instance parameters of the batched workload: triangles log-uniform in [2k, 50k],
    P1 or P2 by a fair coin, N uniform in {16, 20, ..., 48}, Knudsen log-uniform 1e-4..1."""
    r = splitmix64_uniform(seed, 4 * count).reshape(count, 4)
    out = []
    for i in range(count):
        tri = math.exp(math.log(2000.0) + r[i, 0] * (math.log(50000.0) - math.log(2000.0)))
        m = max(2, int(round(math.sqrt(tri / 2.0))))
        kx = 1 if r[i, 1] < 0.5 else 2
        nv = 16 + 4 * int(r[i, 2] * 9)
        kn = 10.0 ** (-4.0 + 4.0 * r[i, 3])
        out.append(dict(seed=seed * 1000 + i, n_side=m, kx=kx, n_v=nv, knudsen=kn))
    return out
