"""Edge cases on the CPU: invalid problems are rejected by the oracle and by the C ABI
(host-side validation in bgk_create needs no GPU and never launches a kernel on bad
input), and the degenerate velocity grid of a single cell per dimension (extended to
+-infinity on both sides) keeps the projection exact."""
import ctypes as C

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_19150_b300 import bgk, synth


def _create(dim, kx, xyz, cells, n1d=8, kv=3, L=6.0, integ="BE", collision=0, walls=(0,) * 6):
    lib = bgk.load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    m = bgk.Mesh(dim, kx, xyz.shape[0], bgk._ptr(xyz), cells.shape[0], bgk._ptr(cells))
    vg = bgk.VGrid(L, n1d, kv)
    ph = bgk.Physics(1.0, bgk.INTEGRATORS[integ], 0.0, 10.0, collision, (C.c_int * 6)(*walls))
    h = C.c_void_p()
    rc = lib.bgk_create(C.byref(m), C.byref(vg), C.byref(ph), None, C.byref(h))
    return rc


def test_invalid_problems_are_rejected_before_any_device_work():
    m = synth.square_mesh(2, 0)
    # vertex index out of range
    bad = m.cells.copy()
    bad[0, 0] = 10 ** 6
    assert _create(2, 1, m.xyz, bad) == bgk.BGK_E_INVALID
    # degenerate (zero-area) triangle
    deg = m.cells.copy()
    deg[0] = [deg[0, 0], deg[0, 0], deg[0, 1]]
    assert _create(2, 1, m.xyz, deg) == bgk.BGK_E_INVALID
    # P2 tetrahedra are not supported; unknown dimension
    c = synth.cube_mesh(1, 0)
    assert _create(3, 2, c.xyz, c.cells) == bgk.BGK_E_INVALID
    assert _create(4, 1, c.xyz, c.cells) == bgk.BGK_E_INVALID
    # velocity grid: points not a multiple of k_v + 1, k_v out of range, too many points
    assert _create(2, 1, m.xyz, m.cells, n1d=10, kv=3) == bgk.BGK_E_INVALID
    assert _create(2, 1, m.xyz, m.cells, n1d=12, kv=5) == bgk.BGK_E_INVALID
    assert _create(2, 1, m.xyz, m.cells, n1d=132, kv=3) == bgk.BGK_E_INVALID
    assert _create(2, 1, m.xyz, m.cells, L=-1.0) == bgk.BGK_E_INVALID
    # empty mesh
    assert _create(2, 1, m.xyz, np.zeros((0, 3), dtype=np.int32)) == bgk.BGK_E_INVALID
    # a non-conforming mesh: one square split twice along different diagonals
    xyz = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    cells = np.array([[0, 1, 2], [0, 2, 3], [0, 1, 3]], dtype=np.int32)  # three triangles overlap
    assert _create(2, 1, xyz, cells) == bgk.BGK_E_INVALID
    # unknown collision model or boundary kind (only the first 2d wall entries are read)
    assert _create(2, 1, m.xyz, m.cells, collision=3) == bgk.BGK_E_INVALID
    assert _create(2, 1, m.xyz, m.cells, walls=(0, 0, 3, 0, 0, 0)) == bgk.BGK_E_INVALID
    assert _create(2, 1, m.xyz, m.cells, walls=(0, -1, 0, 0, 0, 0)) == bgk.BGK_E_INVALID
    assert _create(3, 1, c.xyz, c.cells, walls=(0, 0, 0, 0, 0, 9)) == bgk.BGK_E_INVALID
    # quadrilaterals: a non-parallelogram cell; a quad with k_x = 2
    lib = bgk.load()
    q = np.array([[0, 0], [1.2, 0.1], [1.0, 0.9], [-0.1, 1.1]], dtype=np.float64)
    qc = np.array([[0, 1, 2, 3]], dtype=np.int32)
    for kx, xyz in ((1, q), (2, np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64))):
        mq = bgk.Mesh(2, kx, 4, bgk._ptr(xyz), 1, bgk._ptr(qc), 1)
        h = C.c_void_p()
        assert lib.bgk_create(C.byref(mq), C.byref(bgk.VGrid(6.0, 8, 3)), C.byref(bgk.Physics(1.0, 0, 0.0, 10.0)),
                              None, C.byref(h)) == bgk.BGK_E_INVALID
    # and the oracle refuses the same bad inputs
    with pytest.raises(ValueError):
        Oracle(2, 1, m.xyz, bad, 8, 3, 6.0)
    with pytest.raises(ValueError):
        Oracle(2, 1, m.xyz, m.cells, 10, 3, 6.0)


@pytest.mark.parametrize("kv", [1, 2, 3, 4])
def test_single_velocity_cell_projection_is_exact(kv):
    """One velocity cell per dimension: both ends extended to infinity (App. B)."""
    m = synth.square_mesh(1, 0)
    o = Oracle(2, 1, m.xyz, m.cells, kv + 1, kv, 3.0)
    _, w, _, w1 = o.velocity()
    for (u, th) in [(0.0, 1.0), (1.5, 0.5), (-2.0, 2.0)]:
        c = o.project_1d(u, th)
        assert abs(np.dot(w1, c) - 1.0) < 1e-13
        if kv >= 2:
            nut = np.tile([1.3, u, -0.5 * u, th], (o.nnode, 1))
            U = o.moments(o.maxwellian(nut))[0]
            exact = [1.3, 1.3 * u, -0.65 * u, 0.5 * 1.3 * (u * u + 0.25 * u * u) + 1.3 * th]
            np.testing.assert_allclose(U, exact, rtol=1e-12, atol=1e-13)


def test_one_cell_mesh_all_faces_on_the_boundary():
    """A single triangle: every face is a boundary face, every sweep graph has one node."""
    xyz = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    o = Oracle(2, 1, xyz, cells, 8, 3, 6.0)
    assert o.build_dags() == 0
    for j in range(o.nv):
        gen, lag, G = o.generations(j)
        assert G == 1 and gen[0] == 0
    nut = np.tile([1.0, 0.0, 0.0, 1.0], (o.nnode, 1))
    f0 = o.maxwellian(nut)
    o.set_physics(5.0, 0.01, "DIRK3")
    f1, it, meas, st = o.step(f0, f0)
    assert st == 0
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-14 * np.abs(f0).max())
