"""The element choice of the Sod strip (reading of Sec. 5.1.1's grid), checked with the
oracle at small velocity grids: at the paper's dt = 1.76e-3, P1 triangles let the
temperature go negative one cell downwind of the initial jump within two steps, while the
paper's Q1 quadrilaterals and P2 triangles stay physical; and the workload's geometry is the
paper's strip."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_19150_b300 import synth


def _steps(w, k):
    o = Oracle.from_workload(w)
    o.build_dags()
    o.set_physics(w.nu, w.dt, "BE", 1e-8 / max(1.0, w.nu * w.dt), 3000)
    f, fbc = o.maxwellian(w.init), o.maxwellian(w.inflow)
    for _ in range(k):
        f, it, meas, st = o.step(f, fbc)
        if st:
            return st
    return 0


def test_strip_geometry_is_the_papers():
    w = synth.workload_sod_strip(n_v=8)
    x = w.mesh.xyz
    assert w.mesh.cells.shape == (256 * 6, 4)
    np.testing.assert_allclose([x[:, 0].min(), x[:, 0].max(), x[:, 1].min(), x[:, 1].max()],
                               [-1, 1, -3 / 128, 3 / 128], atol=1e-15)
    p = x[w.mesh.cells]
    np.testing.assert_allclose(p[:, 0] + p[:, 2], p[:, 1] + p[:, 3], atol=1e-15)   # parallelograms
    assert w.walls == {"y-": "reflect", "y+": "reflect"} and w.dt == 1.76e-3
    cent = p.mean(1)[:, 0]
    n0 = w.init.reshape(-1, 4, 4)[:, 0, 0]
    assert np.all(n0[cent < 0] == 1.0) and np.all(n0[cent > 0] == 0.125)


@pytest.mark.parametrize("kind,physical", [("q1", True), ("p2", True), ("p1", False)])
def test_sod_strip_elements_at_the_papers_time_step(kind, physical):
    w = synth.workload_sod_strip(n_v=8, knudsen=1.0, quads=kind == "q1", kx=2 if kind == "p2" else 1)
    st = _steps(w, 2)
    assert (st == 0) == physical, st


def test_disc_problem_geometry():
    w = synth.workload_sod_2d(n=40, n_v=8)
    p = w.mesh.xyz[w.mesh.cells]
    inside = w.init.reshape(-1, 4, 4)[:, 0, 0] == 1.0
    area = (np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 3, 1] - p[:, 0, 1]))[inside]).sum()
    assert abs(area - np.pi * 0.16) < 0.05 * np.pi * 0.16
    assert w.walls is None and w.cfl == 7.0
