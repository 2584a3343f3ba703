"""Shared helpers of the GPU parity tests (no solver arithmetic here)."""
import numpy as np

from oracle.oracle import Oracle
from paper_2608_19150_b300 import bgk, synth


def make_pair(w, **kw):
    """The same workload on the CUDA path and on the oracle."""
    s = bgk.Solver.from_workload(w, **kw)
    o = Oracle.from_workload(w)
    o.build_dags()
    return s, o


def rel_err(a, b):
    """max |a - b| / max |b| (norm-wise relative error)."""
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / np.abs(b).max())


def small_shock_tube(n=12, kx=2, n_v=16, integrator="DIRK3", knudsen=1e-3):
    return synth.workload_shock_tube(n_side=n, seed=1, kx=kx, n_v=n_v, knudsen=knudsen, integrator=integrator)


def twisted_workload(n=3, n_v=8, integrator="BE"):
    m = synth.twisted_cube_mesh(n, 0, 0.25, 2.0)
    x = synth.node_coords(m, 1).reshape(-1, 3)
    nn = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 2])
    u = np.zeros_like(x)
    th = 1.0 + 0.1 * np.cos(2 * np.pi * x[:, 1])
    init = np.concatenate([nn[:, None], u, th[:, None]], axis=1)
    inflow = np.concatenate([np.ones((nn.size, 1)), u, np.ones((nn.size, 1))], axis=1)
    return synth.Workload("twisted", m, 1, n_v, 3, 6.0, 1e-2, integrator, 8.0, init, inflow)
