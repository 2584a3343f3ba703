"""Ordinate-sharded sweep, in-process on one GPU (Sec. 4: the ordinates' sweeps are
independent given the Maxwellian of the current moments; the sum over ordinates in
Eq. moments is the only coupling).  The parts' partial moments add up to the moments; the
parts' range sweeps with the summed moments reproduce the full sweep bit for bit; and a
Picard iteration run part by part, with the partial moments summed in part order between
sweeps, reproduces a backward-Euler step of the solver (same iteration count, f within the
FP64 tolerance)."""
import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, shard, synth

from gpu_common import rel_err, small_shock_tube, twisted_workload

pytestmark = pytest.mark.gpu


def _cases():
    return {"p2_tri": small_shock_tube(n=8, kx=2, n_v=16, integrator="BE"),
            "p1_tet": twisted_workload(3, 8)}


def _summed_moments(s, parts):
    import torch
    bufs = []
    for a, b in parts:
        buf = torch.empty((s.nnode, s.dim + 2), dtype=torch.float64, device="cuda")
        s.moments_range_device(a, b, buf.data_ptr())
        bufs.append(buf)
    tot = bufs[0].clone()
    for b_ in bufs[1:]:
        tot += b_
    return tot


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["p2_tri", "p1_tet"])
def test_partial_moments_add_up(name, precision):
    w = _cases()[name]
    s = bgk.Solver.from_workload(w, precision=precision)
    s.set_state_maxwellian(w.init)
    full = s.get_moments()
    for nparts in (1, 3):
        parts = shard.ordinate_shards(w.n_v, s.dim, nparts)
        tot = _summed_moments(s, parts).cpu().numpy()
        assert rel_err(tot, full) < 1e-13


def test_range_rejects_partial_outer_index():
    w = _cases()["p2_tri"]
    s = bgk.Solver.from_workload(w)
    import torch
    buf = torch.empty((s.nnode, s.dim + 2), dtype=torch.float64, device="cuda")
    with pytest.raises(bgk.BgkError):
        s.moments_range_device(0, w.n_v + 1, buf.data_ptr())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["p2_tri", "p1_tet"])
def test_range_sweeps_reproduce_the_full_sweep(name, precision):
    import torch
    w = _cases()[name]
    s1 = bgk.Solver.from_workload(w, precision=precision)
    s1.set_state_maxwellian(w.init)
    s1.set_inflow_maxwellian(w.inflow)
    U = torch.empty((s1.nnode, s1.dim + 2), dtype=torch.float64, device="cuda")
    s1.get_moments_device(U.data_ptr())
    s1.sweep(0.0, 0.0)
    f_full = s1.get_f(s1.fdtype)
    s2 = bgk.Solver.from_workload(w, precision=precision)
    s2.set_state_maxwellian(w.init)
    s2.set_inflow_maxwellian(w.inflow)
    for a, b in reversed(shard.ordinate_shards(w.n_v, s2.dim, 3)):   # any order of the parts
        s2.sweep_range(a, b, U.data_ptr())
    np.testing.assert_array_equal(s2.get_f(s2.fdtype), f_full)


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet"])
def test_sharded_picard_step_matches_the_step(name):
    import torch
    w = _cases()[name]
    ref = bgk.Solver.from_workload(w)
    ref.set_state_maxwellian(w.init)
    ref.set_inflow_maxwellian(w.inflow)
    st = ref.step(1)
    s = bgk.Solver.from_workload(w)
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    parts = shard.ordinate_shards(w.n_v, s.dim, 4)
    tol = 1e-8 / max(1.0, w.nu * s.dt)
    U_old = _summed_moments(s, parts)
    d = s.dim
    its = 0
    for its in range(1, 200):
        for a, b in parts:
            s.sweep_range(a, b, U_old.data_ptr())
        U_new = _summed_moments(s, parts)
        dU, Uo = (U_new - U_old).cpu().numpy(), U_old.cpu().numpy()
        n = np.linalg.norm
        m0 = n(dU[:, 0]) / n(Uo[:, 0])
        m1 = n(dU[:, 1:1 + d]) / max(n(Uo[:, 1:1 + d]), n(Uo[:, 0]))
        m2 = n(dU[:, -1]) / n(Uo[:, -1])
        U_old = U_new
        if max(m0, m1, m2) < tol:
            break
    assert its == st.iterations[0]
    assert rel_err(s.get_f(), ref.get_f()) < 1e-12


@pytest.mark.parametrize("name", ["p2_tri", "p1_tet"])
def test_sharded_be_steps_with_one_handle_per_shard(name):
    """shard.sharded_be_steps over four Solver handles (one per shard, as four devices would
    hold them; the summed moments added in shard order) reproduces three backward-Euler
    steps of one handle: the same Picard counts, and every shard's ordinates within 1e-12."""
    w = _cases()[name]
    ref = bgk.Solver.from_workload(w)
    ref.set_state_maxwellian(w.init)
    ref.set_inflow_maxwellian(w.inflow)
    its_ref = [ref.step(1).iterations[0] for _ in range(3)]
    ranges = shard.ordinate_shards(w.n_v, ref.dim, 4)
    parts = []
    for a, b in ranges:
        s = bgk.Solver.from_workload(w)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        parts.append(shard.SolverShard(s, a, b))
    its = shard.sharded_be_steps(parts, lambda U: U, ref.dim, w.nu, ref.dt, 1e-8, 3)
    assert its == its_ref
    fr = ref.get_f()
    for p, (a, b) in zip(parts, ranges):
        assert rel_err(p.s.get_f()[a:b], fr[a:b]) < 1e-12
