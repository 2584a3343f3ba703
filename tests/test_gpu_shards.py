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


@pytest.mark.parametrize("integ", ["BE", "DIRK2", "DIRK3", "BSTABLE2", "BDF2"])
@pytest.mark.parametrize("name", ["p2_tri", "p1_tet"])
def test_sharded_steps_with_one_handle_per_shard(name, integ):
    """shard.sharded_steps over four Solver handles (one per part, as four devices would hold
    them; the library sums the partial moments in part order and computes the measure)
    reproduces three steps of one handle for every integrator: the same Picard counts in
    every stage, and every part's ordinates within 1e-12."""
    import torch
    w = _cases()[name]
    w = synth.Workload(w.name, w.mesh, w.kx, w.n_v, w.k_v, w.L, w.knudsen, integ, w.cfl, w.init, w.inflow)
    ref = bgk.Solver.from_workload(w)
    ref.set_state_maxwellian(w.init)
    ref.set_inflow_maxwellian(w.inflow)
    its_ref = []
    for _ in range(3):
        st = ref.step(1)
        its_ref.append(list(st.iterations)[:st.n_stages])
    ranges = shard.ordinate_shards(w.n_v, ref.dim, 4)
    stream = torch.cuda.current_stream().cuda_stream
    parts = []
    for k, (a, b) in enumerate(ranges):
        # two parts on torch's stream, two on streams of their own (host-ordered)
        s = bgk.Solver.from_workload(w, stream=stream if k % 2 == 0 else None)
        s.set_state_maxwellian(w.init)
        s.set_inflow_maxwellian(w.inflow)
        parts.append(shard.SolverShard(s, a, b))
    assert [p.same_stream for p in parts] == [True, False, True, False]
    its = shard.sharded_steps(parts, 3)
    assert its == its_ref, (its, its_ref)
    fr = ref.get_f()
    scale = np.abs(fr).max()          # the FP64 tolerance is relative to the array's scale
    for p, (a, b) in zip(parts, ranges):
        assert np.abs(p.s.get_f()[a:b] - fr[a:b]).max() / scale < 1e-12
    assert parts[0].s.time() == ref.time()


def test_shard_calls_refuse_mixed_precision_and_out_of_order_use():
    w = _cases()["p2_tri"]
    m = bgk.Solver.from_workload(w, precision="mixed")
    m.set_state_maxwellian(w.init)
    with pytest.raises(bgk.BgkError):
        m.shard_step_begin()
    s = bgk.Solver.from_workload(w)
    s.set_state_maxwellian(w.init)
    with pytest.raises(bgk.BgkError):
        s.shard_stage_begin(0)            # no step open
    n, tol = s.shard_step_begin()
    assert n == 1 and tol == pytest.approx(1e-8 / max(1.0, w.nu * s.dt))
    with pytest.raises(bgk.BgkError):
        s.shard_stage_begin(1)            # backward Euler has one stage


def test_fixed_order_sum_and_measure_on_device():
    """bgk_sum_partials_device adds the parts in order; bgk_conv_measure_device gives the
    measure of Eq. (convergence-criteria) of two moment arrays (numpy reference)."""
    import torch
    w = _cases()["p2_tri"]
    s = bgk.Solver.from_workload(w)
    g = torch.Generator().manual_seed(3)
    parts = (torch.rand((3, s.nnode, s.dim + 2), generator=g, dtype=torch.float64) - 0.5) * torch.tensor(
        [1.0, 1e3, 1e-3, 10.0], dtype=torch.float64)
    d = parts.cuda()
    out = torch.empty((s.nnode, s.dim + 2), dtype=torch.float64, device="cuda")
    s.sum_partials_device(d.data_ptr(), 3, out.data_ptr())
    s.synchronize()
    expect = parts[0] + parts[1] + parts[2]
    assert torch.equal(out.cpu(), expect)
    Uo = (expect + 2.0).cuda()
    Un = Uo * (1.0 + 1e-4 * torch.rand(Uo.shape, generator=g, dtype=torch.float64).cuda())
    m = s.conv_measure_device(Un.data_ptr(), Uo.data_ptr())
    a, b = Un.cpu().numpy(), Uo.cpu().numpy()
    nrm = np.linalg.norm
    ref = max(nrm(a[:, 0] - b[:, 0]) / nrm(b[:, 0]),
              nrm(a[:, 1:3] - b[:, 1:3]) / max(nrm(b[:, 1:3]), nrm(b[:, 0])),
              nrm(a[:, 3] - b[:, 3]) / nrm(b[:, 3]))
    assert m == pytest.approx(ref, rel=1e-12)
