"""Checkpoint / resume and the lagged-edge export.

- bgk_save / bgk_load: a handle resumed from a checkpoint takes the next step bit for bit
  as the saving handle does (f, iteration counts), for one-stage, multi-stage and BDF2
  (history) integrators and the mixed-precision path; files that do not match the problem
  are refused with BGK_E_IO.
- bgk_get_lagged_edges: the lagged edges of every ordinate equal the oracle's (Tarjan + DFS
  from the smallest cell id, Sec. 4.1) on a mesh whose sweep graphs have cycles."""
import os

import numpy as np
import pytest

from paper_2608_19150_b300 import bgk, synth

from gpu_common import make_pair, twisted_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integ,precision", [("BE", "fp64"), ("DIRK3", "fp64"), ("BDF2", "fp64"),
                                             ("BDF2", "mixed"), ("DIRK2", "fp32")])
def test_resume_is_bit_identical(tmp_path, integ, precision):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, integrator=integ, knudsen=0.05)
    tau = 1e-6 if precision == "fp32" else 1e-8
    a = bgk.Solver.from_workload(w, precision=precision, tau=tau)
    a.set_state_maxwellian(w.init)
    a.set_inflow_maxwellian(w.inflow)
    a.step(2)
    path = str(tmp_path / "state.bgk")
    a.save(path)
    st_a = a.step(1)
    f_a = a.get_f(a.fdtype)
    b = bgk.Solver.from_workload(w, precision=precision, tau=tau)
    b.set_inflow_maxwellian(w.inflow)
    b.load(path)
    assert b.time()[0] == 2
    st_b = b.step(1)
    np.testing.assert_array_equal(b.get_f(b.fdtype), f_a)
    assert list(st_b.iterations) == list(st_a.iterations)
    assert list(st_b.iterations_fp32) == list(st_a.iterations_fp32)
    assert a.time() == b.time() and a.time()[0] == 3


def test_mismatched_or_broken_files_are_refused(tmp_path):
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, knudsen=0.05)
    a = bgk.Solver.from_workload(w)
    a.set_state_maxwellian(w.init)
    path = str(tmp_path / "state.bgk")
    a.save(path)
    other = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, knudsen=0.07)    # another nu
    b = bgk.Solver.from_workload(other)
    with pytest.raises(bgk.BgkError) as e:
        b.load(path)
    assert e.value.status == bgk.BGK_E_IO
    c = bgk.Solver.from_workload(w, precision="fp32")                          # another storage type
    with pytest.raises(bgk.BgkError) as e:
        c.load(path)
    assert e.value.status == bgk.BGK_E_IO
    for kw in ({"collision": "linear"}, {"walls": {"y-": "reflect"}}):         # another model or walls
        x = bgk.Solver.from_workload(w, **kw)
        with pytest.raises(bgk.BgkError) as e:
            x.load(path)
        assert e.value.status == bgk.BGK_E_IO
    same = bgk.Solver.from_workload(w)
    same.load(path)
    with open(path, "r+b") as fh:                                               # truncated
        fh.truncate(os.path.getsize(path) // 2)
    d = bgk.Solver.from_workload(w)
    with pytest.raises(bgk.BgkError) as e:
        d.load(path)
    assert e.value.status == bgk.BGK_E_IO
    with pytest.raises(bgk.BgkError) as e:
        d.load(str(tmp_path / "missing.bgk"))
    assert e.value.status == bgk.BGK_E_IO


def test_failed_load_never_leaves_mixed_state(tmp_path):
    """A file refused at its header leaves the state as it was (the next step equals the
    step of an untouched handle); a file that matches but ends early leaves no state, so a
    step is refused (BGK_E_INVALID) until a state is set again."""
    w = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, knudsen=0.05)
    a = bgk.Solver.from_workload(w)
    a.set_state_maxwellian(w.init)
    a.set_inflow_maxwellian(w.inflow)
    a.step(1)
    path = str(tmp_path / "state.bgk")
    a.save(path)
    other = synth.workload_p1_square(n_side=6, n_v=12, k_v=2, knudsen=0.07)
    bad_header = str(tmp_path / "other.bgk")
    o = bgk.Solver.from_workload(other)
    o.set_state_maxwellian(other.init)
    o.save(bad_header)
    truncated = str(tmp_path / "short.bgk")
    with open(path, "rb") as src, open(truncated, "wb") as dst:
        dst.write(src.read()[: os.path.getsize(path) * 2 // 3])
    ref = bgk.Solver.from_workload(w)
    ref.set_state_maxwellian(w.init)
    ref.set_inflow_maxwellian(w.inflow)
    ref.step(1)
    b = bgk.Solver.from_workload(w)
    b.set_state_maxwellian(w.init)
    b.set_inflow_maxwellian(w.inflow)
    b.step(1)
    with pytest.raises(bgk.BgkError) as e:
        b.load(bad_header)
    assert e.value.status == bgk.BGK_E_IO
    st_b, st_r = b.step(1), ref.step(1)
    np.testing.assert_array_equal(b.get_f(), ref.get_f())
    assert list(st_b.iterations) == list(st_r.iterations)
    with pytest.raises(bgk.BgkError) as e:
        b.load(truncated)
    assert e.value.status == bgk.BGK_E_IO
    with pytest.raises(bgk.BgkError) as e:
        b.step(1)
    assert e.value.status == bgk.BGK_E_INVALID
    b.load(path)                                  # a good file restores a usable state
    st_b, st_a = b.step(1), a.step(1)
    np.testing.assert_array_equal(b.get_f(), a.get_f())
    assert list(st_b.iterations) == list(st_a.iterations)


def test_lagged_edges_match_the_oracle():
    w = twisted_workload(3, 8)
    s, o = make_pair(w)
    total = 0
    for j in range(s.nv):
        e = s.lagged_edges(j)
        gen, _ = s.generations(j)
        _, lag, _ = o.generations(j)
        want = set()
        for d in range(o.ncell):
            nb = o.cell(d)["nbr"]
            for f in range(lag.shape[1]):
                if lag[d, f]:
                    want.add((int(nb[f]), d))
        got = set((int(u), int(d)) for u, d in e)
        assert got == want, j
        for u, d in got:
            assert gen[u] >= gen[d]
        total += len(got)
    assert total == s.lagged > 0
