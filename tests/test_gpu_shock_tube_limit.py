"""The shock tube's loss of positivity is the method's, not the GPU path's.

Unlimited P2 DG at the 8:1 density jump of the shock-tube workload undershoots behind the
jump until the temperature of one node turns negative (positivity of the discrete
solution is not guaranteed, Sec. 1/3.3; no limiter is part of the method).  On 16x16
squares with 8x8 velocities at CFL 10 the oracle reports it in the sixth step.  The CUDA
path, FP64 and mixed precision, must agree with the oracle step by step up to that point
(f within 1e-12, equal Picard counts for FP64) and report BGK_E_NONPHYSICAL in the same
step.  The benchmark restores its input state before every step, so it runs any number of
steps on this workload."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2608_19150_b300 import bgk

from gpu_common import make_pair, rel_err, small_shock_tube

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_oracle(o, w, dt, steps):
    o.set_physics(w.nu, dt, "DIRK3", 1e-8, 1000)
    f = o.maxwellian(w.init)
    fbc = o.maxwellian(w.inflow)
    out = []
    for _ in range(steps):
        f, it, _, status = o.step(f, fbc)
        out.append((status, list(it), f.copy()))
        if status != 0:
            break
    return out


def test_gpu_and_oracle_turn_nonphysical_in_the_same_step():
    w = small_shock_tube(n=16, kx=2, n_v=8, integrator="DIRK3")
    s, o = make_pair(w)
    ref = _run_oracle(o, w, s.dt, 12)
    assert ref[-1][0] == 5, "the oracle stays physical: the premise of this test changed"
    k_fail = len(ref) - 1
    assert k_fail >= 3
    s.set_state_maxwellian(w.init)
    s.set_inflow_maxwellian(w.inflow)
    for k, (status, it, f) in enumerate(ref):
        if status == 0:
            st = s.step(1)
            assert list(st.iterations) == it, (k, list(st.iterations), it)
            assert rel_err(s.get_f(), f) < 1e-12, (k, rel_err(s.get_f(), f))
        else:
            with pytest.raises(bgk.BgkError) as e:
                s.step(1)
            assert e.value.status == bgk.BGK_E_NONPHYSICAL, k
    # the mixed path (FP32 phase, then FP64) fails in the same step as well
    m = bgk.Solver.from_workload(w, precision="mixed")
    m.set_state_maxwellian(w.init)
    m.set_inflow_maxwellian(w.inflow)
    for k in range(k_fail):
        m.step(1)
        assert rel_err(m.get_f(), ref[k][2]) < 1e-6, k
    with pytest.raises(bgk.BgkError) as e:
        m.step(1)
    assert e.value.status == bgk.BGK_E_NONPHYSICAL


def test_bench_runs_past_the_nonphysical_time():
    """bench.py on the same small shock tube with more warm-up and timed steps than the
    problem stays physical for: every step starts from the restored input state."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--n-side", "16", "--n-v", "8", "--steps", "8",
           "--warmup", "3", "--sweep-reps", "2", "--no-cpu-baseline"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["steps"] == 8 and line["value"] > 0
    assert len(line["picard_iterations"]) == 8
    # the same input state every step: the same iteration counts every step
    assert all(i == line["picard_iterations"][0] for i in line["picard_iterations"])
    for key in ("roofline", "e2e", "plain_fp64"):
        assert line[key], key
    assert np.isfinite(line["roofline"]["frac"])
