"""The benchmark's JSON contract on CPU: the reference arm (the oracle) prints one line with
the keys the contract names, for small configurations of the workloads; and the launch tally of a
step counts the wall refresh once per iteration."""
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


@pytest.mark.parametrize("args", [["--workload", "sod2d", "--n-side", "12", "--n-v", "8"],
                                  ["--workload", "sod", "--n-side", "16", "--n-v", "8"],
                                  ["--workload", "p1_square"],
                                  ["--workload", "shock_tube", "--n-side", "8", "--n-v", "8"]])
def test_reference_arm_prints_one_contract_line(args):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"] + args,
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    # the oracle's OpenMP build on every core this process may use
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert "OpenMP" in d["cpu_baseline"]["sample"] and d["cpu_baseline"]["cpu_model"]
    assert ("wall faces" in d["cpu_baseline"]["sample"]) == (args[1] == "sod")   # the strip has walls


def test_launch_tally_counts_the_wall_refresh():
    sys.path.insert(0, ROOT)
    import bench
    st = SimpleNamespace(n_stages=2, iterations=[3, 4, 0], iterations_fp32=[5, 0, 0])
    plain = bench.launches_per_step(st)
    walls = bench.launches_per_step(st, walls=True)
    # one refresh per FP64 iteration (7) and per FP32 iteration (5)
    assert walls - plain == 7 + 5


def test_launch_tally_counts_the_refinement_iterations():
    sys.path.insert(0, ROOT)
    import bench
    st = SimpleNamespace(n_stages=1, iterations=[3, 0, 0], iterations_fp32=[5, 0, 0])
    full = bench.launches_per_step(st)
    refined = bench.launches_per_step(st, refine=True)
    # the first FP64 iteration as before (5); each later one 5 kernels with the projected
    # Maxwellian (factor change, source change, sweep, update with moments, test), 6 with
    # the other collision models (factor pass and difference)
    assert refined - full == 0
    assert bench.launches_per_step(st, refine=True, projected=False) - full == 2 * (6 - 5)
    # walls: the refresh in every iteration, corrections included
    assert bench.launches_per_step(st, refine=True, walls=True) - refined == 3 + 5
