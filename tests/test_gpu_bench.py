"""bench.py end to end on a small cube: one JSON line with the keys of the benchmark
contract, and an end-to-end leg that replays the timed steps bit for bit."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_on_a_small_cube():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cells", "8", "--steps", "6", "--warmup", "3",
           "--skip-serving", "--skip-cpu-baseline", "--fp64-steps", "1", "--profile-steps", "2",
           "--steady-steps", "12"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches", "roofline"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 6 and line["warmup"] == 3
    assert line["gpu_launches"] > 0
    assert line["e2e"]["replay_bit_identical"] is True
    assert line["e2e"]["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] > 0
    rf = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert 0 < rf["frac"] < 1.5
    assert line["fp64"]["value"] > 0
    assert line["mixed_error_vs_fp64"]["force_rmse_eV_per_A"] < 1e-3
    st = line["steady_state"]
    assert st["steps"] == 12 and st["value"] > 0 and st["ms_per_build"] > 0
    assert 0 <= st["rebuild_share"] < 1
