"""Multi-rank aggregation of bench.py on CPU (gloo, world size 2).

Each rank times its own replica; the job's rate is all ranks' atom-steps over the
slowest rank's time.  Runs two gloo processes on 127.0.0.1; no GPU involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times_ms, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max = bench.max_over_ranks(times_ms[rank], dist, "cpu")
        out.put((rank, ms_max, bench.whole_job_rate(1000, 50, world, ms_max)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [10.0, 12.5]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 12.5
        assert rate == pytest.approx(1000 * 50 * 2 / 12.5e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(884736, 200, 1, 1000.0) == pytest.approx(884736 * 200.0)


def test_reference_arm_line_on_cpu():
    """bench.py --impl reference times the FP64 oracle on the host cores and prints the
    contract's line (a short budget here)."""
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3",
           "--ref-budget-s", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["unit"] == "atom-steps/s"


def test_reference_arm_other_ranks_exit_quietly(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup, ref_budget_s = 1, 3, 1.0
    assert bench.run_reference(A()) == 0


def test_roofline_arithmetic_and_traffic_guard(tmp_path, monkeypatch):
    """The per-kernel roofline is algorithmic work / measured time / peak, and a committed DRAM
    capture is only used while the evaluation kernels' sources hash to the recorded value."""
    import bench
    from paper_2606_14073_gb300 import flops
    fl = flops.per_atom(62.0, 16.0)
    prof = {"rad_fwd": 2.0, "ang_fwd": 1.0, "network": 0.4, "backward": 4.0}   # ms over 2 steps
    out = bench.kernel_rooflines(fl, prof, 2, 1_000_000, 80.0)
    assert abs(out["backward"]["achieved_tflops"] - fl["backward"] * 1e6 / 2e-3 / 1e12) < 1e-9
    assert abs(out["backward"]["frac"] - out["backward"]["achieved_tflops"] / 80.0) < 1e-12
    assert abs(out["network"]["achieved_gbs"] - bench.NETWORK_BYTES_PER_ATOM * 1e6 / 0.2e-3 / 1e9) < 1e-6
    # traffic: accepted with the current hash, refused with any other
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2606_14073_gb300").symlink_to(os.path.join(ROOT, "paper_2606_14073_gb300"))
    h = bench.kernel_source_hash()
    (prof_dir / "traffic_backward.txt").write_text(f"kernel_sources_sha256_16: {h}\ndram_bytes_per_launch_full_size: 123\n")
    assert bench.committed_traffic("backward") == 123.0
    (prof_dir / "traffic_backward.txt").write_text("kernel_sources_sha256_16: 0000\ndram_bytes_per_launch_full_size: 123\n")
    assert bench.committed_traffic("backward") is None


def test_neighbour_counts_of_the_crystal():
    """Mean neighbour counts inside 6 and 4 A on the seeded B20 cube: close to the density estimate
    (0.0771 atoms/A^3) and to the values the algorithmic-work counts use."""
    import bench
    from paper_2606_14073_gb300 import workloads as W
    nr, na = bench.neighbour_counts(W.fege_cube(8))
    assert abs(nr - 62.0) < 1.0 and abs(na - 16.0) < 1.0
