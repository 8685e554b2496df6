#!/usr/bin/env python
"""Benchmark of the NEP-SPIN spin-lattice step on GB300.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full pass of the hot path over the 884,736-atom FeGe B20 workload
(48^3 cells, ferromagnetic z with a 5 degree random cant, 300 K Langevin, dt 1 fs):
integrator first half, conditional neighbour rebuild, descriptor, network,
backward, force/field gather and spin corrector.  The timed region replays
captured CUDA graphs; its working set (~10 GB) is far larger than L2, so no
flush is needed between steps.

Under torchrun (N > 1) every rank runs its own replica of the workload on its
GPU (replicas only: the method has no data-path exchange between replicas);
value = atoms x steps of all ranks / max over ranks of the timed region.

--impl reference times the FP64 CPU oracle on the host cores instead (a bounded
sample of the same workload recipe per step) and prints the same kind of line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s on 1 GB300, mixed vs FP64 at stated force error; p99 replica latency"
UNIT = "atom-steps/s"
WORKLOAD = "fege_b20_48c_884736"
DT, TEMP, FIELD = 1.0, 300.0, (0.0, 0.0, 0.0)
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM on sm_100-class GPUs


def fp32_peak_tflops(device: int, sm_max_mhz: float | None):
    """FP32 FMA peak of the device: SM count from the device attribute x 128 lanes x 2 FLOP x the
    maximum SM clock (nvidia-smi's clocks.max.sm seen during the run, else MEASURED_PEAKS.json)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = sm_max_mhz or float((measured_peaks() or {}).get("sm_max_mhz", 2070.0))
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, sms, mhz


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 0.25 * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in load), sm_max_mhz=max(r["max"] for r in rows),
                    power_w_max=max(r["power"] for r in rows), samples=len(rows), reasons=sorted(reasons))


# ---------------------------------------------------------------- helpers
def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (x itself when not distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(atoms_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Atom-steps per second of the whole job: every rank steps its own replica of
    atoms_per_rank atoms, and the job takes as long as its slowest rank."""
    return atoms_per_rank * steps * world / (ms_max * 1e-3)


def neighbour_counts(wl, positions=None, sample=20000, seed=0):
    """Mean in-cutoff neighbour counts (6 A, 4 A) on a sample of atoms of the periodic
    workload wl, at its initial positions or at the given ones."""
    from scipy.spatial import cKDTree
    pos = np.mod(wl.positions if positions is None else positions, wl.box)
    tree = cKDTree(pos, boxsize=wl.box)
    idx = np.random.default_rng(seed).choice(wl.n, min(sample, wl.n), replace=False)
    nr = tree.query_ball_point(pos[idx], 6.0, return_length=True).mean() - 1.0
    na = tree.query_ball_point(pos[idx], 4.0, return_length=True).mean() - 1.0
    return float(nr), float(na)


# files holding the evaluation kernels' device code (a committed DRAM capture of one of
# them is only used while these are unchanged)
EVAL_KERNEL_SOURCES = ("sl_common.cuh", "sl_eval2.cuh", "sl_eval2.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_14073_gb300", "csrc")
    for f in EVAL_KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/traffic_<kernel>.txt, if that
    capture was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"traffic_{kernel}.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


DTYPE_MIXED = ("f32 descriptor and backward, network on tensor cores as f16 hi/lo pairs with f32 accumulation, "
               "f64 state and integration")

# Landau onsite coefficients (a, b) per species for --longitudinal runs, eV: minimum at |S|^2 = 1.25
LONG_LANDAU = [[-0.2, 0.08], [-0.2, 0.08]]

NETWORK_BYTES_PER_ATOM = 66 * 4 * 2 + 4    # descriptors in, network gradient out, E_i (FP32)


def kernel_rooflines(fl, prof, steps, n, peak_alu):
    """Fraction of its own roofline for each evaluation kernel: the descriptor and backward
    kernels against the FP32 FMA peak (algorithmic FLOP per atom, flops.py), the tensor-core
    network against the measured HBM bandwidth (its FP32 operands in and gradient out)."""
    out = {}
    for k in ("rad_fwd", "ang_fwd", "backward"):
        ms = prof[k] / steps
        tf = fl[k] * n / (ms * 1e-3) / 1e12
        out[k] = {"bound": "alu", "achieved_tflops": tf, "frac": tf / peak_alu}
    peaks = measured_peaks() or {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ms = prof["network"] / steps
    gbs = NETWORK_BYTES_PER_ATOM * n / (ms * 1e-3) / 1e9
    out["network"] = {"bound": "hbm", "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return None


def oracle_rate(steps: int, warmup: int, cells: int, threads_note=True):
    """Oracle MD steps on a cells^3 sample of the workload recipe; returns (atom-steps/s, atoms, seconds)."""
    from oracle import oracle as O
    from paper_2606_14073_gb300 import nep_params, workloads as W
    p = nep_params.load()
    m = O.Model(p)
    wl = W.fege_cube(cells, T=TEMP, spin_mode="canted", seed=W.STRUCTURE_SEED0 + 2, n_steps=1)
    st = O.State(wl.positions, wl.velocities, wl.spins, wl.species, wl.box, wl.periodic)
    if warmup:
        O.run(m, st, warmup, DT, TEMP, FIELD, seed=wl.seed)
    else:
        O.run(m, st, 0, DT, TEMP, FIELD, seed=wl.seed)   # initial forces outside the timed region
    t0 = time.perf_counter()
    O.run(m, st, steps, DT, TEMP, FIELD, seed=wl.seed)
    dt = time.perf_counter() - t0
    return wl.n * steps / dt, wl.n, dt


def pick_oracle_cells(total_steps: int, budget_s: float):
    """Largest cube whose total_steps oracle steps fit budget_s, from a quick calibration."""
    rate, _, _ = oracle_rate(1, 0, 8)
    atoms = rate * budget_s / max(total_steps, 1)
    cells = int(round((atoms / 8.0) ** (1.0 / 3.0)))
    return max(4, min(48, cells)), rate


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from oracle import oracle as O
    cells, _ = pick_oracle_cells(args.steps + args.warmup, budget_s=args.ref_budget_s)
    rate, atoms, secs = oracle_rate(args.steps, args.warmup, cells)
    cores = O.num_threads()
    sample = (f"{cells}^3 B20 cells = {atoms} atoms of the {WORKLOAD} recipe (same density, spins, 300 K), "
              f"{args.steps} oracle MD steps timed after {args.warmup} warm-up steps")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_atoms": atoms, "dt_fs": DT, "T_K": TEMP},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_e2e(args, sysm, wl, world, barrier, dist, torch, st):
    """The timed steps again through the public API from host buffers: st is the state the
    timed region started from, so the call replays the same trajectory (same work)."""
    host = {k: torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory().numpy()
            for k in ("positions", "velocities", "spins", "forces", "fields", "ref_positions")}
    barrier()
    t0 = time.perf_counter()
    sysm.set_state(host["positions"], host["velocities"], host["spins"], host["forces"], host["fields"], st["step"],
                   ref_positions=host["ref_positions"])
    sysm.step(args.steps, DT, TEMP, FIELD)
    out = sysm.get_state()
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, dist, "cuda")
    h2d = sum(host[k].nbytes for k in host)
    d2h = sum(out[k].nbytes for k in ("positions", "velocities", "spins", "forces", "fields", "ref_positions"))
    e2e = {"value": whole_job_rate(wl.n, args.steps, world, e2e_s * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "path": "sl_set_state(host) + sl_step(K) + sl_get_state(host), wall clock, replaying the timed steps "
                   "from their start state", "_out": out}

    return e2e


def forced_rebuild_ms(sysm, repeats=3):
    """Device time of one neighbour-list rebuild of the system's current state: the state is
    set again with list reference positions 10 A away, so the rebuild group of the next profiled
    step runs; the state is restored afterwards (median of `repeats`)."""
    st = sysm.get_state()
    times = []
    for _ in range(repeats):
        sysm.set_state(st["positions"], st["velocities"], st["spins"], st["forces"], st["fields"], st["step"],
                       ref_positions=st["positions"] + 10.0)
        times.append(sysm.step_profiled(1, DT, TEMP, FIELD)["rebuild"])
    sysm.set_state(st["positions"], st["velocities"], st["spins"], st["forces"], st["fields"], st["step"],
                   ref_positions=st["ref_positions"])
    return float(statistics.median(times))


def run_serving(args, params, replica_offset=0):
    """Sweep requests (B20 replicas of 12^3-40^3 cells, 50-320 K, 0-0.5 T, 200-2000 steps) arriving
    as a Poisson process, served with admission by free device memory and chunked batching."""
    from paper_2606_14073_gb300.serving import GpuBackend, Server, poisson_requests
    reqs = poisson_requests(args.serve_requests, args.serve_rate)
    for r in reqs:
        r.replica += replica_offset
    be = GpuBackend(params)
    out = Server(be, max_active=32, chunk=50, creators=4).run(reqs)
    stats = be.batch_stats()
    be.close()
    return {"requests": out["requests"], "arrival_rate_per_s": args.serve_rate,
            "throughput_atom_steps_per_s": out["throughput_atom_steps_per_s"],
            "latency_p50_s": out["latency_p50_s"], "latency_p99_s": out["latency_p99_s"],
            "makespan_s": out["makespan_s"], "memory_waits": out["memory_waits"], "batch": stats,
            "recipe": "cells U{12..40}, T U(50,320) K, B_z U(0,0.5) T, steps U{200..2000}, mixed precision"}


def run_sweep(args):
    """Coloured Suzuki-Trotter spin sweep on a --cells cube (default 12^3 cells, 13,824 atoms):
    2C + 1 evaluations per step with C ~ 230 colours, so a far smaller system than the
    predictor-corrector benchmark; mixed precision, 300 K."""
    import torch
    from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W
    torch.cuda.set_device(0)
    params = nep_params.load()
    cells = args.cells if args.cells != 48 else 12
    wl = W.fege_cube(cells, T=TEMP, spin_mode="canted", seed=W.STRUCTURE_SEED0 + 2, n_steps=1,
                     name=f"fege_b20_{cells}c")
    s = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED)
    s.set_spin_sweep(True)
    s.step(args.warmup, DT, TEMP, FIELD)
    _, _, ev0 = s.sweep_colours(with_colours=False)
    launches0 = s.info()["n_launches"]
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(args.steps, DT, TEMP, FIELD)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    _, nc, ev1 = s.sweep_colours(with_colours=False)
    launches = s.info()["n_launches"] - launches0
    s.destroy()
    value = wl.n * args.steps / secs
    line = _common_line(args, value, 1e3 * secs, args.steps, wl.name,
                        {"atoms": wl.n, "precision": "mixed", "dt_fs": DT, "T_K": TEMP, "B_T": list(FIELD),
                         "spin_update": "coloured Suzuki-Trotter sweep", "l2": "working set in L2 (small system)",
                         "parallelism": "replicas x1"},
                        clk, launches,
                        {"mode": "sweep", "colours_last_step": nc,
                         "evaluations_per_step": (ev1 - ev0) / args.steps,
                         "timing": "wall clock around sl_step (the sweep is driven from the host)"})
    print(json.dumps(line), flush=True)
    return 0


def _common_line(args, value, ms_total, steps, workload, config, clk, launches, extra):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms_total / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_MIXED,
            "data": "synthetic (seeded FeGe B20, random-init NEP of the paper's shape)",
            "config": dict(workload=workload, **config), "clocks": clk, "gpu_launches": launches}
    line.update(extra)
    return line


def sample_neighbour_stats(pos, box, periodic, sample=20000, seed=0):
    """Mean neighbours inside 6 A and 4 A on a sample of atoms (periodic axes wrapped)."""
    from scipy.spatial import cKDTree
    p = np.array(pos, dtype=np.float64)
    bs = np.array(box, dtype=np.float64)
    per = np.asarray(periodic, dtype=bool)
    for a in range(3):
        if per[a]:
            p[:, a] = np.mod(p[:, a], bs[a])
    # non-periodic axes: a box length larger than any separation disables wrapping there
    span = np.where(per, bs, (p.max(axis=0) - p.min(axis=0)) + 100.0)
    p = p - np.where(per, 0.0, p.min(axis=0) - 1.0)
    tree = cKDTree(p, boxsize=span)
    idx = np.random.default_rng(seed).choice(len(p), min(sample, len(p)), replace=False)
    nr = tree.query_ball_point(p[idx], 6.0, return_length=True).mean() - 1.0
    na = tree.query_ball_point(p[idx], 4.0, return_length=True).mean() - 1.0
    return float(nr), float(na)


def run_slab(args):
    """Slab of 160 x 160 x 16 B20 cells (3,276,800 atoms), periodic in x and y, free z
    surfaces, helix along x, B = 0.2 T along z, temperature ramped linearly from 0 to
    280 K over --ramp-steps steps (piecewise constant per captured graph of
    --graph-steps steps).  The timed region is --steps steps from the start of the ramp."""
    import torch
    from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W
    torch.cuda.set_device(0)
    params = nep_params.load()
    wl = W.fege_slab_helix()
    B = tuple(float(x) for x in wl.B)
    stream = torch.cuda.Stream()
    sysm = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED, stream=stream.cuda_stream,
                                  steps_per_graph=args.graph_steps, cap_rad=args.cap_rad, cap_ang=args.cap_ang)
    nr0, na0 = sample_neighbour_stats(wl.positions, wl.box, wl.periodic)
    T_end, ramp = 280.0, float(args.ramp_steps)
    chunk = args.graph_steps

    def temp(step):
        return T_end * min(step, ramp) / ramp

    sysm.step(args.warmup, DT, 0.0, B)        # warm-up (graph capture) before the ramp
    info0 = sysm.info()
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    windows = []
    w0 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    w0.record(stream)
    done, win = 0, 2000
    stopped = None
    while done < args.steps:
        k = min(chunk, args.steps - done)
        try:
            sysm.step(k, DT, temp(done), B)
        except S.SpinlatError as e:   # the library restored the state at the start of the call
            stopped = {"at_step": done, "error": str(e)}
            break
        done += k
        if done % win == 0 or done == args.steps:
            w1 = torch.cuda.Event(enable_timing=True)
            w1.record(stream)
            windows.append((done, w0, w1))
            w0 = w1
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    info1 = sysm.info()
    st = sysm.get_state()
    nr1, na1 = sample_neighbour_stats(st["positions"], wl.box, wl.periodic)
    z = st["positions"][:, 2]
    z_lo, z_hi = float(wl.positions[:, 2].min()), float(wl.positions[:, 2].max())
    left = int(((z < z_lo - 5.0) | (z > z_hi + 5.0)).sum())
    win_rates = [{"end_step": d, "T_K": temp(d), "atom_steps_per_s": wl.n * win / (a.elapsed_time(b) * 1e-3)}
                 for d, a, b in windows if d % win == 0]
    sysm.destroy()
    steps_run = max(done, 1)
    line = _common_line(args, wl.n * steps_run / (ms * 1e-3), ms, steps_run, wl.name,
                        {"atoms": wl.n, "precision": "mixed", "dt_fs": DT, "T_K": f"0 -> 280 over {args.ramp_steps} steps",
                         "B_T": list(B), "periodic": [1, 1, 0], "helix_period_A": float(wl.box[0] / round(wl.box[0] / 700.0)),
                         "steps_per_graph": chunk, "l2": "inputs larger than L2 (~37 GB working set)",
                         "parallelism": "replicas x1"},
                        clk, info1["n_launches"] - info0["n_launches"],
                        {"mode": "slab", "steps_requested": args.steps, "stopped": stopped,
                         "caps": [args.cap_rad, args.cap_ang],
                         "neighbour_builds": info1["n_builds"] - info0["n_builds"],
                         "windows_2000_steps": win_rates,
                         "drift": {"mean_neighbours_6A": [nr0, nr1], "mean_neighbours_4A": [na0, na1],
                                   "atoms_beyond_surfaces_5A": left}})
    print(json.dumps(line), flush=True)
    return 0


def run_replicas(args):
    """64 replicas of uneven size (atoms log-uniform in [4096, 262144], cells per side
    clamp(round((N/8)^(1/3)), 8, 32)), T ~ U(100, 300) K, B_z ~ U(0, 0.5) T, --steps steps
    each in one batched call; mixed timed, FP64 timed over --fp64-steps, and the mixed
    force/field error against FP64 on every replica's initial state."""
    import torch
    from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W
    torch.cuda.set_device(0)
    params = nep_params.load()
    cells, Ts, Bz = W.replica_sizes(64)
    wls = [W.fege_cube(int(c), T=float(t), spin_mode="canted", seed=W.STRUCTURE_SEED0 + 4 + 1000 * (k + 1),
                       n_steps=args.steps, name=f"replica{k}", replica=k) for k, (c, t) in enumerate(zip(cells, Ts))]
    Bs = [(0.0, 0.0, float(b)) for b in Bz]
    atoms = int(sum(w.n for w in wls))
    # error of the mixed form against FP64, replica by replica on the initial states
    se_f = se_h = 0.0
    for k, w in enumerate(wls):
        a = S.system_from_workload(w, params, precision=S.SL_PREC_MIXED, replica=k)
        b = S.system_from_workload(w, params, precision=S.SL_PREC_FP64, replica=k)
        ra, rb = a.energy_forces_fields(want_virial=False), b.energy_forces_fields(want_virial=False)
        se_f += float(((ra["F"] - rb["F"]) ** 2).sum())
        se_h += float(((ra["H"] - rb["H"]) ** 2).sum())
        a.destroy()
        b.destroy()
    err = {"force_rmse_eV_per_A": (se_f / (3 * atoms)) ** 0.5, "field_rmse_eV": (se_h / (3 * atoms)) ** 0.5}

    def timed(prec, steps):
        syss = [S.system_from_workload(w, params, precision=prec, replica=k, steps_per_graph=args.graph_steps)
                for k, w in enumerate(wls)]
        bt = S.Batch(syss)
        bt.step(args.warmup, DT, Ts, Bs)
        st0 = bt.stats()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        t0 = time.perf_counter()
        bt.step(steps, DT, Ts, Bs)     # returns after every replica's stream is done
        secs = time.perf_counter() - t0
        clk = clocks.stop()
        st1 = bt.stats()
        bt.destroy()
        for s in syss:
            s.destroy()
        return atoms * steps / secs, secs, clk, st1["kernel_launches"] - st0["kernel_launches"], \
            {k: st1[k] - st0[k] for k in st1}

    def single(steps):
        """One 884,736-atom cube (48^3 cells), timed the same way (host-synchronous call)."""
        w = W.fege_884k()
        s = S.system_from_workload(w, params, precision=S.SL_PREC_MIXED, steps_per_graph=args.graph_steps)
        s.step(args.warmup, DT, 300.0, (0, 0, 0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps, DT, 300.0, (0, 0, 0))
        secs = time.perf_counter() - t0
        s.destroy()
        return w.n * steps / secs

    v64, s64, _, _, _ = timed(S.SL_PREC_FP64, args.fp64_steps)
    value, secs, clk, launches, bstats = timed(S.SL_PREC_MIXED, args.steps)
    v1 = single(args.steps)
    line = _common_line(args, value, secs * 1e3, args.steps, "fege_b20_64_replicas_4096_262144",
                        {"atoms": atoms, "replicas": 64, "precision": "mixed", "dt_fs": DT,
                         "T_K": "U(100,300) per replica", "B_T": "z, U(0,0.5) per replica",
                         "steps_per_graph": args.graph_steps, "l2": "inputs larger than L2 (~45 GB working set)",
                         "parallelism": "replicas x1 GPU, one batched call"},
                        clk, launches,
                        {"mode": "replicas", "timing": "wall clock around one sl_batch_step (host-synchronous)",
                         "batch": bstats,
                         "single_system": {"value": v1, "unit": UNIT, "atoms": 884736,
                                           "timing": "wall clock around one sl_step of the same steps"},
                         "vs_single_system": value / v1,
                         "fp64": {"value": v64, "unit": UNIT, "steps": args.fp64_steps},
                         "mixed_error_vs_fp64": err,
                         "replica_atoms": [int(w.n) for w in wls]})
    print(json.dumps(line), flush=True)
    return 0


def run_serve_sweep(args):
    """Serving: Poisson arrivals at 0.25, 0.5, 1, 2 and 4 x the saturation request rate
    (measured first from a burst of the same requests).  Requests: cells per side
    U{12..40}, T U[50,320] K, B_z U[0,0.5] T, steps U{200..2000}; --serve-requests each."""
    import torch
    from paper_2606_14073_gb300 import nep_params
    from paper_2606_14073_gb300.serving import GpuBackend, Server, poisson_requests
    torch.cuda.set_device(0)
    params = nep_params.load()
    be = GpuBackend(params)
    burst = poisson_requests(args.serve_requests, 0.0)
    out = Server(be, max_active=32, chunk=50, creators=4).run(burst)
    work = np.mean([8 * r.cells ** 3 * r.n_steps for r in burst])
    sat_rate = out["throughput_atom_steps_per_s"] / work
    rows = [{"rate_multiple": "burst", "arrival_rate_per_s": None,
             **{k: out[k] for k in ("throughput_atom_steps_per_s", "latency_p50_s", "latency_p99_s", "makespan_s",
                                    "memory_waits", "requests", "chunks", "chunk_seconds",
                                    "chunk_atom_steps_per_s")}}]
    for m in [float(x) for x in args.serve_rates.split(",") if x.strip()]:
        reqs = poisson_requests(args.serve_requests, m * sat_rate, seed=20260105 + int(100 * m))
        o = Server(be, max_active=32, chunk=50, creators=4).run(reqs)
        rows.append({"rate_multiple": m, "arrival_rate_per_s": m * sat_rate,
                     **{k: o[k] for k in ("throughput_atom_steps_per_s", "latency_p50_s", "latency_p99_s",
                                          "makespan_s", "memory_waits", "requests", "chunks", "chunk_seconds",
                                          "chunk_atom_steps_per_s")}})
    peak = max(r["throughput_atom_steps_per_s"] for r in rows)
    line = _common_line(args, peak, 0.0, 1, "fege_serving_sweep",
                        {"requests_per_rate": args.serve_requests, "precision": "mixed",
                         "recipe": "cells U{12..40}, T U[50,320] K, B_z U[0,0.5] T, steps U{200..2000}",
                         "l2": "inputs larger than L2", "parallelism": "replicas x1"},
                        None, None,
                        {"mode": "serve-sweep", "saturation_rate_per_s": sat_rate,
                         "mean_atom_steps_per_request": work, "rates": rows})
    line["ms_per_step"] = None
    print(json.dumps(line), flush=True)
    return 0


def run_protocol(args):
    """Production protocol of the paper's texture study (Fig. 7): a thin stripe
    (512 x 96 x 4 B20 cells = 1,572,864 atoms, periodic in x and y, free z surfaces, 1.9 nm
    thick) from random spins at 160 K, with B_z stepping along x through 0, 0.05, 0.1 and
    0.15 T (per-atom field); --steps steps, texture diagnostics (film magnetisation map,
    Berg-Luescher topological charge, mean m_z per field segment) every --diag-every
    steps on the device.  The timed region includes the diagnostics."""
    import torch
    from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W
    torch.cuda.set_device(0)
    params = nep_params.load()
    wl = W.fege_slab_helix(512, 96, 4, seed=W.STRUCTURE_SEED0 + 5, T=160.0)
    spins = W.random_unit_vectors(np.random.Generator(np.random.PCG64(W.STRUCTURE_SEED0 + 6)), wl.n)
    values = (0.0, 0.05, 0.1, 0.15)
    seg = np.clip((wl.positions[:, 0] / wl.box[0] * len(values)).astype(int), 0, len(values) - 1)
    Ba = np.zeros((wl.n, 3))
    Ba[:, 2] = np.asarray(values)[seg]
    stream = torch.cuda.Stream()
    sysm = S.System(wl.positions, spins, wl.box, wl.periodic, wl.species, params, wl.velocities,
                    precision=S.SL_PREC_MIXED, seed=wl.seed, stream=stream.cuda_stream,
                    steps_per_graph=args.graph_steps)
    sysm.set_atom_fields(Ba)
    T, B = 160.0, (0.0, 0.0, 0.0)
    sysm.step(args.warmup, DT, T, B)
    info0 = sysm.info()
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    diag, diag_ms = [], 0.0
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        k = min(args.diag_every, args.steps - done)
        sysm.step(k, DT, T, B)
        done += k
        d0 = time.perf_counter()
        m, q = sysm.texture(2, 4.70)
        na = m.shape[1]
        mz = [float(m[:, int(na * a / 4):int(na * (a + 1) / 4), 2].mean()) for a in range(4)]
        diag_ms += (time.perf_counter() - d0) * 1e3
        diag.append({"step": done, "Q": q, "mean_mz_by_segment": mz})
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    info1 = sysm.info()
    sysm.destroy()
    line = _common_line(args, wl.n * args.steps / secs, secs * 1e3, args.steps, "fege_stripe_512x96x4_field_steps",
                        {"atoms": wl.n, "precision": "mixed", "dt_fs": DT, "T_K": T,
                         "B_T": "z: 0, 0.05, 0.1, 0.15 in four x segments (per-atom field)",
                         "periodic": [1, 1, 0], "start": "random spins", "steps_per_graph": args.graph_steps,
                         "l2": "inputs larger than L2 (~18 GB working set)", "parallelism": "replicas x1"},
                        clk, info1["n_launches"] - info0["n_launches"],
                        {"mode": "protocol", "timing": "wall clock, diagnostics included",
                         "diagnostics_ms_total": diag_ms, "texture_grid_cells": "4.70 A in x and y",
                         "diagnostics": diag, "neighbour_builds": info1["n_builds"] - info0["n_builds"]})
    print(json.dumps(line), flush=True)
    return 0


def run_accuracy(args):
    """Mixed-precision error on identical states along an FP64 trajectory of the 884,736-atom
    workload: the FP64 system runs --fp64-steps steps (default here 1000) at 300 K; at
    steps 0, half and the end its state is copied into a mixed-precision system
    (sl_set_state) and forces and fields are compared over all atoms; the FP64 GPU values
    are checked against the FP64 oracle on a seeded 1% sample (8,847 atoms)."""
    import torch
    from oracle import oracle as O
    from paper_2606_14073_gb300 import nep_params, spinlat as S, workloads as W
    torch.cuda.set_device(0)
    params = nep_params.load()
    model = O.Model(params)
    wl = W.fege_884k()
    total = args.fp64_steps
    checkpoints = [0, total // 2, total]
    sample = np.sort(np.random.default_rng(20260103).choice(wl.n, wl.n // 100, replace=False))
    sysd = S.system_from_workload(wl, params, precision=S.SL_PREC_FP64, steps_per_graph=args.graph_steps)
    sysm = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED, steps_per_graph=args.graph_steps)
    rows, done = [], 0
    t0 = time.perf_counter()
    for c in checkpoints:
        if c > done:
            sysd.step(c - done, DT, TEMP, FIELD)
            done = c
        st = sysd.get_state()
        sysm.set_state(st["positions"], st["velocities"], st["spins"], st["forces"], st["fields"], st["step"],
                       ref_positions=st["ref_positions"])
        rd = sysd.energy_forces_fields(want_virial=False)
        rm = sysm.energy_forces_fields(want_virial=False)
        ref = O.evaluate_subset(model, st["positions"], st["spins"], wl.species, wl.box, wl.periodic, sample, FIELD)
        rows.append({"step": c,
                     "mixed_force_rmse_eV_per_A": float(np.sqrt(((rm["F"] - rd["F"]) ** 2).mean())),
                     "mixed_field_rmse_eV": float(np.sqrt(((rm["H"] - rd["H"]) ** 2).mean())),
                     "mixed_energy_err_eV_per_atom": abs(rm["E"] - rd["E"]) / wl.n,
                     "fp64_vs_oracle_sample_max_rel_F": float(np.abs(rd["F"][sample] - ref["F"]).max() /
                                                              np.abs(ref["F"]).max()),
                     "fp64_vs_oracle_sample_max_rel_H": float(np.abs(rd["H"][sample] - ref["H"]).max() /
                                                              np.abs(ref["H"]).max()),
                     "force_rms_eV_per_A": float(np.sqrt((rd["F"] ** 2).mean()))})
    secs = time.perf_counter() - t0
    sysd.destroy()
    sysm.destroy()
    line = _common_line(args, wl.n * total / secs, secs * 1e3, max(total, 1), WORKLOAD,
                        {"atoms": wl.n, "precision": "FP64 trajectory, mixed evaluated on its states", "dt_fs": DT,
                         "T_K": TEMP, "sample_atoms": int(len(sample)), "l2": "inputs larger than L2",
                         "parallelism": "replicas x1"},
                        None, None,
                        {"mode": "accuracy", "timing": "wall clock of the whole check (FP64 steps, evaluations, "
                                                       "oracle on the sample)", "states": rows})
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2606_14073_gb300 import flops, nep_params, spinlat as S, workloads as W

    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    params = nep_params.load()
    wl = W.fege_884k() if args.cells == 48 else W.fege_cube(args.cells, T=TEMP, spin_mode="canted",
                                                            seed=W.STRUCTURE_SEED0 + 2, n_steps=1,
                                                            name=f"fege_b20_{args.cells}c")
    replica = rank
    stream = torch.cuda.Stream(device=local)
    mid = dict(midpoint_iters=args.midpoint_iters, midpoint_tol=args.midpoint_tol,
               anderson_depth=args.anderson_depth)
    sysm = S.system_from_workload(wl, params, precision=S.SL_PREC_MIXED, replica=replica, stream=stream.cuda_stream,
                                  device=local, steps_per_graph=args.graph_steps, **mid)
    if args.longitudinal > 0:
        sysm.set_longitudinal(True, args.longitudinal, LONG_LANDAU)

    def barrier():
        if dist is not None:
            dist.barrier()

    # force/field error of the mixed form against the FP64 GPU path on the same state
    err = None
    fp64 = None
    if not args.skip_fp64:
        sysd = S.system_from_workload(wl, params, precision=S.SL_PREC_FP64, replica=replica, device=local,
                                      stream=stream.cuda_stream, steps_per_graph=args.graph_steps, **mid)
        if args.longitudinal > 0:
            sysd.set_longitudinal(True, args.longitudinal, LONG_LANDAU)
        rm = sysm.energy_forces_fields(want_virial=False)
        rd = sysd.energy_forces_fields(want_virial=False)
        err = {"reference": "FP64 GPU path (itself within 1e-10 of the FP64 oracle)",
               "force_rmse_eV_per_A": float(np.sqrt(((rm["F"] - rd["F"]) ** 2).mean())),
               "field_rmse_eV": float(np.sqrt(((rm["H"] - rd["H"]) ** 2).mean())),
               "energy_abs_err_eV_per_atom": abs(rm["E"] - rd["E"]) / wl.n,
               "force_rms_eV_per_A": float(np.sqrt((rd["F"] ** 2).mean()))}
        sysd.step(1, DT, TEMP, FIELD)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sysd.step(args.fp64_steps, DT, TEMP, FIELD)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        fp64 = {"value": wl.n * args.fp64_steps / (ms * 1e-3), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": ms / args.fp64_steps}
        sysd.destroy()
        del sysd

    # launch shapes of the evaluation kernels picked by the library's autotuner
    tuned = None
    if not args.no_autotune:
        tuned = sysm.autotune(repeats=5)
        tuned["config"] = sysm.launch_config()

    # warm-up (graph capture happens here)
    sysm.step(args.warmup, DT, TEMP, FIELD)
    start_state = None if args.skip_e2e else sysm.get_state()   # replayed by the end-to-end leg
    info0 = sysm.info()
    launches0 = info0["n_launches"]
    mid0 = sysm.midpoint_evaluations()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sysm.step(args.steps, DT, TEMP, FIELD)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    info1 = sysm.info()
    launches = info1["n_launches"] - launches0
    builds_timed = info1["n_builds"] - info0["n_builds"]
    mid_evals = sysm.midpoint_evaluations() - mid0
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(wl.n, args.steps, world, ms_max)
    end_state = None if args.skip_e2e else sysm.get_state()

    # per-kernel device times (CUDA events between the kernel groups, same stream, no graphs)
    b0 = sysm.info()["n_builds"]
    # the algorithmic work of the profiled steps counts the neighbours of the state they start from
    # (the random-init potential densifies the crystal as the run goes on)
    n_r, n_a = neighbour_counts(wl, sysm.get_state()["positions"])
    prof = sysm.step_profiled(args.profile_steps, DT, TEMP, FIELD)
    builds_prof = sysm.info()["n_builds"] - b0
    # the profiled window holds whole builds; charge them at the timed region's build rate
    per_step = {k: v / args.profile_steps for k, v in prof.items()}
    ms_per_build = (prof["rebuild"] / builds_prof) if builds_prof else None
    if ms_per_build is not None:
        per_step["rebuild"] = ms_per_build * builds_timed / args.steps
    total = sum(per_step.values())
    fl = flops.per_atom(n_r, n_a)
    dom = max(("rad_fwd", "ang_fwd", "network", "backward"), key=lambda k: prof[k])
    launch_ms = prof[dom] / args.profile_steps
    achieved = fl[dom] * wl.n / (launch_ms * 1e-3) / 1e12
    peak_derived, n_sms, peak_mhz = fp32_peak_tflops(local, (clk or {}).get("sm_max_mhz"))
    fma32, _ = S.sl_measure_fma_peak(S.SL_PREC_MIXED)
    fma64, _ = S.sl_measure_fma_peak(S.SL_PREC_FP64)
    roofline = {"bound": "alu", "kernel": {"rad_fwd": "k_crad<float>", "ang_fwd": "k_ang_fwd<float>",
                                           "network": "k_mlp_tc", "backward": "k_bwd<float>"}[dom],
                "achieved": achieved, "peak": peak_derived, "unit": "TFLOP/s", "frac": achieved / peak_derived,
                "peak_source": (f"derived: {n_sms} SMs (device attribute) x 128 FP32 lanes x 2 FLOP x {peak_mhz:.0f} MHz "
                                f"(maximum SM clock), FP32 FMA pipe; the FMA microbenchmark measured "
                                f"{fma32 / 1e12:.1f} TFLOP/s"),
                "peak_measured_fp32_fma_tflops": fma32 / 1e12, "peak_measured_fp64_fma_tflops": fma64 / 1e12,
                "algorithmic_flop_per_atom": fl[dom], "mean_neighbours_6A": n_r, "mean_neighbours_4A": n_a,
                "neighbours_counted_at": "the state the profiled steps start from",
                "launch_ms": launch_ms, "traffic": committed_traffic(dom)}
    shares = {k: v / total for k, v in per_step.items()}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.skip_e2e:
        e2e = run_e2e(args, sysm, wl, world, barrier, dist, torch, start_state)
        out = e2e.pop("_out")
        e2e["replay_bit_identical"] = bool(all(np.array_equal(out[k], end_state[k])
                                               for k in ("positions", "velocities", "spins")))

    # steady state: a longer window at the run's own pace, neighbour-list rebuilds included (the
    # K-step window above is short enough to hold none); then the cost of one forced rebuild
    steady = None
    if args.steady_steps > 0:
        info_s0 = sysm.info()
        clocks_s = ClockSampler(local)
        clocks_s.start()
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        sysm.step(args.steady_steps, DT, TEMP, FIELD)
        e1.record(stream)
        e1.synchronize()
        ms_s = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        clk_s = clocks_s.stop()
        builds_s = sysm.info()["n_builds"] - info_s0["n_builds"]
        build_ms = forced_rebuild_ms(sysm)
        steady = {"value": whole_job_rate(wl.n, args.steady_steps, world, ms_s), "unit": UNIT,
                  "steps": args.steady_steps, "ms_per_step": ms_s / args.steady_steps,
                  "neighbour_builds": builds_s, "ms_per_build": build_ms,
                  "rebuild_share": (builds_s * build_ms / ms_s) if build_ms is not None else None,
                  "clocks": clk_s,
                  "window": "the steps after the timed K steps and their end-to-end replay, graphs of "
                            f"{args.graph_steps} steps, the rebuild check on the device every step"}

    # continuous-batching serving run: Poisson sweep requests, p50/p99 time to completion
    serving = None
    if not args.skip_serving:
        serving = run_serving(args, params, replica_offset=1000 * rank)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        from oracle import oracle as O
        cells, _ = pick_oracle_cells(2, budget_s=20.0)
        rate, atoms, secs = oracle_rate(2, 0, cells)
        cores = O.num_threads()
        # the same oracle on one core, over a smaller block of the same recipe
        O.set_num_threads(1)
        rate1, atoms1, secs1 = oracle_rate(2, 0, 10)
        O.set_num_threads(cores)
        rate_c1, atoms_c1, secs_c1 = oracle_rate(100, 0, 4)   # the 512-atom system in full
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"2 oracle MD steps of a {cells}^3-cell ({atoms}-atom) block of the same recipe, {secs:.1f} s",
               "single_core": {"value": rate1, "unit": UNIT,
                               "sample": f"2 oracle MD steps of a 10^3-cell ({atoms1}-atom) block, {secs1:.1f} s"},
               "small_system": {"value": rate_c1, "unit": UNIT, "cores": cores,
                                "sample": f"100 oracle MD steps of the {atoms_c1}-atom 4^3-cell system, {secs_c1:.1f} s"}}

    sysm.destroy()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE_MIXED,
                "data": "synthetic (seeded FeGe B20, random-init NEP of the paper's shape)",
                "config": {"workload": WORKLOAD if args.cells == 48 else wl.name, "atoms": wl.n, "precision": "mixed", "dt_fs": DT, "T_K": TEMP,
                           "B_T": list(FIELD), "steps_per_graph": args.graph_steps,
                           "spin_update": (f"longitudinal moments, alpha {args.longitudinal}, Landau (a, b) "
                                           f"{LONG_LANDAU} eV" if args.longitudinal > 0 else
                                           "predictor-corrector" if args.midpoint_iters == 0 else
                                           f"self-consistent midpoint, cap {args.midpoint_iters}, tol "
                                           f"{args.midpoint_tol}, Anderson depth {args.anderson_depth}"),
                           "l2": "inputs larger than L2 (~10 GB working set)", "parallelism": f"replicas x{world}"},
                "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "neighbour_builds": {"timed_region": builds_timed, "profiled_steps": builds_prof,
                                     "ms_per_build": (steady or {}).get("ms_per_build", ms_per_build)},
                "steady_state": steady,
                "kernel_share": shares, "kernel_ms_per_step": per_step,
                "kernel_roofline": kernel_rooflines(fl, prof, args.profile_steps, wl.n, peak_derived),
                "fp64": fp64, "mixed_error_vs_fp64": err, "serving": serving, "cpu_baseline": cpu,
                "autotune": tuned}
        if args.midpoint_iters > 0:
            line["midpoint_evaluations_per_step"] = mid_evals / args.steps
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--graph-steps", type=int, default=10)
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--steady-steps", type=int, default=200,
                    help="cube: steps of the steady-state window with list rebuilds (0: skip)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=8.0, help="request arrivals per second")
    ap.add_argument("--serve-rates", default="0.25,0.5,1,2,4",
                    help="serve-sweep: arrival rates as multiples of the saturation rate (after the burst)")
    ap.add_argument("--workload", choices=["cube", "slab", "replicas", "serve-sweep", "protocol", "accuracy",
                                           "sweep"],
                    default="cube",
                    help="cube: the 884,736-atom benchmark (default); slab: 3,276,800-atom helix slab with a "
                         "temperature ramp; replicas: 64 uneven replicas in one batched call; serve-sweep: "
                         "Poisson serving at multiples of the saturation rate; protocol: 1.57M-atom stripe at "
                         "160 K in a stepped field with on-device texture diagnostics; accuracy: mixed vs FP64 "
                         "on identical states at steps 0, half and the end of an FP64 trajectory (--fp64-steps); "
                         "sweep: the coloured Suzuki-Trotter spin update on a 12^3-cell cube")
    ap.add_argument("--diag-every", type=int, default=500, help="protocol: steps between texture diagnostics")
    ap.add_argument("--ramp-steps", type=int, default=20000, help="slab: length of the 0 -> 280 K ramp")
    ap.add_argument("--cap-rad", type=int, default=160, help="slab: radial candidate-list capacity")
    ap.add_argument("--cap-ang", type=int, default=64, help="slab: angular candidate-list capacity")
    ap.add_argument("--midpoint-iters", type=int, default=0,
                    help="cube: cap of the self-consistent midpoint spin update (0: predictor-corrector)")
    ap.add_argument("--midpoint-tol", type=float, default=1e-6)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--anderson-depth", type=int, default=0)
    ap.add_argument("--ref-budget-s", type=float, default=150.0,
                    help="reference arm: seconds of oracle work the sample is sized for")
    ap.add_argument("--longitudinal", type=float, default=0.0,
                    help="cube: damping alpha of the longitudinal moment mode (0: unit spins)")
    ap.add_argument("--cells", type=int, default=48, help="B20 cells per side (48: the benchmark workload; "
                                                           "smaller values are for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "slab":
        return run_slab(args)
    if args.workload == "replicas":
        return run_replicas(args)
    if args.workload == "serve-sweep":
        return run_serve_sweep(args)
    if args.workload == "protocol":
        return run_protocol(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "accuracy":
        return run_accuracy(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
