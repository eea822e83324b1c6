#!/usr/bin/env python3
"""Throughput of the coupled diffuse-interface MRT lattice Boltzmann step.

One bench step is one coupled time step (phase field, solute, heat and flow,
plus the wall kernels) over the whole grid of the multi-seed thermosolutal
workload: 4096 x 4096 nodes, 64 seeds (dart throwing, spacing >= 200, radii
6-10, orientations in [0, 45 deg), RNG seed 3), Delta = 0.45, eps = 0.04,
periodic in x, no-slip walls in y, buoyancy on, FP32 populations.  The state
(about 4 GB) is far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-LB MLUPS and % of HBM roofline; surrogate speedup at matched tip error"
UNIT = "MLUPS"
# Algorithmic HBM bytes per node per coupled step (n_sub = 1): every population
# read once and written once, the six FP32 history scalars read and written,
# and the one-byte grain id read when the domain holds several grains.
# Population bytes per node: FP32 24 x 4 = 96; 16-bit storage 21 x 2 + 3 x 4
# (the scalar rest populations stay FP32) = 54.
POP_BYTES = {"fp32": 96, "fp16": 54, "bf16": 54}
HIST_PLANES = 6


def algorithmic_bytes_per_node(storage: str, grains: bool) -> int:
    return POP_BYTES[storage] * 2 + HIST_PLANES * 2 * 4 + (1 if grains else 0)


def parse():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--n", type=int, default=4096, help="grid side (default: the 4096^2 workload)")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16/BF16 storage lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 256-domain leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate leg")
    ap.add_argument("--no-substeps", action="store_true", help="skip the n_sub = 15 flow-sub-step leg")
    ap.add_argument("--substep-n", type=int, default=1024,
                    help="grid side of the n_sub = 15 leg (default: the paper's 1024^2 flow configuration)")
    ap.add_argument("--surrogate-train-steps", type=int, default=1500)
    ap.add_argument("--surrogate-windows", type=int, default=400)
    ap.add_argument("--reference-seconds", type=float, default=90.0,
                    help="wall-clock target of the --impl reference run (sizes its oracle window)")
    return ap.parse_args()


# ------------------------------------------------------------ ranks (N > 1)
# One process per GPU, each stepping its own replica of the workload: the
# ranks exchange nothing on the data path, only the timing (a barrier on both
# sides of the timed region and the maximum time over ranks).
def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    """Maximum of x over the ranks (all-reduce of one FP64 value on `device`)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, nodes_per_rank: int, steps: int, ms: float) -> float:
    """Lattice updates of all ranks per second (millions): every rank steps
    its own replica of `nodes_per_rank` nodes, in `ms` (the slowest rank)."""
    return world * nodes_per_rank * steps / (ms / 1e3) / 1e6


def workload(n: int):
    from paper_2209_01444_gb300 import workloads as W

    if n == 4096:
        return W.multi_seed()
    count = max(1, (n // 512) ** 2)
    return W.multi_seed(n=n, count=count, min_spacing=min(200.0, n / 4))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C++ source without comments and whitespace (string literals in these
    files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the fused kernel's code: the device header and the part of
    lbm_step.cu up to the end of k_coupled_step (the batched, flow-only and
    wall kernels that follow it do not change its traffic), comments and
    whitespace left out."""
    csrc = os.path.join(ROOT, "paper_2209_01444_gb300", "csrc")
    with open(os.path.join(csrc, "lbm_device.cuh")) as fh:
        head = fh.read()
    with open(os.path.join(csrc, "lbm_step.cu")) as fh:
        text = fh.read()
    cut = text.find("// Descriptors of the batch being stepped")
    body = text if cut < 0 else text[:cut]
    return hashlib.sha256((_code_only(head) + _code_only(body)).encode()).hexdigest()[:16]


def recorded_traffic(key: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "fused_step_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == key and parts[1] == src:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            pass
    return local_rank


ACCURACY_FIELDS = ("phi", "C", "theta", "ux", "uy")


def field_errors(got: dict, ref: dict, theta_scale: float) -> dict:
    """max|X - X_ref| / max(max|X_ref|, floor) per field, the floors of the
    parity tests (phi, C: 1; theta: |theta0|).  Both velocity components are
    measured against the largest speed |u| of the reference (floor 1e-6), the
    scale of the velocity: a cross-stream component that is still tiny next to
    the stream is not measured against its own maximum."""
    floor = {"phi": 1.0, "C": 1.0, "theta": theta_scale}
    out = {k: float(np.abs(got[k] - ref[k]).max() / max(float(np.abs(ref[k]).max()), floor[k]))
           for k in ref if k in floor}
    if "ux" in ref and "uy" in ref:
        speed = max(float(np.hypot(ref["ux"], ref["uy"]).max()), 1e-6)
        for k in ("ux", "uy"):
            out[k] = float(np.abs(got[k] - ref[k]).max() / speed)
    return out


def drift(sim, m_end) -> dict:
    """Relative change of the solute and enthalpy sums over the run (the
    walls of the workload are closed to both)."""
    c0, h0 = sim.sums0
    return {"sum_C_rel_drift": (m_end["sum_C"] - c0) / abs(c0), "sum_H_rel_drift": (m_end["sum_H"] - h0) / abs(h0)}


def cpu_oracle_one_core(case, side: int = 256, target_s: float = 3.0) -> dict:
    """The same oracle on one host thread (a subprocess started with
    OMP_NUM_THREADS=1), on a side x side window for about target_s seconds."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import bench
from oracle import oracle as O
case = bench.workload({case.params["nx"]})
p = dict(case.params); p["nx"] = p["ny"] = {side}; p["bc"] = ("periodic",) * 4
o = O.Oracle(p)
N = case.params["nx"]; x0 = (N - {side}) // 2
o.init_seeds_window(case.seeds, case.U0, case.theta0, x0, x0, N, case.params["ny"], True, False)
t = time.perf_counter(); o.step(2); per = (time.perf_counter() - t) / 2
n = int(max(3, min(400, {target_s} / max(per, 1e-6))))
t = time.perf_counter(); o.step(n); dt = time.perf_counter() - t
print(json.dumps({{"n": n, "dt": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": side * side * d["n"] / d["dt"] / 1e6, "unit": UNIT, "cores": 1,
            "sample": f"{side}x{side} window, {d['n']} coupled steps, FP64, {d['dt']:.1f} s"}


def cpu_oracle_batch_domain(small: dict) -> tuple[dict, dict]:
    """The FP64 oracle on the batched sweep's smallest domain for the steps
    the batched FP16 run took: its throughput on the host cores, and the
    batched run's field errors against it (the parity metric)."""
    from oracle import oracle as O

    c = small["case"]
    o = O.Oracle(c.params)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    t = time.perf_counter()
    o.step(small["steps"])
    dt = time.perf_counter() - t
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nx, ny = c.params["nx"], c.params["ny"]
    timing = {"value": nx * ny * small["steps"] / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
              "sample": f"domain {small['domain']} ({nx}x{ny}) of the batched sweep, {small['steps']} coupled "
                        f"steps, FP64, {dt:.1f} s"}
    errs = field_errors(small["fields"], o.fields(), abs(c.theta0))
    return timing, {"domain": small["domain"], "nx": nx, "ny": ny, "steps": small["steps"], "errors": errs}


def cpu_oracle_sample(case, target_s: float = 15.0, side: int = 1024, max_steps: int = 400):
    """The FP64 oracle on a side x side window of the workload (seeded in the
    coordinates of the full grid), run for about target_s seconds."""
    from oracle import oracle as O

    p = dict(case.params)
    p["nx"] = p["ny"] = side
    p["bc"] = ("periodic",) * 4
    o = O.Oracle(p)
    N = case.params["nx"]
    x0 = y0 = (N - side) // 2
    o.init_seeds_window(case.seeds, case.U0, case.theta0, x0, y0, N, case.params["ny"], True, False)
    t = time.perf_counter()
    o.step(2)
    per = (time.perf_counter() - t) / 2
    n = int(max(3, min(max_steps, target_s / max(per, 1e-6))))
    t = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": side * side * n / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{side}x{side} window at ({x0},{y0}) of the {N}x{N} workload, {n} coupled steps, "
                      f"FP64, {dt:.1f} s"}


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores: each step is one coupled
    step of a square window of the workload, the window sized so that the
    whole --warmup + --steps run takes about 90 s."""
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    case = workload(args.n)
    from oracle import oracle as O

    def window(side):
        p = dict(case.params)
        p["nx"] = p["ny"] = side
        p["bc"] = ("periodic",) * 4
        o = O.Oracle(p)
        x0 = (args.n - side) // 2
        o.init_seeds_window(case.seeds, case.U0, case.theta0, x0, x0, args.n, args.n, True, False)
        return o

    probe = window(256)
    t = time.perf_counter()
    probe.step(3)
    rate = 256 * 256 * 3 / (time.perf_counter() - t)
    del probe
    total = max(args.steps + args.warmup, 1)
    side = int((args.reference_seconds * rate / total) ** 0.5) // 64 * 64
    side = max(64, min(1024, args.n, side))
    o = window(side)
    o.step(max(args.warmup, 0))
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    value = side * side * args.steps / dt / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{side}x{side} window of the {args.n}x{args.n} workload per step, FP64 oracle"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"multi_seed_thermosolutal_{args.n}x{args.n}", "nodes": side * side,
                   "sample_window": side},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def substep_leg(lbm, torch, stream, max_over_ranks, barrier, n: int = 1024, steps: int = 128):
    """The paper's flow configuration with two-time-scaling: the isothermal
    alloy with inflow (1 W0/tau0), outflow and symmetry walls, Pr = 23.1 and
    n_sub = 15 flow sub-steps per coupled step (Secs. 4.2-4.3), one seed, FP32.
    Algorithmic bytes per node and coupled step: the fused step's 240 plus 14
    sub-steps of 72 (nine flow populations read and written)."""
    from paper_2209_01444_gb300 import workloads as W

    p = W.solutal_params(n, flow=True)
    sim = lbm.Simulation(p, "fp32", stream=stream)
    sim.init_seeds(np.array([[0.5 * n, 0.5 * n, 10.0, 0.0]]), -0.55, 0.0)
    sim.step(32)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1)) / steps
    bpn = 240 + 14 * 72
    peak, kind = peaks()
    achieved = bpn * n * n / (ms / 1e3) / 1e9
    bad = sim.metrics(0.5 * n, 0.5 * n, 0.0, check=False)["nonfinite"]
    # the flow sub-step kernel alone, CUDA events around each launch on the stream
    sim.set_profiling(True, "substep")
    sim.step(16)
    sms, slaunches = sim.kernel_time()
    sim.set_profiling(False)
    s_ms = sms / max(slaunches, 1)
    s_bpn = 80  # nine FP32 flow populations read and written, phi^n and the frozen force read
    s_ach = s_bpn * n * n / (s_ms / 1e3) / 1e9
    return {"workload": f"solutal alloy with inflow {n}x{n}, n_sub = 15 (Pr = 23.1), inflow/outflow/symmetry walls",
            "steps": steps, "ms_per_step": ms, "value": n * n / (ms / 1e3) / 1e6, "unit": "MLUPS",
            "bytes_per_node": bpn, "achieved_gbs": achieved, "frac_of_peak": achieved / peak, "peak_kind": kind,
            "roofline": {"bound": "hbm", "kernel": "k_flow_substep", "achieved": s_ach, "peak": peak,
                         "unit": "GB/s", "frac": s_ach / peak, "bytes_per_node": s_bpn, "kernel_ms": s_ms,
                         "launches": slaunches, "peak_kind": kind,
                         "note": ("the flow state of this grid stays in L2 between sub-steps"
                                  if n * n * 80 < 129e6 else "flow state larger than L2")},
            "nonfinite": bad}


def batch_leg(lbm, torch, stream, steps, world, max_over_ranks, barrier):
    """256 independent domains (sides log-uniform in 128..1024, Delta, eps,
    orientation and inflow drawn per domain, RNG seed 4) in one batched
    persistent launch with FP16 storage and an autotuned tile height, against
    the plain FP32 path: the same domains stepped one after another through
    single-domain handles."""
    from paper_2209_01444_gb300 import workloads as W

    cases = W.batch_domains()
    nodes = sum(c.nodes for c in cases)
    b = lbm.Batch([c.params for c in cases], "fp16", stream=stream)
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
    cache = os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300", "batch_tiling.txt")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    ty = b.tune(cache)
    tiles_per_cta = b.tiles_per_cta
    b.step(16)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(16, steps // 4)
    e0.record(stream)
    b.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = world * nodes * k / (ms / 1e3) / 1e6
    # the batched kernel alone: CUDA events around each launch (direct launches)
    b.set_profiling(True)
    b.step(8)
    bkms, blaunch = b.kernel_time()
    b.set_profiling(False)
    b_ms = bkms / max(blaunch, 1)
    # per node: 16-bit populations and FP32 history read and written; each
    # domain holds one grain, so no grain map is read
    b_bpn = algorithmic_bytes_per_node("fp16", False)
    peak, kind = peaks()
    b_ach = b_bpn * nodes / (b_ms / 1e3) / 1e9
    bad = sum(b.metrics(j, *c.seeds[0][:2], c.seeds[0][3])["nonfinite"] for j, c in enumerate(cases[:8]))
    # accuracy of the batched FP16 run: its first domains against the plain
    # FP32 path after the same 16 + k + 8 steps (the tuner restores the state it times on)
    errs = []
    for j, c in enumerate(cases[:4]):
        ref = lbm.Simulation(c.params, "fp32", stream=stream)
        ref.init_seeds(c.seeds, c.U0, c.theta0)
        ref.step(16 + k + 8)
        errs.append(field_errors(b.fields(j, ACCURACY_FIELDS), ref.fields(ACCURACY_FIELDS), abs(c.theta0)))
        del ref
    worst = {f: max(e[f] for e in errs) for f in errs[0]}
    # the smallest domain's fields, for the CPU baseline leg's FP64 oracle run
    j_small = min(range(len(cases)), key=lambda i: cases[i].nodes)
    small = {"domain": j_small, "case": cases[j_small], "steps": 16 + k + 8,
             "fields": b.fields(j_small, ACCURACY_FIELDS)}
    del b
    # plain FP32 path, one domain after another
    sims = []
    for c in cases:
        s_ = lbm.Simulation(c.params, "fp32", stream=stream)
        s_.init_seeds(c.seeds, c.U0, c.theta0)
        sims.append(s_)
    k2 = 32
    for s_ in sims:
        s_.step(16)
    torch.cuda.synchronize()
    e0.record(stream)
    for s_ in sims:
        s_.step(k2)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = max_over_ranks(e0.elapsed_time(e1))
    seq_value = world * nodes * k2 / (seq_ms / 1e3) / 1e6
    del sims
    return {"workload": "256 domains, sides log-uniform 128..1024 (seed 4), inflow/outflow/symmetry walls",
            "nodes": nodes, "storage": "fp16", "tile_height": ty, "tiles_per_cta": tiles_per_cta, "steps": k,
            "value": value, "unit": UNIT,
            "ms_per_step": ms / k, "sequential_fp32_value": seq_value, "speedup_vs_sequential_fp32": value / seq_value,
            "roofline": {"bound": "hbm", "kernel": "k_batch_step", "achieved": b_ach, "peak": peak, "unit": "GB/s",
                         "frac": b_ach / peak, "bytes_per_node": b_bpn, "kernel_ms": b_ms, "launches": blaunch,
                         "peak_kind": kind},
            "nonfinite_domains_of_first_8": bad, "field_error_vs_fp32_first_4_domains": worst,
            "velocity_error_scale": "largest speed |u| of the reference",
            "_smallest_domain": small}


def surrogate_leg(lbm, torch, stream, max_over_ranks, barrier, train_steps: int = 1500, windows: int = 400,
                  per_generator: int = 8, side: int = 512, data_windows: int = 400, lr: float = 1e-3,
                  pushforward: float = 0.3, audits=(4, 8), lb_first: int = 40, short_warm: int = 2000,
                  short_windows: int = 40, batch: int = 4, drift_factor: float = 2.5):
    """The learned surrogate against the plain LB on the forced-flow case
    (1024^2, one seed, inflow u_x = 0.01).

    Training: (t, t + 50) pairs of LB trajectories on side^2 domains from the
    three workload generators (workloads.surrogate_training_set: the forced-
    flow dendrite, the parameter sweep's draws, crops of the multi-seed
    thermosolutal box; per_generator each), 400 windows from the seed, with
    the push-forward samples of surrogate.train_rollout.

    Long run (the headline): `windows` windows of K = 50 steps from the seed;
    the first lb_first windows by the LB, then the audited rollout with the
    drift budget of surrogate.rollout (tip tolerance 1 lattice unit; each
    audit charged drift_factor = 2.5 times its error per network window, the
    ratio of measured rollout drift to one-window error), one run per audit
    period in `audits`.  Short run: short_windows windows after
    short_warm LB steps.  Reports the device time of the plain LB and of each
    rollout and the final tip difference to the plain LB; the headline speedup
    is the best long-run one whose final tip difference is within the
    tolerance."""
    from paper_2209_01444_gb300 import surrogate as S, workloads as W

    K, tol = 50, 1.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    cases = W.surrogate_training_set(n=side, per_generator=per_generator, rng_seed=5)
    snaps = S.make_snapshots(cases, K=K, windows=data_windows)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    mean, std_in, std_out = S.normalisation(snaps[:-1].reshape(-1, side, side, 5), snaps[1:].reshape(-1, side, side, 5))
    net = S.UNet(batch, side, side, stream=stream)
    net.set_params(W.unet_params(S.param_shapes(), 3))
    net.set_norm(mean, std_in, std_out)
    torch.cuda.synchronize()
    ev0.record(stream)
    hist = S.train_rollout(net, snaps, steps=train_steps, lr=lr, seed=1, log_every=max(1, train_steps // 100),
                           pushforward=pushforward)
    ev1.record(stream)
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    params = net.params()
    del net, snaps
    torch.cuda.empty_cache()
    case = W.forced_flow(1024)
    cx, cy = float(case.seeds[0][0]), float(case.seeds[0][1])
    ev = S.UNet(1, 1024, 1024, stream=stream)
    ev.set_params(params)
    ev.set_norm(mean, std_in, std_out)

    def fresh(warm=0):
        s_ = lbm.Simulation(case.params, "fp32", stream=stream)
        s_.init_seeds(case.seeds, case.U0, case.theta0)
        if warm:
            s_.step(warm)
        return s_

    def tips(s_):
        m = s_.metrics(cx, cy, check=False)
        return np.array([m["tip_px"], m["tip_mx"], m["tip_py"]])

    def timed(fn):
        torch.cuda.synchronize()
        barrier()
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return out, max_over_ranks(ev0.elapsed_time(ev1))

    def compare(warm, n_windows, policies, first, budget=None):
        ref = fresh(warm)
        _, lb_ms = timed(lambda: ref.step(K * n_windows))
        tip_ref = tips(ref)
        del ref
        runs = []
        for a in policies:
            sur = fresh(warm)
            st, ms = timed(lambda: S.rollout(sur, ev, n_windows, K, tol, audit_every=a, backoff=4, cx=cx, cy=cy,
                                             lb_first=first, drift_budget=budget, drift_factor=drift_factor))
            err = float(np.abs(tips(sur) - tip_ref).max())
            runs.append({"audit_every": a, "ms": ms, "speedup_vs_plain_lb": lb_ms / ms, "final_tip_error_lu": err,
                         "windows_by_network": st["surrogate"], "audited": st["audited"],
                         "rejected_audits": st["rejected"], "nonfinite_windows": st["nonfinite"],
                         "lb_first": st["lb_first"],
                         "lb_after_budget": st["lb_after_budget"], "drift_charged_lu": st["drift_charged"],
                         "audit_tip_error_max_lu": max(st["tip_err"]) if st["tip_err"] else None})
            del sur
        return lb_ms, tip_ref, runs

    lb_ms, tip_ref, runs = compare(0, windows, audits, lb_first)
    # the fallback applied per window only (an audit re-runs its stretch when
    # that one window's tip error exceeds the tolerance), without the drift
    # budget: faster, but the final state drifts from the plain LB
    _, _, per_window = compare(0, windows, (audits[0],), lb_first, budget=float("inf"))
    s_lb_ms, _, s_runs = compare(short_warm, short_windows, (4,), 0)
    xin = torch.zeros(1, 1024, 1024, 5, device="cuda")
    yout = torch.empty_like(xin)
    for _ in range(3):
        ev.forward(xin, yout)
    _, fwd10 = timed(lambda: [ev.forward(xin, yout) for _ in range(10)])
    ok = [r for r in runs if r["final_tip_error_lu"] <= tol]
    best = max(ok, key=lambda r: r["speedup_vs_plain_lb"]) if ok else min(runs, key=lambda r: r["final_tip_error_lu"])
    return {
        "workload": f"forced_flow 1024x1024, one seed, inflow u_x = 0.01; {windows} windows of K = {K} steps "
                    f"from the seed, the first {lb_first} by the LB",
        "lb_ms": lb_ms, "tip_tolerance_lu": tol, "final_tips_plain_lb": tip_ref.tolist(),
        "speedup_vs_plain_lb": best["speedup_vs_plain_lb"], "final_tip_error_lu": best["final_tip_error_lu"],
        "matched": best["final_tip_error_lu"] <= tol, "best_audit_every": best["audit_every"],
        "rollouts": runs,
        "per_window_policy": dict(per_window[0], note="audits judge one window each; no drift budget"),
        "short": {"workload": f"{short_windows} windows after {short_warm} LB steps", "lb_ms": s_lb_ms,
                  "rollouts": s_runs},
        "network_forward_ms_1024": fwd10 / 10, "lb_ms_per_window": lb_ms / windows,
        "training": {"data": f"{len(cases)} trajectories {side}^2 ({per_generator} each of the forced-flow dendrite, "
                             f"the parameter sweep's draws and multi-seed thermosolutal crops; seed 5), "
                             f"{data_windows} windows from the seed",
                     "pairs": int(data_windows * len(cases)), "data_s": t_data, "steps": train_steps, "batch": batch,
                     "pushforward": pushforward, "lr": lr, "ms": train_ms,
                     "loss_first": hist[0][1],
                     # mean of the sampled mini-batch losses in each tenth of training (single losses vary
                     # with the share of push-forward samples, whose targets lie two windows ahead)
                     "loss_by_tenth": [float(np.mean([l for (i, l) in hist if k * train_steps <= 10 * i
                                                      < (k + 1) * train_steps] or [float("nan")]))
                                       for k in range(10)]},
    }


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2209_01444_gb300 import build_ext, lbm

    if not os.path.exists(lbm.LIB_PATH):
        build_ext.build()
    lbm.load()

    def barrier_():
        barrier(world)

    def max_ranks(x: float) -> float:
        return max_over_ranks(x, world, dev)

    case = workload(args.n)
    nodes = case.nodes
    stream = torch.cuda.current_stream()

    def timed_run(storage: str, steps: int, warmup: int, clocks: bool):
        sim = lbm.Simulation(case.params, storage, stream=stream)
        sim.init_seeds(case.seeds, case.U0, case.theta0)
        sums0 = sim.metrics(case.seeds[0][0], case.seeds[0][1], case.seeds[0][3], check=False)
        sim.sums0 = (sums0["sum_C"], sums0["sum_H"])
        sim.step(warmup)
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_index(local)) if clocks else None
        if sampler:
            sampler.__enter__()
        barrier_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier_()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = max_ranks(e0.elapsed_time(e1))
        m = sim.metrics(case.seeds[0][0], case.seeds[0][1], case.seeds[0][3], check=False)
        return sim, ms, (sampler.summary() if sampler else None), m

    sim, ms, clk, m = timed_run(args.storage, args.steps, max(args.warmup, 3), clocks=True)
    if m["nonfinite"]:
        raise RuntimeError("non-finite state after the timed run")
    conservation = drift(sim, m)
    ref_fields = sim.fields(ACCURACY_FIELDS) if not args.no_variants and args.storage == "fp32" else None
    value = whole_job_mlups(world, nodes, args.steps, ms)

    # fused-kernel time from CUDA events on the launching stream
    sim.set_profiling(True)
    kp = min(200, max(20, args.steps // 10))
    sim.step(kp)
    kms, launches = sim.kernel_time()
    sim.set_profiling(False)
    k_avg_ms = kms / max(launches, 1)
    grains = len(case.seeds) > 1
    bpn = algorithmic_bytes_per_node(args.storage, grains)
    achieved = bpn * nodes / (k_avg_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    kernel_name = "k_coupled_step"
    traffic = recorded_traffic(f"multi_seed_{args.n}_{args.storage}")

    # end to end through the C ABI from pinned host memory: load the initial
    # state, run the steps, read the fields back
    fresh = lbm.Simulation(case.params, args.storage, stream=stream)
    fresh.init_seeds(case.seeds, case.U0, case.theta0)
    blob = fresh.save()
    del fresh
    pinned = torch.empty(len(blob), dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = memoryview(blob)
    e2e_steps = args.steps
    e2e_sim = lbm.Simulation(case.params, args.storage, stream=stream)
    names = ("phi", "C", "theta", "ux", "uy")
    # the caller's page-locked result array, allocated once like the input
    fields_out = torch.empty((len(names), case.params["ny"], case.params["nx"]), dtype=torch.float32,
                             pin_memory=True).numpy()
    import ctypes as ct

    torch.cuda.synchronize()
    barrier_()
    t0 = time.perf_counter()
    rc = e2e_sim.lib.lbm_load_state(e2e_sim.h, ct.c_void_p(pinned.data_ptr()), len(blob))
    if rc:
        raise RuntimeError(e2e_sim.lib.lbm_last_error(e2e_sim.h).decode())
    t_load = time.perf_counter()
    e2e_sim.step(e2e_steps)
    e2e_sim.synchronize()
    t_steps = time.perf_counter()
    out = e2e_sim.fields_f32(names, out=fields_out)
    t1 = time.perf_counter()
    e2e_phases = {"load_state": (t_load - t0) * 1e3, "steps": (t_steps - t_load) * 1e3,
                  "get_fields": (t1 - t_steps) * 1e3}
    barrier_()
    e2e_s = max_ranks(t1 - t0)
    e2e_value = whole_job_mlups(world, nodes, e2e_steps, e2e_s * 1e3)
    # lbm_get_fields_f32 copies the requested FP32 fields (nx * ny values each) to the host
    d2h = len(names) * case.params["nx"] * case.params["ny"] * 4
    del out, fields_out

    variants = {}
    if not args.no_variants and args.storage == "fp32":
        for st in ("fp16", "bf16"):
            vs, vms, _, vm = timed_run(st, args.steps, max(args.warmup, 3), clocks=False)
            # accuracy at the FP32 run's step count, before the kernel timing takes more steps
            v_err = (field_errors(vs.fields(ACCURACY_FIELDS), ref_fields, abs(case.theta0))
                     if not vm["nonfinite"] else None)
            vs.set_profiling(True)
            vs.step(kp)
            vkms, vlaunches = vs.kernel_time()
            vs.set_profiling(False)
            v_ms = vkms / max(vlaunches, 1)
            vbpn = algorithmic_bytes_per_node(st, grains)
            v_ach = vbpn * nodes / (v_ms / 1e3) / 1e9
            # all 24 populations in 16 bits (the three rest planes too): 24 x 2 x 2 + 48 history (+ grain id)
            all16 = 24 * 2 * 2 + HIST_PLANES * 2 * 4 + (1 if grains else 0)
            variants[st] = {"value": whole_job_mlups(world, nodes, args.steps, vms), "unit": UNIT,
                            "speedup_vs_fp32": ms / vms, "nonfinite": vm["nonfinite"],
                            "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": v_ach, "peak": peak,
                                         "unit": "GB/s", "frac": v_ach / peak, "bytes_per_node": vbpn,
                                         "kernel_ms": v_ms, "peak_kind": peak_kind,
                                         "traffic": recorded_traffic(f"multi_seed_{args.n}_{st}"),
                                         "frac_at_all_16bit_bytes": all16 * nodes / (v_ms / 1e3) / 1e9 / peak,
                                         "all_16bit_bytes_per_node": all16}}
            if v_err is not None:
                variants[st]["field_error_vs_fp32"] = v_err
                variants[st]["conservation"] = drift(vs, vm)
            del vs
    del ref_fields

    substeps = None
    if not args.no_substeps:
        substeps = substep_leg(lbm, torch, stream, max_ranks, barrier_, n=args.substep_n)

    batch = None
    if not args.no_batch:
        batch = batch_leg(lbm, torch, stream, args.steps, world, max_ranks, barrier_)

    surrogate = None
    if not args.no_surrogate:
        surrogate = surrogate_leg(lbm, torch, stream, max_ranks, barrier_, args.surrogate_train_steps,
                                  args.surrogate_windows)

    if rank != 0:
        return
    cpu = None
    small = batch.pop("_smallest_domain") if batch else None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(case)
        cpu["one_core"] = cpu_oracle_one_core(case)
        if small is not None:
            cpu["batch_domain"], batch["vs_oracle_smallest_domain"] = cpu_oracle_batch_domain(small)
    wall_launches = (0 if case.params["bc"][2] == "periodic" else 1) + (0 if case.params["bc"][0] == "periodic" else 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.storage == "fp32" else f"f32 compute, {args.storage} storage",
        "data": "synthetic",
        "config": {"workload": f"multi_seed_thermosolutal_{args.n}x{args.n}", "nodes": nodes,
                   "seeds": len(case.seeds), "storage": args.storage, "n_sub": case.params["n_sub"],
                   "walls": "periodic x, no-slip y", "l2": "state larger than L2 (no flush)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": kernel_name, "bytes_per_node": bpn,
                     "kernel_ms": k_avg_ms, "peak_kind": peak_kind},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": len(blob) / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps,
                "what": "lbm_load_state from pinned host memory, lbm_step(steps), lbm_get_fields_f32 of 5 fields into pinned host memory",
                "phases_ms": e2e_phases},
        "gpu_launches": args.steps * (1 + wall_launches),
        "conservation": conservation,
        "clocks": clk,
        "cpu_baseline": cpu,
        "variants": variants,
        "flow_substeps": substeps,
        "batch": batch,
        "surrogate": surrogate,
        "metrics_after_run": {"solid_fraction": m["solid_fraction"], "tip_px": m["tip_px"]},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
