#!/usr/bin/env python3
"""Throughput of the coupled two-fluid lattice step on GB300.

Default workload: the activity sweep zeta in {0, 0.002, 0.005, 0.01} on
256x256 periodic grids (lambda 0.7, K 0.04, drag 0.01, tau 1), FP32, run as
one batch of four instances.  One bench step = one coupled lattice step of
all four instances (two D2Q9 fluids, forces, five Cahn-Hilliard and
Beris-Edwards sub-steps).  The state (~44 MB) fits in L2, so L2 is flushed
(256 MiB write) before every timed step and each step is timed alone with
CUDA events on the solver's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sweep256|single2048]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own copy of
the workload with its own seed (independent ensemble members, weak scaling);
only the timing is reduced across ranks (max).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS & % HBM roofline; surrogate/FP16 vs plain FP32 at stated error"
UNIT = "MLUPS"
BYTES_PER_SITE = 168  # FP32: 18 populations read + written (144 B) + phi, Q read + written (24 B)
FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "sweep256": dict(nx=256, ny=256, zetas=[0.0, 0.002, 0.005, 0.01],
                     name="zeta sweep {0,0.002,0.005,0.01} x 256x256, FP32, lambda 0.7, K 0.04"),
    "single2048": dict(nx=2048, ny=2048, zetas=[0.005],
                       name="single 2048x2048, FP32, zeta 0.005, lambda 0.7, K 0.04"),
}


# --------------------------------------------------------------- ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seed(base_seed: int, rank: int) -> int:
    """Each rank simulates independent ensemble members: seed offset by rank."""
    return base_seed + 1000003 * rank


def aggregate(per_rank_seconds, sites_per_rank: int, steps: int):
    """Whole-job throughput: all ranks' site updates over the slowest rank's time."""
    t = max(per_rank_seconds)
    total = sites_per_rank * steps * len(per_rank_seconds)
    return total / t / 1e6, t


def reduce_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------- roofline inputs
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_00445_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, only if it was
    taken from the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    sha = kernel_source_sha()
    for ln in lines:
        kv = dict(tok.split("=", 1) for tok in ln.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source_sha") == sha:
            return float(kv["bytes_per_launch"])
    return None


# ------------------------------------------------------------ oracle arm
def oracle_sample(nx, ny, zeta, seed, budget_s, max_steps=None):
    """Time the FP64 oracle on one instance of the workload (host cores)."""
    import numpy as np

    from oracle import twofluid as O
    from paper_2511_00445_gb300 import inputs
    p = O.Params(nx=nx, ny=ny, zeta=zeta)
    up, ut = inputs.initial_draws(seed, nx, ny)
    Q = O.q_from_director(0.01, np.pi * ut)
    s = O.state_from_fields(0.5 + 0.01 * (2 * up - 1), Q[0, 0], Q[0, 1], p)
    s = O.step(s, p)  # warm-up
    n, t0 = 0, time.perf_counter()
    while True:
        s = O.step(s, p)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and n >= max_steps):
            break
    return nx * ny * n / el / 1e6, n, el


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    nx, ny = wl["nx"], wl["ny"]
    zeta = wl["zetas"][len(wl["zetas"]) // 2]
    import numpy as np

    from oracle import twofluid as O
    from paper_2511_00445_gb300 import inputs
    p = O.Params(nx=nx, ny=ny, zeta=zeta)
    up, ut = inputs.initial_draws(0, nx, ny)
    Q = O.q_from_director(0.01, np.pi * ut)
    s = O.state_from_fields(0.5 + 0.01 * (2 * up - 1), Q[0, 0], Q[0, 1], p)
    for _ in range(args.warmup):
        s = O.step(s, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = O.step(s, p)
    el = time.perf_counter() - t0
    sites = nx * ny
    val = sites * args.steps / el / 1e6
    sample = (f"one instance (zeta={zeta}) of the {len(wl['zetas'])}-instance workload, "
              f"{nx}x{ny}, {args.steps} steps per run")
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 initial condition, Sec. III)",
        "config": {"workload": wl["name"], "sites_per_step": sites, "kind": "FP64 numpy oracle"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# -------------------------------------------------------------- our arm
def run_ours(args, wl):
    import torch

    from paper_2511_00445_gb300 import build as bld
    rank, world, local = dist_env()
    if rank == 0:
        bld.build()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        if rank != 0:
            bld.build()
    else:
        torch.cuda.set_device(local)
    from paper_2511_00445_gb300 import _binding as B
    dev = torch.device("cuda", local)
    params = [B.SolverParams(nx=wl["nx"], ny=wl["ny"], zeta=z) for z in wl["zetas"]]
    sites = wl["nx"] * wl["ny"] * len(params)
    tf = B.TwoFluid(params, device=dev)
    tf.init_fields(seed=rank_seed(0, rank), phi0=0.5, dphi=0.01, S0=0.01)
    stream = tf.stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            tf.step(1)
    torch.cuda.synchronize(dev)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = tf.kernel_launches()
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            tf.step(1)
            b.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    launches = tf.kernel_launches() - launches0
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    sec_local = sum(ms) / 1e3
    sec = reduce_max(sec_local, world, dev)
    value, _ = aggregate([sec] * world, sites, args.steps)
    ms_per_step = sec / args.steps * 1e3
    tf.sync()
    c = tf.conserved(0)  # finite state check after the timed region

    peak, peak_kind = measured_peaks()
    # With five sub-steps every timed step is one launch of the fused kernel.
    kernel_name = "k_fused<1,1>" if launches == args.steps else "tf_step (per-stage kernels)"
    achieved = BYTES_PER_SITE * sites / (statistics.mean(ms) / 1e3) / 1e9
    traffic = recorded_traffic(kernel_name, args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": kernel_name, "bytes_per_site": BYTES_PER_SITE,
                "launches_per_step": launches / args.steps}

    # End to end through the host-buffer entry point: raw state in from pinned
    # host memory, one step, raw state out, synchronised; wall clock.
    e2e = None
    if not args.no_e2e:
        nb = tf.state_bytes()
        h_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        tf.advance_host(None, 0, h_in.data_ptr())
        for _ in range(3):
            tf.advance_host(h_in.data_ptr(), 1, h_out.data_ptr())
        k_e2e = max(10, min(args.steps, 100))
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            tf.advance_host(h_in.data_ptr(), 1, h_out.data_ptr())
        el = reduce_max(time.perf_counter() - t0, world, dev)
        e2e = {"value": sites * k_e2e * world / el / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "api": "tf_advance_host (raw state in, 1 step, raw state out)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mlups, n, el = oracle_sample(wl["nx"], wl["ny"], wl["zetas"][len(wl["zetas"]) // 2], 0,
                                     budget_s=args.cpu_seconds)
        cpu = {"value": mlups, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 numpy oracle, one {wl['nx']}x{wl['ny']} instance, {n} steps "
                         f"({el:.1f} s) after one warm-up step"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded SplitMix64 initial condition of Sec. III)",
            "config": {"workload": wl["name"], "sites_per_step": sites, "instances": len(params),
                       "l2": "flushed (256 MiB write) before every timed step",
                       "timing": "CUDA events per step on the solver stream"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
            "state_check": {"nonfinite": c[7], "sum_phi": c[0]},
        }
        print(json.dumps(out), flush=True)
    tf.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sweep256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
