#!/usr/bin/env python3
"""Throughput of the coupled two-fluid lattice step on GB300.

Default workload: one 2048 x 2048 periodic instance (zeta 0.005, lambda 0.7,
K 0.04, drag 0.01, tau 1), FP32, the size at which the step's HBM roofline
is measured (state ~0.9 GB, far larger than the 129 MB L2).  One bench step =
one coupled lattice step (two D2Q9 fluids, forces, five Cahn-Hilliard and
Beris-Edwards sub-steps) = one launch of the steady-state kernel.  Steps run
back to back; each is bracketed by CUDA events on the solver's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload single2048|single1024|sweep256|ensemble48|surrogate256]
                    [--storage f32|f16|bf16] [--kernel auto|tile|strip]

--workload sweep256 is the activity sweep zeta in {0, 0.002, 0.005, 0.01} on
four 256 x 256 instances; its state (~44 MB) fits in L2, so L2 is flushed
(256 MiB write) before every timed step there.

--workload ensemble48 steps 48 instances of three sizes (the parameter-sweep
ensemble) through the ensemble API with the launch shape its autotuner chose
(one persistent launch for all steps, one launch per step over every tile of
every group, or each group's own planned launches recorded into one graph),
and also times the same instances stepped context by context.

--storage f16|bf16 stores the populations as 16-bit deviations (FP32
arithmetic).  Such a run also times the FP32 storage on the same workload
(speedup) and reports how far the two trajectories are apart after
--error-steps steps from one initial state (fields, L and the energy
spectrum of instance 0 at the end, and L, E and the spectrum averaged over
the second half of the run, beside the same averages of an FP32 run from
another seed: the spread chaotic sampling alone gives).

Prints one JSON line (rank 0).  Under torchrun each rank runs its own copy of
the workload with its own seed (independent replicas, weak scaling); only the
timing is reduced across ranks (max).
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
# Algorithmic bytes per site and step: 18 populations read + written (FP32:
# 144 B, 16-bit storage: 72 B) + phi, Q read + written (24 B).
BYTES_PER_SITE = {"f32": 168, "f16": 96, "bf16": 96}
FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "sweep256": dict(nx=256, ny=256, zetas=[0.0, 0.002, 0.005, 0.01],
                     name="zeta sweep {0,0.002,0.005,0.01} x 256x256, FP32, lambda 0.7, K 0.04"),
    "single1024": dict(nx=1024, ny=1024, zetas=[0.005],
                       name="single 1024x1024, FP32, zeta 0.005, lambda 0.7, K 0.04"),
    "single2048": dict(nx=2048, ny=2048, zetas=[0.005], large=True,
                       name="single 2048x2048, FP32, zeta 0.005, lambda 0.7, K 0.04"),
    # 48 instances: sizes {128, 256, 512}^2 (16 each); parameter combination
    # c = b mod 27 over zeta x lambda x K (lexicographic); seed b.
    "ensemble48": dict(nx=512, ny=512, zetas=[0.005], ensemble=True,
                       name="ensemble of 48: 16 x 128^2 + 16 x 256^2 + 16 x 512^2, FP32, "
                            "zeta {0.001,0.005,0.01} x lambda {0.3,0.7,1.1} x K {0.02,0.04,0.08}"),
}
WORKLOADS["surrogate256"] = dict(
    nx=256, ny=256, zetas=[0.0, 0.002, 0.005, 0.01], surrogate=True,
    name="U-Net surrogate, 4 levels x 32 base channels, BF16, 256x256, horizon 50 steps, "
         "trained on the zeta sweep {0,0.002,0.005,0.01}")
ENS_ZETA, ENS_LAMBDA, ENS_K = (0.001, 0.005, 0.01), (0.3, 0.7, 1.1), (0.02, 0.04, 0.08)


def ensemble_members(B, storage):
    """Per size group: the instances' parameters and seeds (b = 0..47)."""
    groups = []
    for gi, n in enumerate((128, 256, 512)):
        plist, seeds = [], []
        for b in range(16 * gi, 16 * gi + 16):
            c = b % 27
            plist.append(B.SolverParams(nx=n, ny=n, zeta=ENS_ZETA[c // 9], lam=ENS_LAMBDA[(c // 3) % 3],
                                        K=ENS_K[c % 3], storage=storage))
            seeds.append(b)
        groups.append((plist, seeds))
    return groups


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
class NvmlClocks:
    """SM clock and clock-event reasons read in-process through the driver's
    NVML library every 2 ms while the timed region runs (read-only queries).
    Raises OSError when NVML cannot be used; ClockSampler then falls back to
    nvidia-smi."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, cuda_index: int):
        import ctypes
        self.ct = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.lib = lib
        idx = cuda_index
        try:
            import torch
            idx = torch.cuda._get_nvml_device_index(cuda_index)
        except Exception:
            pass
        self.h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.stop_flag = threading.Event()

    def _clock(self, fn):
        v = self.ct.c_uint()
        return v.value if fn(self.h, self.ct.c_int(1), self.ct.byref(v)) == 0 else None   # 1: SM

    def _loop(self):
        while not self.stop_flag.is_set():
            mhz = self._clock(self.lib.nvmlDeviceGetClockInfo)
            r = self.ct.c_ulonglong()
            ok = self.get_reasons(self.h, self.ct.byref(r)) == 0
            if mhz is not None and ok:
                self.samples.append((mhz, r.value))
            self.stop_flag.wait(0.002)

    def start(self):
        self.samples = []
        self.stop_flag.clear()
        self.th = threading.Thread(target=self._loop, daemon=True)
        self.th.start()

    def stop(self):
        self.stop_flag.set()
        self.th.join(timeout=2)
        return self.summarise(self.samples, self._clock(self.lib.nvmlDeviceGetMaxClockInfo))

    @classmethod
    def summarise(cls, samples, smax):
        """(SM MHz, clock-event reason bits) samples -> the JSON `clocks` object."""
        if not samples:
            return None
        reasons = sorted({nm for _, bits in samples for b, nm in cls.REASONS.items() if bits & b})
        return {"sm_mhz": statistics.median(m for m, _ in samples), "sm_max_mhz": smax,
                "reasons": reasons, "when": "during the timed region", "samples": len(samples),
                "source": "NVML every 2 ms"}


class ClockSampler:
    """Clocks during the timed region: NVML in-process when the driver's
    library loads (NvmlClocks), else nvidia-smi samples every 50 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.mark = 0
        try:
            self.nvml = NvmlClocks(gpu_index)
        except (OSError, AttributeError):
            self.nvml = None

    def start(self):
        """Start sampling.  The nvidia-smi path returns once its first sample
        is in (at most ~3 s), so that the timed region that follows is covered
        from its start; that first sample, taken before the region, is left out."""
        if self.nvml is not None:
            self.nvml.start()
            return
        self.mark = 0
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)
        self.mark = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            return self.nvml.stop()
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)     # the reader has taken every line nvidia-smi wrote
        self.at_end = False
        self.lines = self.lines[self.mark:]
        if not self.lines:
            # the timed region was shorter than the sampler's start-up: one query
            # right at its end, while the clocks still reflect the load
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=10).stdout
                self.lines = [ln.strip() for ln in out.splitlines() if ln.strip()]
                self.at_end = True
            except (OSError, subprocess.SubprocessError):
                pass
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
                "when": "at the end of the timed region" if self.at_end else "during the timed region",
                "samples": len(sm)}


# ----------------------------------------------------- roofline inputs
NOMINAL_HBM_GBS = 7900.0     # GB300 HBM3e nominal bandwidth, for context beside the measured peak


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Sources the per-context fused kernel is compiled from.
FUSED_SOURCES = ("tf_device.cuh", "tf_fused.cu", "tf_fused.cuh", "tf_strip.cuh", "tf_internal.h", "tf_pair.cuh",
                 "tf_ptx.cuh", "tf_check.cuh")


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_00445_gb300", "csrc")
    for f in FUSED_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str, storage: str = "f32"):
    """DRAM bytes per launch from a committed ncu summary, only if it was
    taken from the current kernel sources (and the same population storage)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    sha = kernel_source_sha()
    for ln in lines:
        kv = dict(tok.split("=", 1) for tok in ln.split() if "=" in tok)
        if (kv.get("kernel") == kernel and kv.get("workload") == workload
                and kv.get("source_sha") == sha and kv.get("storage", "f32") == storage):
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


def _oracle_worker(job):
    nx, ny, zeta, seed, budget_s = job
    return oracle_sample(nx, ny, zeta, seed, budget_s)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_all_cores(nx, ny, zeta, budget_s, procs):
    """The FP64 oracle on every host core: `procs` spawned processes, each
    stepping its own instance (different seeds) for budget_s seconds; the
    sum of their site-update rates.  Each process runs single-threaded
    numpy (BLAS threads pinned to one)."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                          "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(nx, ny, zeta, k, budget_s) for k in range(procs)])
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(r[0] for r in res), sum(r[1] for r in res), max(r[2] for r in res)


def cpu_baseline(nx, ny, zeta, budget_s):
    """The oracle as it stands on the machine's host cores: one core, then all
    cores, each on instances of at most 512 x 512 sites of the workload's
    parameters (the oracle's cost per site update does not depend on the
    grid size; a 2048^2 instance would take several seconds per step)."""
    sx, sy = min(nx, 512), min(ny, 512)
    one, n1, el1 = oracle_sample(sx, sy, zeta, 0, budget_s=budget_s)
    procs = host_cores()
    allc, nall, elall = oracle_all_cores(sx, sy, zeta, budget_s, procs)
    return {"value": allc, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"FP64 numpy oracle, {procs} processes each stepping its own {sx}x{sy} "
                      f"instance (zeta {zeta}) for ~{budget_s:.0f} s ({nall} steps in all)",
            "one_core": {"value": one, "unit": UNIT, "cores": 1,
                         "sample": f"one {sx}x{sy} instance, {n1} steps ({el1:.1f} s) after one "
                                   f"warm-up step"}}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each timed step is a bounded sample of the workload: one oracle step of
    # one instance, cut to 128 x 128 sites for the 2048^2 workload (same
    # parameters; the oracle's cost per site update does not depend on size)
    nx, ny = (min(wl["nx"], 128), min(wl["ny"], 128)) if wl.get("large") else (wl["nx"], wl["ny"])
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
    sample = (f"one {nx}x{ny} instance (zeta={zeta}) with the workload's parameters, "
              f"{args.steps} oracle steps on one host core")
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
def time_steps(tf, flush, steps: int, warmup: int, world: int, dev, clocks=None):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    solver stream (after an L2 flush when `flush` is a buffer; back to back
    when it is None, for states far larger than L2); barrier + synchronize on
    both sides."""
    import torch
    stream = tf.stream
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            if flush is not None:
                flush.zero_()
            tf.step(1)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if clocks is not None:
        clocks.start()
    launches0 = tf.kernel_launches()
    with torch.cuda.stream(stream):
        for a, b in evs:
            if flush is not None:
                flush.zero_()
            a.record(stream)
            tf.step(1)
            b.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    launches = tf.kernel_launches() - launches0
    clk = clocks.stop() if clocks is not None else None
    return [a.elapsed_time(b) for a, b in evs], launches, clk


def trajectory_gap(B, params, seed: int, steps: int, storage: int, dev) -> dict:
    """Instance 0 of the workload advanced `steps` steps from one initial
    state with FP32 storage and with `storage`: max field differences
    normalised by the FP32 field's spread, and the relative differences of
    L (Eq. 27), <|u_c|^2>/2 and the energy spectrum (Eq. 22) shells."""
    import numpy as np
    runs, means = {}, {}
    # time averages of L, E and the spectrum over the second half of the run
    # (about 50 samples), the comparison that still means something once the
    # chaotic trajectories have separated pointwise; "control" is an FP32 run
    # from another seed, the spread that chaotic sampling alone gives them
    every = max(1, steps // 100)
    for mode in (B.STORE_F32, storage, "control"):
        tf = B.TwoFluid([params[0].with_(storage=B.STORE_F32 if mode == "control" else mode)], device=dev)
        tf.init_fields(seed=seed + (1000 if mode == "control" else 0), phi0=0.5, dphi=0.01, S0=0.01)
        done, samples = 0, []
        while done < steps:
            k = min(every, steps - done)
            tf.step(k)
            done += k
            if 2 * done > steps:
                E, Et = tf.energy_spectrum(0)
                samples.append((tf.length_scale(0), Et, E))
        flds = {k: tf.read_field(0, f) for k, f in (
            ("phi", B.FIELD_PHI), ("Qxx", B.FIELD_QXX), ("Qxy", B.FIELD_QXY),
            ("u1x", B.FIELD_U1X), ("u1y", B.FIELD_U1Y), ("u2x", B.FIELD_U2X), ("u2y", B.FIELD_U2Y))}
        E, Et = tf.energy_spectrum(0)
        runs[mode] = (flds, tf.length_scale(0), E, Et)
        means[mode] = (float(np.mean([x[0] for x in samples])), float(np.mean([x[1] for x in samples])),
                       np.mean([x[2] for x in samples], axis=0), len(samples))
        tf.close()
    (f0, L0, E0, Et0), (f1, L1, E1, Et1) = runs[B.STORE_F32], runs[storage]
    mL0, mE0, mS0, ns = means[B.STORE_F32]
    mlive = mS0 > 1e-3 * mS0.max()

    def mean_gaps(m):
        mL, mE, mS, _ = m
        return {"L_mean_rel": abs(mL - mL0) / mL0, "E_total_mean_rel": abs(mE - mE0) / mE0,
                "E_shell_mean_l1": float(np.abs(mS - mS0).sum() / mS0.sum()),
                "E_shell_mean_rel_max": float((np.abs(mS - mS0)[mlive] / mS0[mlive]).max())}

    def gap(a, b):
        sp = float(np.abs(a - a.mean()).max()) or float(np.abs(a).max()) or 1.0
        return float(np.abs(b - a).max()) / sp
    uscale = max(float(np.abs(f0[k] - f0[k].mean()).max()) for k in ("u1x", "u1y", "u2x", "u2y"))
    ugap = {k: float(np.abs(f1[k] - f0[k]).max()) / uscale for k in ("u1x", "u1y", "u2x", "u2y")}
    live = E0 > 1e-3 * E0.max()
    return {"steps": steps, "phi": gap(f0["phi"], f1["phi"]),
            "Q": max(gap(f0["Qxx"], f1["Qxx"]), gap(f0["Qxy"], f1["Qxy"])),
            "u": max(ugap.values()), "L_rel": abs(L1 - L0) / L0,
            "E_total_rel": abs(Et1 - Et0) / Et0,
            "E_shell_rel_max": float((np.abs(E1 - E0)[live] / E0[live]).max()),
            "mean_samples": ns, **mean_gaps(means[storage]),
            "control_fp32_other_seed": mean_gaps(means["control"]),
            "normalisation": "max |X_16 - X_32| / max |X_32 - <X_32>| (u: largest u spread); "
                             "means over the second half of the run"}


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
    storage = B.STORAGE_NAMES[args.storage]
    params = [B.SolverParams(nx=wl["nx"], ny=wl["ny"], zeta=z, storage=storage) for z in wl["zetas"]]
    sites = wl["nx"] * wl["ny"] * len(params)
    seed = rank_seed(0, rank)
    tf = B.TwoFluid(params, device=dev)
    tf.set_step_kernel(args.kernel)
    tf.init_fields(seed=seed, phi0=0.5, dphi=0.01, S0=0.01)
    tf_state_gb = tf.state_bytes() / 1e9
    step_kernel = tf.step_kernel()
    flush = None if wl.get("large") else torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    ms, launches, clk = time_steps(tf, flush, args.steps, args.warmup, world, dev, clocks)
    sec_local = sum(ms) / 1e3
    sec = reduce_max(sec_local, world, dev)
    value, _ = aggregate([sec] * world, sites, args.steps)
    ms_per_step = sec / args.steps * 1e3
    tf.sync()
    c = tf.conserved(0)  # finite state check after the timed region

    peak, peak_kind = measured_peaks()
    bps = BYTES_PER_SITE[args.storage]
    # With five sub-steps every timed step is one launch of the steady-state kernel.
    kernel_name = ("tf_step (per-stage kernels)" if launches != args.steps else
                   "k_strip" if step_kernel == B.KERNEL_STRIP else "k_fused<1,1>")
    achieved = bps * sites / (statistics.mean(ms) / 1e3) / 1e9
    traffic = recorded_traffic(kernel_name, args.workload, args.storage)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": kernel_name, "bytes_per_site": bps,
                "launches_per_step": launches / args.steps,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS}

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
               "api": "tf_advance_host (raw state in, 1 step, raw state out; pipelined per instance on "
                      "batches, per row band on a single instance)"}
    tf.close()

    # 16-bit storage: FP32 storage on the same workload, timed the same way,
    # and the distance between the two trajectories.
    precision = None
    if storage != B.STORE_F32:
        ref = B.TwoFluid([p.with_(storage=B.STORE_F32) for p in params], device=dev)
        ref.set_step_kernel(args.kernel)
        ref.init_fields(seed=seed, phi0=0.5, dphi=0.01, S0=0.01)
        ms32, _, _ = time_steps(ref, flush, args.steps, args.warmup, world, dev)
        ref.close()
        sec32 = reduce_max(sum(ms32) / 1e3, world, dev)
        value32, _ = aggregate([sec32] * world, sites, args.steps)
        precision = {"storage": args.storage, "f32_value": value32, "speedup_vs_f32": value / value32,
                     "gap_vs_f32": trajectory_gap(B, params, seed, args.error_steps, storage, dev)
                     if rank == 0 else None}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl["nx"], wl["ny"], wl["zetas"][len(wl["zetas"]) // 2], args.cpu_seconds)

    if rank == 0:
        name = wl["name"] if storage == B.STORE_F32 else wl["name"].replace(
            "FP32", f"FP32 arithmetic, {args.storage.upper()} population storage")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded SplitMix64 initial condition of Sec. III)",
            "config": {"workload": name, "sites_per_step": sites, "instances": len(params),
                       "storage": args.storage,
                       "l2": ("not flushed: the state (~%.2f GB) is far larger than L2, "
                              "steps run back to back" % (tf_state_gb,)) if flush is None
                             else "flushed (256 MiB write) before every timed step",
                       "timing": "CUDA events per step on the solver stream"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
            "state_check": {"nonfinite": c[7], "sum_phi": c[0]},
        }
        if precision is not None:
            out["precision"] = precision
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ensemble(args, wl):
    """48 instances of three sizes stepped through the ensemble API with the
    launch shape its autotuner picked (one persistent launch per K steps or
    one launch per step over all groups' tiles), against the same instances
    stepped context by context with one launch per group and step."""
    import torch

    from paper_2511_00445_gb300 import build as bld
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    bld.build()
    from paper_2511_00445_gb300 import _binding as B
    dev = torch.device("cuda", local)
    storage = B.STORAGE_NAMES[args.storage]
    spec = ensemble_members(B, storage)

    def make():
        grp = []
        for plist, seeds in spec:
            tf = B.TwoFluid(plist, device=dev)
            for k, sd in enumerate(seeds):
                tf.init_fields(seed=rank_seed(sd, rank), phi0=0.5, dphi=0.01, S0=0.01, inst=k)
            grp.append(tf)
        return grp
    sites = sum(p.nx * p.ny for plist, _ in spec for p in plist)
    grp = make()
    ens = B.Ensemble(grp)
    ens.autotune(max(2, min(8, args.warmup)))
    ens.step(args.warmup)
    ens.sync()
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    l0 = ens.launches()
    with torch.cuda.stream(ens.stream):
        a.record(ens.stream)
        ens.step(args.steps)
        b.record(ens.stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    launches = ens.launches() - l0
    clk = clocks.stop()
    ens.sync()
    sec = reduce_max(a.elapsed_time(b) / 1e3, world, dev)
    value, _ = aggregate([sec] * world, sites, args.steps)
    cfg = ens.config()
    c = grp[2].conserved(0)
    ens.close()
    for tf in grp:
        tf.close()

    # The same instances stepped per context: one launch per group and step.
    grp = make()
    for tf in grp:
        tf.step(args.warmup)
    torch.cuda.synchronize(dev)
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(grp[0].stream):
        a2.record(grp[0].stream)
        for _ in range(args.steps):
            for tf in grp:
                tf.step(1)
        b2.record(grp[0].stream)
    torch.cuda.synchronize(dev)
    sec_pc = reduce_max(a2.elapsed_time(b2) / 1e3, world, dev)
    value_pc, _ = aggregate([sec_pc] * world, sites, args.steps)
    for tf in grp:
        tf.close()

    peak, peak_kind = measured_peaks()
    bps = BYTES_PER_SITE[args.storage]
    achieved = bps * sites / (sec / args.steps) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                "kernel": ("k_ens (persistent, all steps in one launch)" if cfg["persistent"] else
                           "each group's own planned kernel (k_strip / k_fused<1,1>), one launch "
                           "per group and step" if cfg["group_plans"] else
                           "k_ens_step (one launch per step over every tile of every group)"),
                "bytes_per_site": bps,
                "launches_per_step": launches / args.steps,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(256, 256, 0.005, args.cpu_seconds)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded SplitMix64 initial condition of Sec. III, seed = member index)",
            "config": {"workload": wl["name"], "sites_per_step": sites, "instances": 48,
                       "storage": args.storage,
                       "l2": "not flushed: the state (~1.2 GB) is far larger than L2",
                       "timing": "CUDA events around the ensemble's launches of all K steps",
                       "autotuned": cfg},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": None, "clocks": clk, "gpu_launches": launches,
            "per_context": {"value": value_pc, "unit": UNIT,
                            "how": "same 48 instances as 3 contexts, one launch per context and step",
                            "ensemble_speedup": value / value_pc},
            "state_check": {"nonfinite": c[7], "sum_phi": c[0]},
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def unet_flops(levels: int, c0: int, n: int) -> float:
    """Multiply-adds x 2 of one forward pass on an n x n lattice."""
    ch = [c0 << l for l in range(levels)]
    f, prev = 0.0, 8
    for l in range(levels):
        px = (n >> l) ** 2
        f += 2 * px * 9 * (prev * ch[l] + ch[l] * ch[l])
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        px = (n >> l) ** 2
        f += 2 * px * 9 * ((ch[l + 1] + ch[l]) * ch[l] + ch[l] * ch[l])
    return f + 2 * n * n * c0 * 7


def run_surrogate(args, wl):
    """Train the surrogate on the sweep's trajectories, then time one
    prediction (horizon steps of one instance) against the plain step doing
    the same horizon, and state the prediction's error on a held-out seed."""
    import numpy as np
    import torch

    from paper_2511_00445_gb300 import build as bld
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    bld.build()
    from paper_2511_00445_gb300 import _binding as B
    dev = torch.device("cuda", local)
    nx, horizon, levels, c0 = wl["nx"], 50, 4, 32
    zetas = wl["zetas"]
    sur = B.Surrogate(levels=levels, base_channels=c0, nx=nx, ny=nx, max_batch=4, max_pairs=64,
                      horizon=horizon, device=dev)
    sur.init_weights(7)
    slot = 0
    for sd in (1, 2):
        tf = B.TwoFluid([B.SolverParams(nx=nx, ny=nx, zeta=z) for z in zetas], device=dev)
        tf.init_fields(rank_seed(sd, rank), phi0=0.5, dphi=0.01, S0=0.3)
        tf.step(400)
        for _ in range(8):
            for b in range(len(zetas)):
                sur.add_pair(slot + b, tf, b, 0)
            tf.step(horizon)
            for b in range(len(zetas)):
                sur.add_pair(slot + b, tf, b, 1)
            slot += len(zetas)
        tf.close()
    sur.fit_normalisation(slot)
    train_steps = 800
    t0 = time.perf_counter()
    losses = sur.train(slot, steps=train_steps, batch=4, lr=1e-3, seed=3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0

    # held-out seed: prediction vs the solver, and persistence
    def state(seed):
        tf = B.TwoFluid([B.SolverParams(nx=nx, ny=nx, zeta=z) for z in zetas], device=dev)
        tf.init_fields(seed, phi0=0.5, dphi=0.01, S0=0.3)
        tf.step(600)
        return tf
    truth, pred = state(rank_seed(11, rank)), state(rank_seed(11, rank))
    L0 = [truth.length_scale(b) for b in range(len(zetas))]
    E0 = [truth.energy_spectrum(b) for b in range(len(zetas))]
    truth.step(horizon)
    for b in range(len(zetas)):
        sur.predict(pred, b)
    err = {"L_rel": [], "L_rel_persist": [], "E_total_rel": [], "E_total_rel_persist": [],
           "E_shell_l1": [], "E_shell_l1_persist": []}
    for b in range(len(zetas)):
        Lt, Lp = truth.length_scale(b), pred.length_scale(b)
        (Et, Ett), (Ep, Ept) = truth.energy_spectrum(b), pred.energy_spectrum(b)
        err["L_rel"].append(abs(Lp - Lt) / Lt)
        err["L_rel_persist"].append(abs(L0[b] - Lt) / Lt)
        err["E_total_rel"].append(abs(Ept - Ett) / Ett)
        err["E_total_rel_persist"].append(abs(E0[b][1] - Ett) / Ett)
        err["E_shell_l1"].append(float(np.abs(Ep - Et).sum() / Et.sum()))
        err["E_shell_l1_persist"].append(float(np.abs(E0[b][0] - Et).sum() / Et.sum()))
    err = {k: float(np.mean(v)) for k, v in err.items()}

    # timing: one prediction (one instance, horizon steps) vs the plain step
    one = B.TwoFluid(B.SolverParams(nx=nx, ny=nx, zeta=0.005), device=dev)
    one.init_fields(5, phi0=0.5, dphi=0.01, S0=0.3)
    one.step(100)
    stream = one.stream
    for _ in range(args.warmup):
        sur.predict(one, 0)
    torch.cuda.synchronize(dev)
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(args.steps):
            sur.predict(one, 0)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_pred = a.elapsed_time(b_) / 1e3 / args.steps
    one.step(args.warmup * horizon)
    torch.cuda.synchronize(dev)
    plain_clocks = ClockSampler(torch.cuda.current_device())
    plain_clocks.start()
    with torch.cuda.stream(stream):
        a.record(stream)
        one.step(args.steps * horizon)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    clk_plain = plain_clocks.stop()
    t_plain = a.elapsed_time(b_) / 1e3 / args.steps
    one.close()
    # the whole sweep (four instances) predicted as one batch vs the batched plain step
    sweep = state(rank_seed(21, rank))
    for _ in range(args.warmup):
        sur.predict(sweep, -1)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(args.steps):
            sur.predict(sweep, -1)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    t_pred4 = a.elapsed_time(b_) / 1e3 / args.steps
    sweep.step(args.warmup * horizon)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        a.record(stream)
        sweep.step(args.steps * horizon)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    t_plain4 = a.elapsed_time(b_) / 1e3 / args.steps
    sites = nx * nx
    value = horizon * sites / t_pred / 1e6
    plain = horizon * sites / t_plain / 1e6
    flops = unet_flops(levels, c0, nx)
    peak = 1919.9
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
        peak_kind = "measured burst"
    except (OSError, KeyError, ValueError):
        peak_kind = "fallback"
    achieved = flops / t_pred / 1e12
    train_flops = 3 * flops * 4 * train_steps / t_train / 1e12
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_pred * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (solver trajectories from the seeded initial condition of Sec. III)",
            "config": {"workload": wl["name"], "sites_per_step": sites,
                       "step": "one prediction = 50 lattice steps of one 256^2 instance",
                       "value": "equivalent MLUPS = 50 x sites / prediction time",
                       "l2": "not flushed (activations of one prediction ~60 MB)",
                       "timing": "CUDA events around K predictions on the solver stream"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "whole prediction (tcgen05 convolutions + element-wise)",
                         "flops_per_prediction": flops},
            "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": None,
            "surrogate": {"plain_value": plain, "plain_clocks": clk_plain, "speedup_vs_plain": value / plain,
                          "sweep4": {"value": horizon * 4 * sites / t_pred4 / 1e6,
                                     "plain_value": horizon * 4 * sites / t_plain4 / 1e6,
                                     "speedup_vs_plain": t_plain4 / t_pred4,
                                     "tflops": flops * 4 / t_pred4 / 1e12,
                                     "how": "four sweep instances predicted as one batch vs "
                                            "the plain step of the same batch"},
                          "error_vs_solver_heldout": err, "train_steps": train_steps,
                          "train_pairs": slot, "train_seconds": t_train,
                          "train_tflops": train_flops,
                          "loss_first_last": [float(np.mean(losses[:5])), float(np.mean(losses[-20:]))]},
        }
        print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2000 for single2048, 200 otherwise)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="single2048")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32",
                    help="population storage (arithmetic is FP32 in every mode)")
    ap.add_argument("--kernel", choices=["auto", "tile", "strip"], default="auto",
                    help="steady-state kernel (auto: strip on grids of several tile waves)")
    ap.add_argument("--error-steps", type=int, default=200,
                    help="steps of the FP32-vs-16-bit trajectory comparison")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.steps is None:
        args.steps = 2000 if wl.get("large") else 200
    if args.impl == "reference":
        run_reference(args, wl)
    elif wl.get("ensemble"):
        run_ensemble(args, wl)
    elif wl.get("surrogate"):
        run_surrogate(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
