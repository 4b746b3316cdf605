"""Per-run metrics log: one JSON object per line (JSONL) every `every` steps.

`run_logged(tf, steps, every, path)` steps a TwoFluid context and, before the
first step and after every `every` steps, appends one line per instance with
the run's parameters and the Sec. IV observables the library evaluates on the
GPU: sum phi and total momentum (FP64 reductions), L(t) from the structure
factor, E(t) = <|u_c|^2>/2, the inter-phase velocity and vorticity differences
and RMS values, the concentration spread, and the stepping rate of the
interval (MLUPS and the 168 B/site HBM rate of FP32 storage, wall clock of
the interval including the reads).  All arithmetic is in the library; this
module only formats what it returns.
"""
from __future__ import annotations

import dataclasses
import json
import time
from typing import IO, Iterable

# Algorithmic HBM bytes per site and step of the fused step by population storage.
BYTES_PER_SITE = {0: 168, 1: 96, 2: 96}     # TF_STORE_F32, TF_STORE_F16, TF_STORE_BF16


def record(tf, inst: int, step: int, params, mlups: float | None, seconds: float | None) -> dict:
    """The log line of instance `inst` at step `step` (no stepping)."""
    cons = tf.conserved(inst, check=False)
    pd = tf.phase_difference(inst)
    _, e_total = tf.energy_spectrum(inst)
    phi_mean, phi_std = tf.phi_stats(inst)
    line = {
        "step": int(step), "instance": int(inst),
        "params": {k: v for k, v in dataclasses.asdict(params).items()},
        "sum_phi": float(cons[0]), "sum_rho": [float(cons[1]), float(cons[2])],
        "momentum": [float(cons[3]), float(cons[4])], "nonfinite": int(cons[7]),
        "L": float(tf.length_scale(inst)), "E": float(e_total),
        "delta_u_rms": float(pd[0]), "delta_w_rms": float(pd[1]),
        "u1_rms": float(pd[2]), "uc_rms": float(pd[3]), "w1_rms": float(pd[4]),
        "wc_rms": float(pd[5]), "phi_mean": float(phi_mean), "phi_std": float(phi_std),
    }
    if mlups is not None:
        line["mlups"] = float(mlups)
        line["hbm_gbs"] = float(mlups) * 1e6 * BYTES_PER_SITE.get(params.storage, 168) / 1e9
        line["seconds"] = float(seconds)
    return line


def write_lines(out: IO[str], lines: Iterable[dict]) -> None:
    for ln in lines:
        out.write(json.dumps(ln, sort_keys=True) + "\n")
    out.flush()


def run_logged(tf, steps: int, every: int, path: str, params=None, append: bool = False) -> int:
    """Step `tf` by `steps` steps, logging every `every` steps to `path`.

    params: the SolverParams of each instance (a list, or one for all); by
    default those the context was created with.  Returns the lines written.
    """
    if steps < 0 or every < 1:
        raise ValueError("steps must be >= 0 and every >= 1")
    plist = params if params is not None else tf.params
    if not isinstance(plist, (list, tuple)):
        plist = [plist] * tf.batch
    sites = sum(p.nx * p.ny for p in plist)
    n = 0
    with open(path, "a" if append else "w") as out:
        step0 = tf.step_count()
        write_lines(out, [record(tf, b, step0, plist[b], None, None) for b in range(tf.batch)])
        n += tf.batch
        done = 0
        while done < steps:
            k = min(every, steps - done)
            t0 = time.perf_counter()
            tf.step(k)
            tf.sync()
            sec = time.perf_counter() - t0
            done += k
            mlups = sites * k / sec / 1e6
            write_lines(out, [record(tf, b, step0 + done, plist[b], mlups, sec)
                              for b in range(tf.batch)])
            n += tf.batch
    return n
