"""Writes longrun_ensemble_64.json: the FP64 oracle's statistics of a chaotic
ensemble, the expected values of tests/test_gpu_longrun_chaotic.py.

Calls only oracle/ and the seeded input generators.  Thirty-two seeds of
the correctness configuration (64 x 64, Sec. III parameter set of the oracle's
defaults) at activity zeta = 0.02, each started from the Sec. III initial
condition (phi = 0.5 + 0.01 (2U - 1), director angle pi U', S0 = 0.01, fluids
at rest) and run for 40 000 lattice steps.  Two trajectories of this flow that
start 1e-7 apart separate to O(1) differences in phi by step ~7500, so the
record after step 10 000 is chaotic.  Every 250 steps the domain length L(t)
(Sec. IV, Eq. 27) is recorded; the kinetic-energy spectrum of the mixture
velocity (Eq. 22) is averaged over the records after step 10 000.

Statistical floor: the mean spectrum of one half of the seeds differs from the
other half's by a few percent in the box-scale shell (k = 1, about half of
the energy), so the ensemble is large enough that two independent 32-seed
means differ there by about 2% (one standard deviation).

Run time: about 13 minutes per 8 seeds on 8 host cores (one process per seed).
    python tests/golden/make_longrun_ensemble.py            # every seed
    python tests/golden/make_longrun_ensemble.py 8 9 10     # add or redo seeds
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SEEDS = list(range(32))
ZETA = 0.02
STEPS, EVERY, WINDOW_FROM = 40000, 250, 10000
OUT = os.path.join(HERE, "longrun_ensemble_64.json")


def one_seed(seed: int):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import numpy as np
    from oracle import twofluid as O
    from paper_2511_00445_gb300 import inputs

    p = O.Params(nx=64, ny=64, zeta=ZETA)
    up, ut = inputs.initial_draws(seed, p.nx, p.ny)
    Q = O.q_from_director(0.01, np.pi * ut)
    s = O.state_from_fields(0.5 + 0.01 * (2.0 * up - 1.0), Q[0, 0], Q[0, 1], p)
    L, E_win, n_win = [], 0.0, 0
    for r in range(STEPS // EVERY):
        s = O.run(s, p, EVERY)
        L.append(float(O.length_scale(s.phi)))
        if (r + 1) * EVERY > WINDOW_FROM:
            mc = O.macro(s, p)
            E_win = E_win + O.energy_spectrum(O.mixture_velocity(s.phi, mc["u1"], mc["u2"]))[0]
            n_win += 1
    return seed, L, (E_win / n_win).tolist()


def main(argv):
    todo = [int(a) for a in argv] or SEEDS
    assert all(s in SEEDS for s in todo), todo
    with mp.get_context("spawn").Pool(min(len(todo), os.cpu_count() or 1)) as pool:
        res = pool.map(one_seed, todo)
    doc = {"L": {}, "spectrum_window_mean": {}}
    if argv and os.path.exists(OUT):
        with open(OUT) as fh:
            doc = json.load(fh)
    doc["source"] = "oracle/twofluid.py (FP64), written by tests/golden/make_longrun_ensemble.py"
    doc["config"] = {"nx": 64, "ny": 64, "zeta": ZETA, "phi0": 0.5, "dphi": 0.01, "S0": 0.01,
                     "seeds": SEEDS, "steps": STEPS, "every": EVERY, "window_from": WINDOW_FROM}
    for seed, L, E in res:
        doc["L"][str(seed)] = [float(f"{v:.10g}") for v in L]
        doc["spectrum_window_mean"][str(seed)] = [float(f"{v:.10g}") for v in E]
    for key in ("L", "spectrum_window_mean"):
        doc[key] = {k: doc[key][k] for k in sorted(doc[key], key=int)}
    missing = [s for s in SEEDS if str(s) not in doc["L"]]
    assert not missing, f"seeds without a record: {missing}"
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=0)
        fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
