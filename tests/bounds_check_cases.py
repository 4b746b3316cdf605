"""Cases run with the bounds-check build of the library (libtwofluid_bc.so).

Run as a script (``python tests/bounds_check_cases.py OUT.npz`` with the
TF_LIBRARY environment variable naming the library): every case steps small,
ragged and degenerate grids through the tile kernel, the strip kernel, the
per-stage kernels and ensembles (persistent and per-step launches), checks that tf_sync / tf_ensemble_sync
report no failed index check, and saves the resulting fields.  The GPU test
runs the same cases with the normal library and compares them bitwise.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_00445_gb300 import _binding as B  # noqa: E402

FIELDS = [B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_U1X, B.FIELD_U2Y, B.FIELD_F1 + 5,
          B.FIELD_F2 + 7]
CASES = [  # (nx, ny, kernel, n_sub, storage, steps)
    (1, 1, "tile", 5, B.STORE_F32, 6), (2, 7, "tile", 5, B.STORE_F32, 6),
    (5, 3, "tile", 5, B.STORE_F32, 6), (33, 17, "tile", 5, B.STORE_F32, 6),
    (64, 48, "tile", 5, B.STORE_F16, 6), (9, 7, "tile", 3, B.STORE_F32, 4),
    (4, 4, "strip", 5, B.STORE_F32, 6), (4, 12, "strip", 5, B.STORE_F32, 6),
    (20, 3, "strip", 5, B.STORE_F32, 6), (100, 36, "strip", 5, B.STORE_F32, 6),
    (196, 40, "strip", 5, B.STORE_BF16, 6),
]


def run_cases() -> dict:
    out = {}
    for nx, ny, kernel, n_sub, storage, steps in CASES:
        p = B.SolverParams(nx=nx, ny=ny, n_sub=n_sub, storage=storage, zeta=0.01)
        tf = B.TwoFluid([p, p.with_(zeta=0.002)])
        if n_sub == 5:
            tf.set_step_kernel(kernel)
        tf.init_fields(3, phi0=0.5, dphi=0.05, S0=0.2)
        tf.step(steps - 2)
        tf.read_field(1, B.FIELD_PHI)          # epilogue, then prologue on the next step
        tf.step(2)
        tf.sync()                              # raises on TF_ERR_BOUNDS
        for inst in range(2):
            for f in FIELDS:
                out[f"{nx}x{ny}_{kernel}_{n_sub}_{storage}_{inst}_{f}"] = tf.read_field(inst, f)
        tf.close()
    # ensembles of ragged groups: the persistent launch (candidate 0), the
    # per-step launches with both tile shapes (candidates 6, 7) and the groups'
    # own launches (candidate 8)
    base = B.SolverParams(zeta=0.01)
    for cand in (0, 6, 7, 8):
        groups = [B.TwoFluid([base.with_(nx=40, ny=36), base.with_(nx=40, ny=36, lam=1.1)]),
                  B.TwoFluid(base.with_(nx=33, ny=17)), B.TwoFluid(base.with_(nx=100, ny=70))]
        for g, tf in enumerate(groups):
            for k in range(tf.batch):
                tf.init_fields(10 * g + k, phi0=0.5, dphi=0.05, S0=0.2, inst=k)
        ens = B.Ensemble(groups)
        ens.select(cand)
        ens.step(5)
        ens.sync()
        ens.close()
        for g, tf in enumerate(groups):
            for inst in range(tf.batch):
                for f in FIELDS:
                    out[f"ens{cand}_{g}_{inst}_{f}"] = tf.read_field(inst, f)
            tf.close()
    return out


if __name__ == "__main__":
    res = run_cases()
    np.savez(sys.argv[1], **res)
    print("bounds-check cases ok:", len(res), "arrays, library", B.LIB_PATH)
