"""What FP32 arithmetic alone does to the method (CPU only).

The GPU parity bar is max |X_gpu - X_oracle| <= 1e-5 of the oracle field's
spread after 200 steps.  On grids a few sites wide the passive velocity u2 is
~100x smaller than u1 (its spread is ~1% of u1's at 8 x 8), and there no FP32
evaluation of the method meets that bar against u2's own spread.  The
float32 restatement in fp32_restatement.py (no code shared with the CUDA
library) shows it: after 200 steps of the 8 x 8 correctness run it departs
from the FP64 oracle by more than 1e-5 of u2's own spread, while it stays
below 1e-6 of the shared velocity scale (the larger spread of u1 and u2).
From 32 x 32 up the same restatement meets 1e-5 of every field's own spread,
u2 included; the GPU tests use u2's own spread there.
"""
import numpy as np
import pytest

import fp32_restatement as R
from oracle import twofluid as O
from paper_2511_00445_gb300 import inputs


def _run(nx, ny, steps=200):
    p = O.Params(nx=nx, ny=ny)
    up, ut = inputs.initial_draws(0, nx, ny)
    phi = 0.5 + 0.01 * (2 * up - 1)
    Q = O.q_from_director(0.01, np.pi * ut)
    s = O.state_from_fields(phi, Q[0, 0], Q[0, 1], p)
    r = R.from_oracle(s)
    for _ in range(steps):
        s = O.step(s, p)
        r = R.step(r, p)
    mc, mr = O.macro(s, p), R.macro(r, p)

    def spread(a):
        return np.abs(a - a.mean()).max()
    uscale = max(spread(c) for c in (*mc["u1"], *mc["u2"]))
    err = {
        "phi": np.abs(r.dphi + 0.5 - s.phi).max() / spread(s.phi),
        "Qxx": np.abs(r.a - s.Qxx).max() / spread(s.Qxx),
        "Qxy": np.abs(r.b - s.Qxy).max() / spread(s.Qxy),
    }
    for k in ("u1", "u2"):
        d = [np.abs(mr[k][c] - mc[k][c]).max() for c in range(2)]
        err[k + "_own"] = max(d[c] / spread(mc[k][c]) for c in range(2))
        err[k + "_shared"] = max(d) / uscale
    return err


def test_fp32_floor_on_8x8_is_above_the_bar_for_u2_own_spread():
    e = _run(8, 8)
    assert e["u2_own"] > 1e-5            # FP32 cannot meet 1e-5 of u2's own spread here
    assert e["u2_shared"] < 1e-6          # ... but is far inside it on the shared scale
    assert e["u1_own"] < 1e-5 and e["Qxx"] < 1e-5 and e["Qxy"] < 1e-5


@pytest.mark.parametrize("nx,ny", [(32, 32), (64, 48)])
def test_fp32_meets_the_bar_on_own_spreads_from_32(nx, ny):
    e = _run(nx, ny)
    for k in ("phi", "Qxx", "Qxy", "u1_own", "u2_own"):
        assert e[k] < 5e-6, (k, e[k])
