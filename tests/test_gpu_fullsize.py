"""Parity at the full benchmarked grid sizes, in the launch configuration the
benchmark times (wide 40 x 30 tiles over several waves; 16-bit storage).

The oracle cannot step a 2048^2 grid in seconds, but one coupled lattice step
has a finite domain of dependence: a site's new state depends only on sites
within a few lattice spacings (streaming and the force stencils of the LBM
stage, then two lattice spacings per finite-difference sub-step: the Laplacian
of mu, itself a Laplacian of phi).  So the oracle steps a window cut, with the
grid's periodic wrap, from the GPU state read back exactly; the window's
sites more than H from its edge must agree with the GPU's own next step.  The
CPU test below checks that property of the oracle itself (a window step equals
the full-grid step in the interior, and a too-narrow margin does not).
"""
import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B
from paper_2511_00445_gb300 import inputs

from helpers import interior, oracle_params, read_state, read_velocities, window_step

H = 16            # window margin: more than the dependence radius of one step
WIN = 32          # compared interior of each window
# One FP32 step from identical inputs: max |X_gpu - X_oracle| over the field's
# spread.  Measured on GB300: 0.8-2.4e-7 for phi, Q, populations and
# velocities at every size here (the arithmetic is deterministic, so the
# figure is the same on every run); an indexing or tile-seam mistake is O(1e-2).
TOL_1STEP = 1e-6
UNIT_ROUNDOFF = {B.STORE_F16: 2.0**-11, B.STORE_BF16: 2.0**-8}


# ------------------------------------------------------------------ CPU pin of the method

def _developed_state(n=48, steps=6):
    p = O.Params(nx=n, ny=n, zeta=0.01)
    u_phi, u_theta = inputs.initial_draws(3, n, n)
    phi = 0.5 + 0.2 * (2 * u_phi - 1)
    th = np.pi * u_theta
    s = O.state_from_fields(phi, 0.3 * np.cos(2 * th), 0.3 * np.sin(2 * th), p)
    return O.run(s, p, steps), p


def test_window_step_equals_full_step():
    """Oracle step of a wrapped window == full-grid oracle step, in the
    window's interior, for a margin of H; a margin of 4 is too narrow."""
    s, p = _developed_state()
    full = O.step(s, p)
    mfull = O.macro(full, p)
    x0, y0, w, h = 40, 37, 16, 16          # crosses the wrap in both directions
    ys = (y0 + np.arange(h)) % p.ny
    xs = (x0 + np.arange(w)) % p.nx
    sel = np.ix_(ys, xs)
    nxt, mc = window_step(s, p, x0, y0, w, h, H)
    pairs = [(nxt.phi, full.phi), (nxt.Qxx, full.Qxx), (nxt.Qxy, full.Qxy),
             (nxt.f1, full.f1), (nxt.f2, full.f2), (mc["u1"], mfull["u1"]), (mc["u2"], mfull["u2"])]
    for got, want in pairs:
        want_w = want[..., ys[:, None], xs[None, :]] if want.ndim == 3 else want[sel]
        assert np.max(np.abs(interior(got, H, w, h) - want_w)) <= 1e-14
    narrow, _ = window_step(s, p, x0, y0, w, h, 4)
    assert np.max(np.abs(interior(narrow.phi, 4, w, h) - full.phi[sel])) > 1e-9


# ------------------------------------------------------------------ GPU at full size

def _origins(nx, ny, seed):
    """Window origins: both wrap seams, the grid's middle and seeded random
    positions (every 32 x 32 window spans tile seams of either geometry)."""
    rng = np.random.default_rng(seed)
    fixed = [(0, 0), (nx - WIN // 2, ny - WIN // 2), (nx // 2 - 3, ny // 2 + 5)]
    rand = [(int(rng.integers(0, nx)), int(rng.integers(0, ny))) for _ in range(3)]
    return fixed + rand


def _wrap_sel(nx, ny, x0, y0):
    ys = (y0 + np.arange(WIN)) % ny
    xs = (x0 + np.arange(WIN)) % nx
    return ys, xs


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,storage", [
    (2048, 2048, B.STORE_F32),      # the single-instance HBM workload, several waves of wide tiles
    (1040, 1000, B.STORE_F32),      # ragged tiles, rows a multiple of 4
    (1030, 1000, B.STORE_F32),      # rows not a multiple of 4 (per-element row loads)
    (1024, 1024, B.STORE_F16),      # the reduced-precision workload
    (1024, 1024, B.STORE_BF16),
], ids=["2048-f32", "1040x1000-f32", "1030x1000-f32", "1024-f16", "1024-bf16"])
def test_full_size_step_matches_oracle_windows(nx, ny, storage):
    from paper_2511_00445_gb300 import build
    build.build()
    sp = B.SolverParams(nx=nx, ny=ny, zeta=0.005, storage=storage)
    tf = B.TwoFluid(sp)
    tf.init_fields(0, phi0=0.5, dphi=0.01, S0=0.01)
    tf.step(30)
    tf.sync()
    ref = read_state(tf, 0)
    op = oracle_params(sp)
    tf.step(1)
    tf.sync()
    got = read_state(tf, 0)
    gu1, gu2 = read_velocities(tf, 0)

    # normalisers: spread of each field over the whole grid before the step
    def spr(a):
        return float(np.abs(a - a.mean()).max())
    scale = {"phi": spr(ref.phi), "Qxx": spr(ref.Qxx), "Qxy": spr(ref.Qxy)}
    for x0, y0 in _origins(nx, ny, seed=nx + ny + storage):
        ys, xs = _wrap_sel(nx, ny, x0, y0)
        sel = np.ix_(ys, xs)
        nxt, mc = window_step(ref, op, x0, y0, WIN, WIN, H)
        for name, want in (("phi", nxt.phi), ("Qxx", nxt.Qxx), ("Qxy", nxt.Qxy)):
            err = np.max(np.abs(getattr(got, name)[sel] - interior(want, H, WIN, WIN))) / scale[name]
            assert err <= TOL_1STEP, (name, x0, y0, err)
        for fam in ("f1", "f2"):
            want = interior(getattr(nxt, fam), H, WIN, WIN)
            have = getattr(got, fam)[:, ys[:, None], xs[None, :]]
            dev_want = want - want.mean(axis=(1, 2), keepdims=True)
            floor = TOL_1STEP * np.abs(dev_want).max()
            if storage == B.STORE_F32:
                assert np.max(np.abs(have - want)) <= floor, (fam, x0, y0)
            else:
                # one rounding of the stored deviation d = f - w_i after an
                # FP32 evaluation: within one unit in the last place (2 u_s |d|),
                # or half the spacing of FP16 subnormals of d * 2^12 (2^-37)
                base = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
                d = want - base
                bar = 2.0 * UNIT_ROUNDOFF[storage] * np.abs(d) + floor + 2.0**-37
                assert np.all(np.abs(have - want) <= bar), (fam, x0, y0)
        if storage == B.STORE_F32:
            uscale = max(spr(c) for c in (*gu1, *gu2))
            for g, k in ((gu1, "u1"), (gu2, "u2")):
                err = np.max(np.abs(g[:, ys[:, None], xs[None, :]] - interior(mc[k], H, WIN, WIN))) / uscale
                assert err <= TOL_1STEP, (k, x0, y0, err)
