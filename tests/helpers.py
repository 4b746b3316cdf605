"""Shared test helpers: GPU <-> oracle state transfer and the parity metric."""
import numpy as np

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B

# Parity bar after 200 steps in FP32: max |X_gpu - X_oracle| normalised by the
# oracle field's own spread max |X - <X>| (pointwise relative error of fields
# that sit near a constant, phi ~ 1/2, u ~ 0, is ill-posed).  Velocities are
# reported both against their own spread ("u1_own", "u2_own") and against the
# shared scale of the flow, the larger spread of u1 and u2 ("u1", "u2").  On
# grids below 32 x 32 u2 can be ~100x smaller than u1, and a float32
# restatement of the step (tests/fp32_restatement.py, checked in
# tests/test_fp32_floor.py) already departs from the FP64 oracle by more than
# 1e-5 of u2's own spread there; from 32 x 32 up every field, u2 included, is
# held to its own spread.
TOL_200 = 1e-5
OWN_SPREAD_MIN = 32     # grids with nx, ny >= this use the own-spread bars


def oracle_params(sp: B.SolverParams) -> O.Params:
    return O.Params(nx=sp.nx, ny=sp.ny, tau1=sp.tau1, tau2=sp.tau2, rho1=sp.rho1, rho2=sp.rho2,
                    gamma=sp.gamma, zeta=sp.zeta, lam=sp.lam, K=sp.K, Gamma_Q=sp.Gamma_Q,
                    A_Q=sp.A_Q, C_Q=sp.C_Q, M=sp.M, A_ch=sp.A_ch, kappa=sp.kappa, n_sub=sp.n_sub,
                    dt=getattr(sp, "dt", 1.0))


def read_state(tf: B.TwoFluid, inst: int) -> O.State:
    """The GPU's current state as an oracle State (exact FP32 values in FP64)."""
    f1 = np.stack([tf.read_field(inst, B.FIELD_F1 + i) for i in range(9)])
    f2 = np.stack([tf.read_field(inst, B.FIELD_F2 + i) for i in range(9)])
    return O.State(f1, f2, tf.read_field(inst, B.FIELD_PHI), tf.read_field(inst, B.FIELD_QXX),
                   tf.read_field(inst, B.FIELD_QXY))


def read_velocities(tf: B.TwoFluid, inst: int):
    u1 = np.stack([tf.read_field(inst, B.FIELD_U1X), tf.read_field(inst, B.FIELD_U1Y)])
    u2 = np.stack([tf.read_field(inst, B.FIELD_U2X), tf.read_field(inst, B.FIELD_U2Y)])
    return u1, u2


def rel_err(got: np.ndarray, want: np.ndarray) -> float:
    """max |got - want| / max |want - <want>|; a field with no spread (a
    single site, a uniform state) is normalised by its magnitude instead."""
    spread = np.abs(want - want.mean()).max()
    if spread == 0.0:
        spread = np.abs(want).max()
    diff = np.abs(got - want).max()
    if spread == 0.0:
        return 0.0 if diff == 0.0 else float("inf")
    return float(diff / spread)


def spread(x: np.ndarray) -> float:
    return float(np.abs(x - x.mean()).max())


def field_errors(tf: B.TwoFluid, inst: int, ref: O.State, p: O.Params) -> dict:
    mc = O.macro(ref, p)
    u1, u2 = read_velocities(tf, inst)
    uscale = max(spread(c) for c in (*mc["u1"], *mc["u2"]))
    if uscale == 0.0:
        uscale = max(float(np.abs(mc["u1"]).max()), float(np.abs(mc["u2"]).max()))

    def uerr(got, want):
        d = float(np.abs(got - want).max())
        return d / uscale if uscale > 0 else (0.0 if d == 0.0 else float("inf"))
    return {
        "phi": rel_err(tf.read_field(inst, B.FIELD_PHI), ref.phi),
        "Qxx": rel_err(tf.read_field(inst, B.FIELD_QXX), ref.Qxx),
        "Qxy": rel_err(tf.read_field(inst, B.FIELD_QXY), ref.Qxy),
        "u1": max(uerr(u1[0], mc["u1"][0]), uerr(u1[1], mc["u1"][1])),
        "u2": max(uerr(u2[0], mc["u2"][0]), uerr(u2[1], mc["u2"][1])),
        "u1_own": max(rel_err(u1[0], mc["u1"][0]), rel_err(u1[1], mc["u1"][1])),
        "u2_own": max(rel_err(u2[0], mc["u2"][0]), rel_err(u2[1], mc["u2"][1])),
    }


def assert_parity(err: dict, nx: int, ny: int, tol: float = TOL_200):
    """The 200-step bar: phi, Q and the shared-scale velocities always; the
    velocities' own spreads as well on grids of at least OWN_SPREAD_MIN."""
    keys = ["phi", "Qxx", "Qxy", "u1", "u2"]
    if nx >= OWN_SPREAD_MIN and ny >= OWN_SPREAD_MIN:
        keys += ["u1_own", "u2_own"]
    for k in keys:
        assert err[k] < tol, (k, err)


# ------------------------------------------------ oracle on windows of a grid
def cut(state: O.State, x0: int, y0: int, w: int, h: int, margin: int) -> O.State:
    """Window [y0 - margin, y0 + h + margin) x [x0 - margin, x0 + w + margin)
    of a periodic state, indices taken modulo the grid."""
    ny, nx = state.phi.shape
    ys = (y0 - margin + np.arange(h + 2 * margin)) % ny
    xs = (x0 - margin + np.arange(w + 2 * margin)) % nx
    sel = np.ix_(ys, xs)
    return O.State(state.f1[:, ys[:, None], xs[None, :]].copy(),
                   state.f2[:, ys[:, None], xs[None, :]].copy(),
                   state.phi[sel].copy(), state.Qxx[sel].copy(), state.Qxy[sel].copy())


def interior(a: np.ndarray, margin: int, w: int, h: int) -> np.ndarray:
    return a[..., margin:margin + h, margin:margin + w]


def window_step(state: O.State, p: O.Params, x0: int, y0: int, w: int, h: int, margin: int):
    """One oracle step of a window (margin on each side); returns the stepped
    window state and its macroscopic fields."""
    win = cut(state, x0, y0, w, h, margin)
    pw = p.with_(nx=w + 2 * margin, ny=h + 2 * margin)
    nxt = O.step(win, pw)
    return nxt, O.macro(nxt, pw)
