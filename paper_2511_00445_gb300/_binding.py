"""Thin ctypes binding of libtwofluid (include/twofluid.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies the device workspace and the stream.  If the
library is missing the import of the binding raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields, replace
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TF_LIBRARY selects another build of the library (the bounds-check build
# libtwofluid_bc.so); by default the library next to this file.
LIB_PATH = os.environ.get("TF_LIBRARY") or os.path.join(HERE, "libtwofluid.so")

TF_OK = 0
TF_ERR_ARG = -1
TF_ERR_CUDA = -2
TF_ERR_NONFINITE = -3
TF_ERR_TIMEOUT = -4
TF_ERR_IO = -5
TF_ERR_WORKSPACE = -6
TF_ERR_TOO_LARGE = -7
TF_ERR_BOUNDS = -8
NOALLOC_MAX_ELEMS = 4096 * 1024

FIELD_PHI, FIELD_QXX, FIELD_QXY = 0, 1, 2
FIELD_U1X, FIELD_U1Y, FIELD_U2X, FIELD_U2Y = 3, 4, 5, 6
FIELD_RHO1, FIELD_RHO2, FIELD_MU = 7, 8, 9
FIELD_E_ELASTIC, FIELD_E_KIN, FIELD_UC_MAG, FIELD_OMEGA_C = 10, 11, 12, 13
CORR_U, CORR_OMEGA, CORR_Q = 0, 1, 2
FIELD_F1, FIELD_F2 = 16, 32
STORE_F32 = 0
STORE_F16 = 1
STORE_BF16 = 2
STORAGE_NAMES = {"f32": STORE_F32, "f16": STORE_F16, "bf16": STORE_BF16}
KERNEL_AUTO, KERNEL_TILE, KERNEL_STRIP = 0, 1, 2
KERNEL_NAMES = {"auto": KERNEL_AUTO, "tile": KERNEL_TILE, "strip": KERNEL_STRIP}
NCONS = 8

# Every symbol include/twofluid.h declares, in declaration order.
EXPORTS = [
    "tf_workspace_bytes", "tf_create", "tf_destroy", "tf_last_error", "tf_init_fields",
    "tf_write_field", "tf_set_equilibrium", "tf_read_field", "tf_step", "tf_set_step_kernel",
    "tf_step_kernel", "tf_sync",
    "tf_step_count", "tf_kernel_launches", "tf_conserved", "tf_n_shell", "tf_shell_counts", "tf_structure_factor",
    "tf_length_scale", "tf_energy_spectrum", "tf_phase_difference", "tf_phi_stats",
    "tf_correlation", "tf_snapshot", "tf_time_correlation", "tf_defects", "tf_reynolds",
    "tf_state_bytes", "tf_advance_host", "tf_save", "tf_load", "tf_plan_tiles",
    "tf_ensemble_workspace_bytes", "tf_ensemble_create", "tf_ensemble_destroy",
    "tf_ensemble_last_error", "tf_ensemble_step", "tf_ensemble_sync", "tf_ensemble_autotune",
    "tf_ensemble_config", "tf_ensemble_launches", "tf_ensemble_candidate", "tf_ensemble_select",
    "tf_ensemble_fault_drill",
    "tf_sur_workspace_bytes", "tf_sur_create", "tf_sur_destroy", "tf_sur_last_error",
    "tf_sur_num_params", "tf_sur_init_weights", "tf_sur_set_weights", "tf_sur_get_weights",
    "tf_sur_forward", "tf_sur_gradients", "tf_sur_add_pair", "tf_sur_fit_normalisation",
    "tf_sur_train", "tf_sur_predict", "tf_sur_judged_predict", "tf_phi_stats_noalloc",
]
SUR_IN, SUR_OUT = 8, 7


class TFSurConfig(ctypes.Structure):
    """Mirror of struct tf_sur_config."""
    _fields_ = [("levels", ctypes.c_int), ("base_channels", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_pairs", ctypes.c_int),
                ("horizon", ctypes.c_int)]
ENS_CANDIDATES = 9
ENS_PERSISTENT_CANDIDATES = 6     # candidates 0..5: one persistent launch; 6, 7: a launch per step
ENS_GROUP_PLANS = 8               # candidate 8: each group's own per-context launches


class TFParams(ctypes.Structure):
    """Mirror of struct tf_params."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n_sub", ctypes.c_int),
                ("storage", ctypes.c_int),
                ("tau1", ctypes.c_double), ("tau2", ctypes.c_double),
                ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
                ("gamma", ctypes.c_double), ("zeta", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("K", ctypes.c_double),
                ("Gamma_Q", ctypes.c_double), ("A_Q", ctypes.c_double), ("C_Q", ctypes.c_double),
                ("M", ctypes.c_double), ("A_ch", ctypes.c_double), ("kappa", ctypes.c_double),
                ("phi_ref", ctypes.c_double), ("dt", ctypes.c_double),
                ("check_every", ctypes.c_int)]


@dataclass(frozen=True)
class SolverParams:
    """Per-instance parameters (lattice units); defaults are the 64x64
    correctness configuration (zeta 0.005, lambda 0.7, K 0.04, drag 0.01,
    tau 1) with the Sec. III constants M 0.2, A 0.05, kappa 0.1, Gamma_Q 0.2, and
    Landau-de Gennes A_Q -0.1, C_Q 0.4 (bulk order 1/2)."""
    nx: int = 64
    ny: int = 64
    n_sub: int = 5
    storage: int = STORE_F32
    tau1: float = 1.0
    tau2: float = 1.0
    rho1: float = 1.0
    rho2: float = 1.0
    gamma: float = 0.01
    zeta: float = 0.005
    lam: float = 0.7
    K: float = 0.04
    Gamma_Q: float = 0.2
    A_Q: float = -0.1
    C_Q: float = 0.4
    M: float = 0.2
    A_ch: float = 0.05
    kappa: float = 0.1
    phi_ref: float = 0.5
    dt: float = 1.0          # FD sub-step = dt / n_sub (1: lattice units)
    check_every: int = 0     # non-finite scan every k steps (0: off)

    def with_(self, **kw) -> "SolverParams":
        return replace(self, **kw)

    def to_c(self) -> TFParams:
        kw = {f.name: getattr(self, f.name) for f in fields(self)}
        kw["lambda_"] = kw.pop("lam")
        return TFParams(**kw)


class TwoFluidError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libtwofluid error {code}: {msg}")
        self.code = code


_lib = None


def load_library() -> ctypes.CDLL:
    """Load libtwofluid.so (built by paper_2511_00445_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2511_00445_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, i64, d, dp, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_size_t)
    P = ctypes.POINTER(TFParams)
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "tf_workspace_bytes": (sz, [P, i]),
        "tf_create": (i, [P, i, vp, sz, vp, ctypes.POINTER(vp)]),
        "tf_destroy": (i, [vp]),
        "tf_last_error": (ctypes.c_char_p, [vp]),
        "tf_init_fields": (i, [vp, i, ctypes.c_uint64, d, d, d]),
        "tf_write_field": (i, [vp, i, i, dp]),
        "tf_set_equilibrium": (i, [vp, i, dp, dp]),
        "tf_read_field": (i, [vp, i, i, dp]),
        "tf_step": (i, [vp, i64]),
        "tf_set_step_kernel": (i, [vp, i]),
        "tf_step_kernel": (i, [vp]),
        "tf_sync": (i, [vp]),
        "tf_step_count": (i64, [vp]),
        "tf_kernel_launches": (i64, [vp]),
        "tf_conserved": (i, [vp, i, dp]),
        "tf_n_shell": (i, [vp]),
        "tf_shell_counts": (i, [vp, dp, i]),
        "tf_structure_factor": (i, [vp, i, dp, i]),
        "tf_length_scale": (i, [vp, i, dp]),
        "tf_energy_spectrum": (i, [vp, i, dp, i, dp]),
        "tf_phase_difference": (i, [vp, i, dp]),
        "tf_phi_stats": (i, [vp, i, dp, dp]),
        "tf_correlation": (i, [vp, i, i, dp, i]),
        "tf_snapshot": (i, [vp, i]),
        "tf_time_correlation": (i, [vp, i, dp]),
        "tf_defects": (i, [vp, i, ctypes.POINTER(ctypes.c_int64)]),
        "tf_reynolds": (i, [vp, i, dp, dp]),
        "tf_state_bytes": (sz, [vp]),
        "tf_advance_host": (i, [vp, vp, i64, vp]),
        "tf_save": (i, [vp, ctypes.c_char_p]),
        "tf_load": (i, [vp, ctypes.c_char_p]),
        "tf_plan_tiles": (i, [i, i, i, ctypes.c_longlong, ctypes.POINTER(i), ctypes.POINTER(i), i]),
        "tf_ensemble_workspace_bytes": (sz, [i]),
        "tf_ensemble_create": (i, [ctypes.POINTER(vp), i, vp, sz, vp, ctypes.POINTER(vp)]),
        "tf_ensemble_destroy": (i, [vp]),
        "tf_ensemble_last_error": (ctypes.c_char_p, [vp]),
        "tf_ensemble_step": (i, [vp, i64]),
        "tf_ensemble_sync": (i, [vp]),
        "tf_ensemble_autotune": (i, [vp, i]),
        "tf_ensemble_config": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                   ctypes.POINTER(i64), dp, ctypes.POINTER(i)]),
        "tf_ensemble_launches": (i64, [vp]),
        "tf_ensemble_candidate": (i, [vp]),
        "tf_ensemble_select": (i, [vp, i]),
        "tf_ensemble_fault_drill": (i, [vp, ctypes.c_uint32, i]),
        "tf_sur_workspace_bytes": (sz, [ctypes.POINTER(TFSurConfig)]),
        "tf_sur_create": (i, [ctypes.POINTER(TFSurConfig), vp, sz, vp, ctypes.POINTER(vp)]),
        "tf_sur_destroy": (i, [vp]),
        "tf_sur_last_error": (ctypes.c_char_p, [vp]),
        "tf_sur_num_params": (i64, [vp]),
        "tf_sur_init_weights": (i, [vp, ctypes.c_uint64]),
        "tf_sur_set_weights": (i, [vp, fp, i64]),
        "tf_sur_get_weights": (i, [vp, fp, i64]),
        "tf_sur_forward": (i, [vp, fp, i, fp]),
        "tf_sur_gradients": (i, [vp, fp, fp, i, dp, fp, i64]),
        "tf_sur_add_pair": (i, [vp, i, vp, i, i]),
        "tf_sur_fit_normalisation": (i, [vp, i]),
        "tf_sur_train": (i, [vp, i, i, i, d, ctypes.c_uint64, dp]),
        "tf_sur_predict": (i, [vp, vp, i]),
        "tf_sur_judged_predict": (i, [vp, vp, vp, i, d, d, dp, ctypes.POINTER(i)]),
        "tf_phi_stats_noalloc": (i, [vp, ctypes.c_longlong, d, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class TwoFluid:
    """A batch of same-size instances on one GPU, behind the C ABI.

    Method names follow the C entry points without their ``tf_`` prefix.
    """

    def __init__(self, params: SolverParams | Sequence[SolverParams], device="cuda", stream=None):
        import torch
        self.lib = load_library()
        plist = [params] if isinstance(params, SolverParams) else list(params)
        self.params = plist
        self.batch = len(plist)
        self.nx, self.ny = plist[0].nx, plist[0].ny
        arr = (TFParams * self.batch)(*[p.to_c() for p in plist])
        self._carr = arr
        nbytes = self.lib.tf_workspace_bytes(arr, self.batch)
        if nbytes == 0:
            raise TwoFluidError(TF_ERR_ARG, "invalid parameters")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        rc = self.lib.tf_create(arr, self.batch, ctypes.c_void_p(aligned), nbytes,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if rc != TF_OK:
            raise TwoFluidError(rc, "tf_create failed")
        self.ctx = ctx
        self.workspace_bytes = nbytes

    # -- helpers
    def _check(self, rc: int):
        if rc != TF_OK:
            raise TwoFluidError(rc, self.lib.tf_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def init_fields(self, seed: int, phi0: float = 0.5, dphi: float = 0.01, S0: float = 0.01,
                    inst: int = -1):
        self._check(self.lib.tf_init_fields(self.ctx, inst, seed, phi0, dphi, S0))

    def write_field(self, inst: int, field: int, values: np.ndarray):
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(self.ny, self.nx)
        self._check(self.lib.tf_write_field(self.ctx, inst, field, _dptr(a)))

    def set_equilibrium(self, inst: int, u1: np.ndarray | None = None, u2: np.ndarray | None = None):
        def conv(u):
            if u is None:
                return None, None
            a = np.ascontiguousarray(u, dtype=np.float64).reshape(2, self.ny, self.nx)
            return a, _dptr(a)
        a1, p1 = conv(u1)
        a2, p2 = conv(u2)
        self._check(self.lib.tf_set_equilibrium(self.ctx, inst, p1, p2))
        del a1, a2

    def read_field(self, inst: int, field: int) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.float64)
        self._check(self.lib.tf_read_field(self.ctx, inst, field, _dptr(out)))
        return out

    def step(self, n: int = 1):
        self._check(self.lib.tf_step(self.ctx, n))

    def sync(self):
        self._check(self.lib.tf_sync(self.ctx))

    def set_step_kernel(self, kind):
        """kind: KERNEL_AUTO / KERNEL_TILE / KERNEL_STRIP or 'auto' / 'tile' / 'strip'."""
        self._check(self.lib.tf_set_step_kernel(self.ctx, KERNEL_NAMES.get(kind, kind)))

    def step_kernel(self) -> int:
        rc = self.lib.tf_step_kernel(self.ctx)
        if rc < 0:
            self._check(rc)
        return rc

    def step_count(self) -> int:
        return int(self.lib.tf_step_count(self.ctx))

    def kernel_launches(self) -> int:
        return int(self.lib.tf_kernel_launches(self.ctx))

    # -- observables
    def conserved(self, inst: int, check: bool = True) -> np.ndarray:
        out = np.empty(NCONS)
        rc = self.lib.tf_conserved(self.ctx, inst, _dptr(out))
        if check or rc != TF_ERR_NONFINITE:
            self._check(rc)
        return out

    def n_shell(self) -> int:
        return int(self.lib.tf_n_shell(self.ctx))

    def shell_counts(self) -> np.ndarray:
        out = np.empty(self.n_shell())
        self._check(self.lib.tf_shell_counts(self.ctx, _dptr(out), out.size))
        return out

    def structure_factor(self, inst: int) -> np.ndarray:
        out = np.empty(self.n_shell())
        self._check(self.lib.tf_structure_factor(self.ctx, inst, _dptr(out), out.size))
        return out

    def length_scale(self, inst: int) -> float:
        out = ctypes.c_double()
        self._check(self.lib.tf_length_scale(self.ctx, inst, ctypes.byref(out)))
        return out.value

    def energy_spectrum(self, inst: int):
        out = np.empty(self.n_shell())
        tot = ctypes.c_double()
        self._check(self.lib.tf_energy_spectrum(self.ctx, inst, _dptr(out), out.size,
                                                ctypes.byref(tot)))
        return out, tot.value

    def phase_difference(self, inst: int) -> np.ndarray:
        out = np.empty(6)
        self._check(self.lib.tf_phase_difference(self.ctx, inst, _dptr(out)))
        return out

    def phi_stats(self, inst: int):
        m, s = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.tf_phi_stats(self.ctx, inst, ctypes.byref(m), ctypes.byref(s)))
        return m.value, s.value

    def correlation(self, inst: int, which: int) -> np.ndarray:
        out = np.empty(self.n_shell())
        self._check(self.lib.tf_correlation(self.ctx, inst, which, _dptr(out), out.size))
        return out

    def snapshot(self, inst: int):
        self._check(self.lib.tf_snapshot(self.ctx, inst))

    def time_correlation(self, inst: int) -> np.ndarray:
        out = np.empty(3)
        self._check(self.lib.tf_time_correlation(self.ctx, inst, _dptr(out)))
        return out

    def defects(self, inst: int) -> np.ndarray:
        out = np.zeros(3, dtype=np.int64)
        self._check(self.lib.tf_defects(self.ctx, inst,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return out

    def reynolds(self, inst: int):
        re, la = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.tf_reynolds(self.ctx, inst, ctypes.byref(re), ctypes.byref(la)))
        return re.value, la.value

    # -- raw state, end-to-end, checkpoints
    def state_bytes(self) -> int:
        return int(self.lib.tf_state_bytes(self.ctx))

    def advance_host(self, h_in_ptr: int | None, n: int, h_out_ptr: int | None):
        self._check(self.lib.tf_advance_host(self.ctx, h_in_ptr, n, h_out_ptr))

    def save(self, path: str):
        self._check(self.lib.tf_save(self.ctx, path.encode()))

    def load(self, path: str):
        self._check(self.lib.tf_load(self.ctx, path.encode()))


class Ensemble:
    """Several TwoFluid groups (each one grid size) stepped by one persistent
    launch per call, behind the tf_ensemble_* entry points.  The groups keep
    their own state and observables; they must share the ensemble's stream
    and must not be stepped on their own while the ensemble exists."""

    def __init__(self, groups: Sequence[TwoFluid]):
        import torch
        self.lib = load_library()
        self.groups = list(groups)
        n = len(self.groups)
        nbytes = self.lib.tf_ensemble_workspace_bytes(n)
        if nbytes == 0:
            raise TwoFluidError(TF_ERR_ARG, "bad group count")
        self.stream = self.groups[0].stream
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.groups[0].device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        arr = (ctypes.c_void_p * n)(*[g.ctx.value for g in self.groups])
        ens = ctypes.c_void_p()
        rc = self.lib.tf_ensemble_create(arr, n, ctypes.c_void_p(aligned), nbytes,
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ens))
        if rc != TF_OK:
            raise TwoFluidError(rc, "tf_ensemble_create failed")
        self.ens = ens

    def _check(self, rc: int):
        if rc != TF_OK:
            raise TwoFluidError(rc, self.lib.tf_ensemble_last_error(self.ens).decode())

    def close(self):
        if getattr(self, "ens", None):
            self.lib.tf_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._check(self.lib.tf_ensemble_step(self.ens, n))

    def sync(self):
        self._check(self.lib.tf_ensemble_sync(self.ens))

    def autotune(self, steps_per_candidate: int = 4):
        self._check(self.lib.tf_ensemble_autotune(self.ens, steps_per_candidate))

    def config(self) -> dict:
        ty, cps, grid, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        tiles = ctypes.c_int64()
        us = np.zeros(ENS_CANDIDATES)
        self._check(self.lib.tf_ensemble_config(self.ens, ctypes.byref(ty), ctypes.byref(cps),
                                                ctypes.byref(grid), ctypes.byref(tiles), _dptr(us),
                                                ctypes.byref(gr)))
        cand = self.candidate()
        return {"candidate": cand, "persistent": cand < ENS_PERSISTENT_CANDIDATES,
                "group_plans": cand == ENS_GROUP_PLANS,
                "tile_y": ty.value, "ctas_per_sm": cps.value, "grid": grid.value,
                "tiles_per_step": tiles.value, "us_per_step": us.tolist(), "graphs": bool(gr.value),
                "note": self.lib.tf_ensemble_last_error(self.ens).decode()}

    def launches(self) -> int:
        return int(self.lib.tf_ensemble_launches(self.ens))

    def candidate(self) -> int:
        return int(self.lib.tf_ensemble_candidate(self.ens))

    def select(self, candidate: int):
        self._check(self.lib.tf_ensemble_select(self.ens, candidate))

    def fault_drill(self, barrier_polls: int = 0, held_cta: int = -1):
        self._check(self.lib.tf_ensemble_fault_drill(self.ens, barrier_polls, held_cta))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Surrogate:
    """The U-Net surrogate behind the tf_sur_* entry points (see twofluid.h).
    Arrays are NHWC float32 numpy arrays; the workspace lives in torch memory."""

    def __init__(self, levels=4, base_channels=32, nx=256, ny=256, max_batch=8, max_pairs=64,
                 horizon=50, device="cuda", stream=None):
        import torch
        self.lib = load_library()
        self.cfg = TFSurConfig(levels, base_channels, nx, ny, max_batch, max_pairs, horizon)
        nbytes = self.lib.tf_sur_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise TwoFluidError(TF_ERR_ARG, "invalid surrogate configuration")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.tf_sur_create(ctypes.byref(self.cfg), ctypes.c_void_p(aligned), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != TF_OK:
            raise TwoFluidError(rc, "tf_sur_create failed")
        self.h = h
        self.n_params = int(self.lib.tf_sur_num_params(h))

    def _check(self, rc: int):
        if rc != TF_OK:
            raise TwoFluidError(rc, self.lib.tf_sur_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tf_sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_weights(self, seed: int):
        self._check(self.lib.tf_sur_init_weights(self.h, seed))

    def set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.lib.tf_sur_set_weights(self.h, _fptr(w), w.size))

    def get_weights(self) -> np.ndarray:
        w = np.empty(self.n_params, dtype=np.float32)
        self._check(self.lib.tf_sur_get_weights(self.h, _fptr(w), w.size))
        return w

    def forward(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty(x.shape[:3] + (SUR_OUT,), dtype=np.float32)
        self._check(self.lib.tf_sur_forward(self.h, _fptr(x), x.shape[0], _fptr(out)))
        return out

    def gradients(self, x: np.ndarray, target: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.tf_sur_gradients(self.h, _fptr(x), _fptr(t), x.shape[0],
                                              ctypes.byref(loss), _fptr(g), g.size))
        return loss.value, g

    def add_pair(self, slot: int, solver: TwoFluid, inst: int, which: int):
        self._check(self.lib.tf_sur_add_pair(self.h, slot, solver.ctx, inst, which))

    def fit_normalisation(self, n_pairs: int):
        self._check(self.lib.tf_sur_fit_normalisation(self.h, n_pairs))

    def train(self, n_pairs: int, steps: int, batch: int, lr: float, seed: int = 0) -> np.ndarray:
        losses = np.zeros(steps)
        self._check(self.lib.tf_sur_train(self.h, n_pairs, steps, batch, lr, seed, _dptr(losses)))
        return losses

    def predict(self, solver: TwoFluid, inst: int):
        self._check(self.lib.tf_sur_predict(self.h, solver.ctx, inst))

    def judged_predict(self, solver: TwoFluid, shadow: TwoFluid, inst: int, max_err_L: float,
                       max_err_E: float):
        out = np.zeros(4)
        back = ctypes.c_int()
        self._check(self.lib.tf_sur_judged_predict(self.h, solver.ctx, shadow.ctx, inst, max_err_L,
                                                   max_err_E, _dptr(out), ctypes.byref(back)))
        return out, bool(back.value)
