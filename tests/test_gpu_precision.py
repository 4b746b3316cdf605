"""16-bit population storage (TF_STORE_F16, TF_STORE_BF16) on the GPU.

The stored value is the deviation d_i = f_i - w_i rounded to the storage
type (FP16 of d_i * 2^12, or BF16 of d_i); every arithmetic operation stays
FP32.  The rounding itself is checked bit for bit against a numpy
restatement of IEEE round-to-nearest-even; the trajectory is checked
against the FP64 oracle with a tolerance that follows from the storage's
unit roundoff u_s: each step rounds every stored deviation once, with
independent signs, so after n steps the relative error of a field grows
like a random walk, sqrt(n) * u_s.
"""
import math

import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B

from helpers import field_errors, oracle_params, read_state

pytestmark = pytest.mark.gpu

CFG0 = B.SolverParams()
UNIT_ROUNDOFF = {B.STORE_F16: 2.0**-11, B.STORE_BF16: 2.0**-8}
MODES = [pytest.param(B.STORE_F16, id="f16"), pytest.param(B.STORE_BF16, id="bf16")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_00445_gb300 import build
    build.build()


def make(params, seed=0):
    tf = B.TwoFluid(params)
    tf.init_fields(seed, phi0=0.5, dphi=0.01, S0=0.01)
    tf.sync()
    return tf


def quantise(d32: np.ndarray, mode: int) -> np.ndarray:
    """FP32 deviations -> the FP32 value the device widens the stored
    16-bit value back to (round to nearest, ties to even)."""
    d32 = np.asarray(d32, np.float32)
    if mode == B.STORE_F16:
        return (d32 * np.float32(4096.0)).astype(np.float16).astype(np.float32) / np.float32(4096.0)
    u = d32.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16      # finite inputs only
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("mode", MODES)
def test_storage_rounding_is_round_to_nearest_even(mode):
    """Population writes round FP32 deviations exactly as IEEE RNE into the
    storage type; reads widen them exactly (w_i added back in FP64)."""
    nx, ny = 24, 16
    tf = make(CFG0.with_(nx=nx, ny=ny, storage=mode))
    rng = np.random.default_rng(11)
    mag = 10.0 ** rng.uniform(-9, 0, size=(ny, nx))          # spans FP16's subnormal range
    for i in (0, 3, 7):
        d = (mag * rng.choice([-1.0, 1.0], size=(ny, nx))).astype(np.float64)
        f = O.WI[i] + d
        tf.write_field(0, B.FIELD_F1 + i, f)
        d32 = (f - O.WI[i]).astype(np.float32)                # the device rounds f - w_i to FP32 first
        want = O.WI[i] + quantise(d32, mode).astype(np.float64)
        assert np.array_equal(tf.read_field(0, B.FIELD_F1 + i), want)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny,steps,zeta,n_sub", [(64, 64, 200, 0.005, 5), (33, 17, 200, 0.005, 5),
                                                    (48, 40, 200, 0.01, 5), (16, 16, 100, 0.005, 3)])
def test_storage_parity_against_oracle(mode, nx, ny, steps, zeta, n_sub):
    """Fused path (n_sub = 5, widths with and without 16-byte row alignment)
    and per-stage path (n_sub = 3) within sqrt(n) * u_s of the FP64 oracle."""
    p = CFG0.with_(nx=nx, ny=ny, zeta=zeta, n_sub=n_sub, storage=mode)
    tf = make(p)
    op = oracle_params(p)
    ref = O.run(read_state(tf, 0), op, steps)
    tf.step(steps)
    errs = field_errors(tf, 0, ref, op)
    tol = math.sqrt(steps) * UNIT_ROUNDOFF[mode]
    # the rounding-model bar is taken on the shared velocity scale at every size
    for k in ("phi", "Qxx", "Qxy", "u1", "u2"):
        assert errs[k] <= tol, (k, errs[k], tol, errs)


@pytest.mark.parametrize("mode", MODES)
def test_storage_phi_mass_unaffected(mode):
    """phi stays FP32: its sum is conserved to FP32 rounding whatever the
    population storage (Cahn-Hilliard flux form, Eq. 1)."""
    tf = make(CFG0.with_(nx=40, ny=36, storage=mode))
    s0 = tf.conserved(0)[0]
    tf.step(300)
    s1 = tf.conserved(0)[0]
    assert abs(s1 - s0) <= 1e-9 * 40 * 36


@pytest.mark.parametrize("mode", MODES)
def test_storage_interleaved_reads_do_not_change_trajectory(mode):
    """Reads complete the pending sub-steps bitwise as the steady-state
    kernel does, in every storage mode."""
    p = CFG0.with_(nx=40, ny=36, zeta=0.01, storage=mode)
    a, b = make(p, seed=3), make(p, seed=3)
    for n in (1, 2, 3, 4):
        a.step(n)
        a.read_field(0, B.FIELD_PHI)
    b.step(10)
    for fld in (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_F1 + 5, B.FIELD_F2 + 2, B.FIELD_U1X):
        assert np.array_equal(a.read_field(0, fld), b.read_field(0, fld)), fld


@pytest.mark.parametrize("mode", MODES)
def test_storage_checkpoint_and_state_size(mode, tmp_path):
    """The raw state holds 2-byte populations; save/load is bitwise."""
    nx, ny = 32, 24
    p = CFG0.with_(nx=nx, ny=ny, storage=mode)
    tf = make(p)
    tf.step(7)
    assert tf.state_bytes() == 18 * nx * ny * 2 + 3 * nx * ny * 4
    path = str(tmp_path / "s.ckpt")
    tf.save(path)
    want = [tf.read_field(0, f) for f in (B.FIELD_PHI, B.FIELD_F1 + 1, B.FIELD_F2 + 8)]
    tf.step(5)
    tf.load(path)
    got = [tf.read_field(0, f) for f in (B.FIELD_PHI, B.FIELD_F1 + 1, B.FIELD_F2 + 8)]
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
