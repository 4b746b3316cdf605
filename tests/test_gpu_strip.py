"""The strip-streaming steady-state kernel against the tile kernel and the oracle.

Both kernels evaluate every site with the same correctly rounded FP32
operations in the same order, so a context stepped with the strip kernel must
hold bitwise the same populations, fields and velocities as one stepped with
the tile kernel; the tile kernel is itself held to the FP64 oracle
(test_gpu_parity.py), and the strip kernel is checked against the oracle here
too.  Cases cover several strips with a ragged last one, segments shorter than
the sub-step halo, grids narrower than the 120-column window (several periodic
wraps in one window row), batches with per-instance parameters and 16-bit
population storage.
"""
import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B

from helpers import assert_parity, field_errors, oracle_params, read_state

pytestmark = pytest.mark.gpu

CFG0 = B.SolverParams()
FIELDS = ([B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_U1X, B.FIELD_U1Y, B.FIELD_U2X,
           B.FIELD_U2Y] + [B.FIELD_F1 + i for i in range(9)] + [B.FIELD_F2 + i for i in range(9)])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_00445_gb300 import build
    build.build()


def make(params, kernel, seed=0, dphi=0.01, S0=0.01):
    tf = B.TwoFluid(params)
    tf.set_step_kernel(kernel)
    tf.init_fields(seed, phi0=0.5, dphi=dphi, S0=S0)
    return tf


def assert_same(a, b, batch):
    for inst in range(batch):
        for fld in FIELDS:
            x, y = a.read_field(inst, fld), b.read_field(inst, fld)
            assert np.array_equal(x, y), (inst, fld, float(np.abs(x - y).max()))


@pytest.mark.parametrize("nx,ny,steps", [(64, 64, 40), (96, 40, 30), (100, 36, 30), (196, 200, 25),
                                         (8, 8, 30), (4, 12, 20), (20, 3, 20), (292, 100, 12)])
def test_strip_bitwise_equals_tile(nx, ny, steps):
    p = CFG0.with_(nx=nx, ny=ny, zeta=0.01)
    a = make(p, "tile", seed=5, dphi=0.05, S0=0.2)
    b = make(p, "strip", seed=5, dphi=0.05, S0=0.2)
    assert a.step_kernel() == B.KERNEL_TILE and b.step_kernel() == B.KERNEL_STRIP
    a.step(steps)
    b.step(steps)
    assert_same(a, b, 1)


def test_strip_bitwise_batch_interleaved_and_storage():
    """A batch of three instances with their own parameters, reads between
    steps (each read completes the pending sub-steps with the FD-only
    epilogue, then the next step starts with the LBM-only prologue)."""
    ps = [CFG0.with_(nx=128, ny=72, zeta=z, lam=l, K=k) for z, l, k in
          ((0.0, 0.3, 0.02), (0.005, 0.7, 0.04), (0.01, 1.1, 0.08))]
    a = make(ps, "tile", seed=9, dphi=0.03, S0=0.1)
    b = make(ps, "strip", seed=9, dphi=0.03, S0=0.1)
    for n in (3, 1, 7):
        a.step(n)
        b.step(n)
        a.read_field(1, B.FIELD_PHI)
        b.read_field(1, B.FIELD_PHI)
    assert_same(a, b, 3)


@pytest.mark.parametrize("storage", [B.STORE_F16, B.STORE_BF16])
def test_strip_bitwise_16bit_storage(storage):
    p = CFG0.with_(nx=136, ny=48, zeta=0.01, storage=storage)
    a = make(p, "tile", seed=3, dphi=0.05, S0=0.2)
    b = make(p, "strip", seed=3, dphi=0.05, S0=0.2)
    a.step(20)
    b.step(20)
    assert_same(a, b, 1)


@pytest.mark.parametrize("nx,ny", [(64, 64), (36, 52)])
def test_strip_parity_against_oracle(nx, ny):
    """200 steps of the correctness configuration with the strip kernel forced."""
    p = CFG0.with_(nx=nx, ny=ny)
    tf = make(p, "strip")
    op = oracle_params(p)
    ref = O.run(read_state(tf, 0), op, 200)
    tf.step(200)
    assert_parity(field_errors(tf, 0, ref, op), nx, ny)


def test_kernel_selection():
    """AUTO takes the strip kernel where its plan fills a wave of resident
    CTAs (2048^2, 1024^2, 4 x 512^2) and the tiles where it would leave SMs
    idle (768^2: 192 strip CTAs; 512^2; the 4 x 256^2 sweep) or cannot run."""
    for n, b in ((2048, 1), (1024, 1), (512, 4)):
        t = B.TwoFluid([CFG0.with_(nx=n, ny=n)] * b)
        assert t.step_kernel() == B.KERNEL_STRIP, (n, b)
        t.close()
    for n, b in ((768, 1), (512, 1), (256, 4)):
        t = B.TwoFluid([CFG0.with_(nx=n, ny=n)] * b)
        assert t.step_kernel() == B.KERNEL_TILE, (n, b)
        t.close()
    big = B.TwoFluid(CFG0.with_(nx=1024, ny=1024))
    big.set_step_kernel("tile")
    assert big.step_kernel() == B.KERNEL_TILE
    big.set_step_kernel("strip")
    assert big.step_kernel() == B.KERNEL_STRIP
    small = B.TwoFluid(CFG0.with_(nx=64, ny=64))
    assert small.step_kernel() == B.KERNEL_TILE
    odd = B.TwoFluid(CFG0.with_(nx=1026, ny=1024))      # rows not 16-byte multiples
    assert odd.step_kernel() == B.KERNEL_TILE
    with pytest.raises(B.TwoFluidError):
        odd.set_step_kernel("strip")
    for t in (big, small, odd):
        t.close()
