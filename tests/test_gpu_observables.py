"""Correlations, defects, energy-density maps and the Reynolds number (Sec. IV)
on the GPU against the FP64 oracle evaluated on the same (read-back) state.

The GPU evaluates the velocities u1, u2 of a state in FP32 (as the step does)
and everything after that in FP64; the oracle evaluates the whole chain in
FP64.  Quantities built from velocities therefore agree to FP32 rounding of
u (tolerances below are a few 1e-6 of the field's own scale); defect counts
are integers decided exactly on both sides and must be equal.
"""
import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B

from helpers import oracle_params, read_state

pytestmark = pytest.mark.gpu

CFG0 = B.SolverParams()


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_00445_gb300 import build
    build.build()


def developed(nx, ny, steps, zeta=0.01, seed=0, **kw):
    p = CFG0.with_(nx=nx, ny=ny, zeta=zeta, **kw)
    tf = B.TwoFluid(p)
    tf.init_fields(seed, phi0=0.5, dphi=0.01, S0=0.3)
    tf.step(steps)
    tf.sync()
    return tf, p


def scaled_err(got, want):
    scale = max(float(np.abs(want).max()), 1e-300)
    return float(np.abs(got - want).max()) / scale


@pytest.mark.parametrize("nx,ny", [(64, 48), (40, 36)])
def test_energy_and_flow_maps(nx, ny):
    tf, p = developed(nx, ny, 150)
    st, op = read_state(tf, 0), oracle_params(p)
    mc = O.macro(st, op)
    uc = O.mixture_velocity(st.phi, mc["u1"], mc["u2"])
    want = {
        B.FIELD_E_ELASTIC: O.elastic_energy_density(st.Qxx, st.Qxy, p.K),
        B.FIELD_E_KIN: O.kinetic_energy_density(st, op),
        B.FIELD_UC_MAG: np.sqrt((uc * uc).sum(axis=0)),
        B.FIELD_OMEGA_C: O.vorticity(uc),
    }
    for fld, w in want.items():
        assert scaled_err(tf.read_field(0, fld), w) <= 1e-5, fld


@pytest.mark.parametrize("nx,ny,steps", [(64, 48, 150), (40, 36, 150), (33, 17, 60)])
def test_spatial_correlations(nx, ny, steps):
    """Power-of-two rows (radix-2 FFT) and other sizes (direct DFT), centred
    u_c and omega_c, uncentred Q, against the direct shifted-sum definition."""
    tf, p = developed(nx, ny, steps)
    st, op = read_state(tf, 0), oracle_params(p)
    want = O.spatial_correlations(st, op)
    for which, w in zip((B.CORR_U, B.CORR_OMEGA, B.CORR_Q), want):
        got = tf.correlation(0, which)
        assert got[0] == pytest.approx(1.0, abs=1e-12)
        assert np.abs(got - w).max() <= 2e-5, (which, np.abs(got - w).max())


def test_time_correlations():
    tf, p = developed(48, 40, 120)
    op = oracle_params(p)
    then = read_state(tf, 0)
    tf.snapshot(0)
    assert np.allclose(tf.time_correlation(0), 1.0, atol=1e-6)
    tf.step(40)
    now = read_state(tf, 0)
    got = tf.time_correlation(0)
    want = O.time_correlations(then, now, op)
    assert np.abs(got - np.array(want)).max() <= 2e-5, (got, want)


@pytest.mark.parametrize("steps", [0, 80])
def test_defect_counts_exact(steps):
    """The random initial director (many defects) and a relaxed one."""
    tf, p = developed(64, 48, steps)
    st = read_state(tf, 0)
    got = tf.defects(0)
    want = O.defect_counts(st.Qxx, st.Qxy)
    assert list(got) == list(want)
    assert got[0] == got[1]          # zero total charge on the torus
    if steps == 0:
        assert got[0] > 100


def test_defects_of_a_written_pair():
    nx, ny = 32, 32
    tf = B.TwoFluid(CFG0.with_(nx=nx, ny=ny))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    th = 0.5 * np.arctan2(y - 16.5, x - 10.5) - 0.5 * np.arctan2(y - 16.5, x - 21.5)
    tf.write_field(0, B.FIELD_QXX, 0.3 * np.cos(2 * th))
    tf.write_field(0, B.FIELD_QXY, 0.3 * np.sin(2 * th))
    assert list(tf.defects(0)) == [1, 1, 0]


def test_reynolds():
    tf, p = developed(48, 40, 100, zeta=0.005)
    Re, La = tf.reynolds(0)
    want_re, want_la = O.reynolds(read_state(tf, 0), oracle_params(p))
    assert La == pytest.approx(want_la, rel=1e-14)
    assert Re == pytest.approx(want_re, rel=1e-5)
    tf0, _ = developed(16, 16, 2, zeta=0.0)
    assert tf0.reynolds(0)[0] == float("inf")


def test_observable_argument_errors():
    tf = B.TwoFluid(CFG0.with_(nx=16, ny=16))
    with pytest.raises(B.TwoFluidError):
        tf.time_correlation(0)        # no snapshot yet
    with pytest.raises(B.TwoFluidError):
        tf.correlation(0, 7)
