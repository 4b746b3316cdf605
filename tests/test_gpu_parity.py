"""GPU (CUDA path through the C ABI) against the FP64 oracle.

Every input is seeded and synthetic; the GPU state is read back exactly and
handed to the oracle, so both start from identical values.
"""
import math

import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import _binding as B
from paper_2511_00445_gb300 import inputs

from helpers import (TOL_200, assert_parity, field_errors, oracle_params, read_state,
                     read_velocities, rel_err)

pytestmark = pytest.mark.gpu

CFG0 = B.SolverParams()  # 64x64 correctness configuration (zeta 0.005, lambda 0.7, K 0.04, ...)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_00445_gb300 import build
    build.build()


def make(params, seed=0, **init):
    tf = B.TwoFluid(params)
    kw = dict(phi0=0.5, dphi=0.01, S0=0.01)
    kw.update(init)
    tf.init_fields(seed, **kw)
    tf.sync()
    return tf


# ------------------------------------------------------------------ init
@pytest.mark.parametrize("nx,ny", [(64, 64), (37, 5), (1, 1)])
def test_init_matches_counter_generator(nx, ny):
    """Sec. III initial condition drawn on the device equals the host draws of
    the same SplitMix64 counters (phi exactly after FP32 rounding, Q to 1 ulp)."""
    tf = make(CFG0.with_(nx=nx, ny=ny), seed=12345, dphi=0.02, S0=0.3)
    up, ut = inputs.initial_draws(12345, nx, ny)
    phi_host = 0.5 + np.float32(0.5 + 0.02 * (2 * up - 1) - 0.5).astype(np.float64)
    assert np.array_equal(tf.read_field(0, B.FIELD_PHI), phi_host)
    Q = O.q_from_director(0.3, np.pi * ut)
    for fld, want in ((B.FIELD_QXX, Q[0, 0]), (B.FIELD_QXY, Q[0, 1])):
        got = tf.read_field(0, fld)
        assert np.all(np.abs(got - want.astype(np.float32)) <= np.spacing(np.float32(0.3)))
    for i in range(9):
        assert np.all(tf.read_field(0, B.FIELD_F1 + i) == O.WI[i])
        assert np.all(tf.read_field(0, B.FIELD_F2 + i) == O.WI[i])


def test_field_roundtrip_and_pull_layout():
    """Writing then reading a population field returns the FP32-rounded values
    (the pull layout shift is undone exactly)."""
    p = CFG0.with_(nx=7, ny=5)
    tf = make(p)
    rng = np.random.default_rng(3)
    for fld in (B.FIELD_F1 + 5, B.FIELD_F2 + 7, B.FIELD_QXY):
        v = 0.03 + 1e-3 * rng.standard_normal((5, 7))
        tf.write_field(0, fld, v)
        got = tf.read_field(0, fld)
        assert np.allclose(got, v, rtol=0, atol=4e-9)


# ------------------------------------------------------------ step parity
def run_pair(p: B.SolverParams, steps: int, seed=0, **init):
    tf = make(p, seed=seed, **init)
    op = oracle_params(p)
    ref = read_state(tf, 0)
    tf.step(steps)
    tf.sync()
    ref = O.run(ref, op, steps)
    return tf, ref, op


@pytest.mark.parametrize("nx,ny,steps", [(8, 8, 200), (16, 16, 200), (64, 64, 200), (64, 48, 200),
                                         (5, 3, 50), (1, 1, 20), (2, 7, 50), (33, 17, 100)])
def test_step_parity(nx, ny, steps):
    """Brute force at small sizes (several tiles plus ragged tails, degenerate
    1x1 and 2-wide grids) after `steps` coupled steps, cfg0 parameters."""
    tf, ref, op = run_pair(CFG0.with_(nx=nx, ny=ny), steps)
    assert_parity(field_errors(tf, 0, ref, op), nx, ny)


@pytest.mark.parametrize("n_sub,nx,ny", [(3, 16, 16), (1, 9, 7), (8, 20, 12)])
def test_step_parity_unfused_path(n_sub, nx, ny):
    """Sub-step counts other than five run the per-stage kernels."""
    tf, ref, op = run_pair(CFG0.with_(nx=nx, ny=ny, n_sub=n_sub), 100)
    assert_parity(field_errors(tf, 0, ref, op), nx, ny)


def test_interleaved_steps_and_reads():
    """Reads between steps complete the pending sub-steps and do not change
    the trajectory: 1+2+3+4 steps with reads in between equal 10 steps."""
    p = CFG0.with_(nx=40, ny=36, zeta=0.01)
    a = make(p, seed=3)
    b = make(p, seed=3)
    for n in (1, 2, 3, 4):
        a.step(n)
        a.read_field(0, B.FIELD_PHI)
        a.conserved(0)
    b.step(10)
    for fld in (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_F1 + 1, B.FIELD_F2 + 8,
                B.FIELD_U1X, B.FIELD_U2Y):
        assert np.array_equal(a.read_field(0, fld), b.read_field(0, fld)), fld
    assert a.step_count() == b.step_count() == 10


def test_step_parity_strong_coupling():
    """Large drag, activity, tumbling and elastic constant; unequal tau and
    densities; a non-symmetric initial condition."""
    p = CFG0.with_(nx=24, ny=20, gamma=0.3, zeta=0.02, lam=1.1, K=0.08, tau1=0.8, tau2=1.4,
                   rho1=1.0, rho2=1.2)
    tf, ref, op = run_pair(p, 100, seed=7, dphi=0.2, S0=0.4)
    assert_parity(field_errors(tf, 0, ref, op), p.nx, p.ny)


def test_batch_zeta_sweep_full_size():
    """The activity sweep zeta in {0, 0.002, 0.005, 0.01} on 256x256 (the
    benchmarked configuration, same launch path): every site of every
    instance after 3 steps."""
    ps = [CFG0.with_(nx=256, ny=256, zeta=z) for z in (0.0, 0.002, 0.005, 0.01)]
    tf = make(ps, seed=0)
    refs = [read_state(tf, b) for b in range(4)]
    tf.step(3)
    tf.sync()
    for b, p in enumerate(ps):
        op = oracle_params(p)
        ref = O.run(refs[b], op, 3)
        assert_parity(field_errors(tf, b, ref, op), p.nx, p.ny)


def test_results_independent_of_tile_rows():
    """The per-context launch cuts the rows into as many tile rows as fill one
    wave of resident CTAs: a batch of four 256x256 instances runs in fewer,
    taller tiles than a single instance does.  Every stored value depends only
    on its dependency cone, so the same instance stepped either way is
    bitwise the same (fields, populations and velocities)."""
    p = CFG0.with_(nx=256, ny=256, zeta=0.01)
    a = make([p] * 4, seed=2)
    b = make(p, seed=2)
    a.step(20)
    b.step(20)
    for fld in (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_F1 + 5, B.FIELD_F2 + 7, B.FIELD_U1X):
        want = b.read_field(0, fld)
        for inst in (0, 3):
            assert np.array_equal(a.read_field(inst, fld), want), (inst, fld)


def test_velocities_match_oracle_macro():
    """Derived Guo velocities of an arbitrary (non-equilibrium) state."""
    p = CFG0.with_(nx=12, ny=10, gamma=0.2, zeta=0.05)
    tf = make(p, seed=4, dphi=0.1, S0=0.3)
    rng = np.random.default_rng(5)
    tf.set_equilibrium(0, 0.01 * rng.standard_normal((2, 10, 12)),
                       0.01 * rng.standard_normal((2, 10, 12)))
    ref = read_state(tf, 0)
    mc = O.macro(ref, oracle_params(p))
    u1, u2 = read_velocities(tf, 0)
    for got, want in ((u1, mc["u1"]), (u2, mc["u2"])):
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    rho1 = tf.read_field(0, B.FIELD_RHO1)
    assert np.abs(rho1 - mc["rho1"]).max() < 1e-6


# --------------------------------------------------------------- invariants
def test_conserved_sums_and_momentum_bookkeeping():
    """FP64 device sums equal the oracle's sums of the same state; Guo's
    first moment gives sum m(n+1) - sum m(n) = sum G(n) on the GPU too."""
    p = CFG0.with_(nx=32, ny=32, zeta=0.05, gamma=0.2)
    tf = make(p, seed=9, dphi=0.1, S0=0.3)
    tf.step(20)
    c0 = tf.conserved(0)
    ref = read_state(tf, 0)
    want = O.conserved(ref, oracle_params(p))
    assert abs(c0[0] - want[0]) < 1e-9 * abs(want[0])
    assert np.allclose(c0[1:3], want[1:3], rtol=1e-12, atol=1e-7)
    scale = np.abs(O.macro(ref, oracle_params(p))["G1"]).max() * p.nx * p.ny
    assert np.allclose(c0[3:7], want[3:7], rtol=0, atol=1e-5 * scale)
    assert c0[7] == 0
    tf.step(1)
    c1 = tf.conserved(0)
    assert np.allclose(c1[3:5] - c0[3:5], c0[5:7], rtol=0, atol=2e-5 * scale)
    # phi mass and fluid masses: constant up to FP32 storage rounding
    tf.step(200)
    c2 = tf.conserved(0)
    assert abs(c2[0] - c0[0]) < 1e-6 * c0[0]
    assert np.allclose(c2[1:3], c0[1:3], rtol=1e-6)


def test_nonfinite_detected():
    p = CFG0.with_(nx=16, ny=16)
    tf = make(p)
    phi = tf.read_field(0, B.FIELD_PHI)
    phi[3, 4] = np.nan
    tf.write_field(0, B.FIELD_PHI, phi)
    with pytest.raises(B.TwoFluidError) as ei:
        tf.conserved(0)
    assert ei.value.code == B.TF_ERR_NONFINITE
    c = tf.conserved(0, check=False)
    assert c[7] >= 1


@pytest.mark.parametrize("n_sub", [5, 3])
def test_check_every_reports_nonfinite_from_tf_sync(n_sub):
    """check_every = k scans the state after every k-th step on the device:
    a NaN written from the host makes the next tf_sync return
    TF_ERR_NONFINITE (no trap, the context stays usable), the code is cleared
    once read, and a clean run never sets it."""
    p = CFG0.with_(nx=24, ny=20, n_sub=n_sub, check_every=4)
    clean = make(p)
    clean.step(9)
    clean.sync()
    tf = make(p)
    tf.step(2)
    phi = tf.read_field(0, B.FIELD_PHI)
    phi[5, 7] = np.nan
    tf.write_field(0, B.FIELD_PHI, phi)
    tf.step(1)                      # step 3: no scan yet
    tf.sync()
    tf.step(1)                      # step 4: scanned
    with pytest.raises(B.TwoFluidError) as ei:
        tf.sync()
    assert ei.value.code == B.TF_ERR_NONFINITE
    tf.sync()                       # cleared once reported
    assert tf.step_count() == 4
    # the context still works: overwrite the state and step on
    tf.init_fields(0, phi0=0.5, dphi=0.01, S0=0.01)
    tf.step(8)
    tf.sync()


def test_step_parity_printed_parameters_literal_dt():
    """The paper's printed Sec. III set (eta = 0.5 as tau = 2, gamma = 0.1,
    K = 0.1, Gamma_Q = 0.2, zeta = 0.01) under the literal time step dt = 0.02
    (dt_fd = dt / 5), which runs stably: GPU against the oracle after 200 steps."""
    p = CFG0.with_(nx=64, ny=64, tau1=2.0, tau2=2.0, gamma=0.1, K=0.1, zeta=0.01, dt=0.02)
    tf, ref, op = run_pair(p, 200)
    assert op.dt == 0.02
    assert_parity(field_errors(tf, 0, ref, op), p.nx, p.ny)


# ------------------------------------------------------------- observables
def test_observables_match_oracle():
    """Structure factor, L(t), kinetic-energy spectrum, phase differences and
    Delta of a developed GPU state, against the oracle on the same fields."""
    for nx, ny in ((64, 64), (32, 16)):
        p = CFG0.with_(nx=nx, ny=ny, zeta=0.01)
        tf = make(p, seed=2)
        tf.step(120)
        ref = read_state(tf, 0)
        op = oracle_params(p)
        S = tf.structure_factor(0)
        Sw = O.structure_factor(ref.phi)
        assert np.allclose(S, Sw, rtol=1e-9, atol=1e-14 * Sw.max())
        assert abs(tf.length_scale(0) - O.length_scale(ref.phi)) < 1e-9 * O.length_scale(ref.phi)
        mc = O.macro(ref, op)
        uc = O.mixture_velocity(ref.phi, mc["u1"], mc["u2"])
        E, Et = tf.energy_spectrum(0)
        Ew, Etw = O.energy_spectrum(uc)
        assert np.allclose(E, Ew, rtol=1e-5, atol=1e-6 * Ew.max())
        assert abs(Et - Etw) < 1e-5 * Etw
        pd = tf.phase_difference(0)
        pdw = O.phase_difference(ref, op)
        assert np.allclose(pd, pdw, rtol=1e-5)
        m, s = tf.phi_stats(0)
        assert abs(m - ref.phi.mean()) < 1e-12 and abs(s - O.std_phi(ref.phi)) < 1e-9 * s
        assert np.array_equal(tf.shell_counts(), O.shell_counts(nx, ny))


def test_spectrum_single_mode():
    """A single Fourier mode of phi lands in one shell with power a^2/2 and
    gives L = 1 / k_m (Sec. IV, Eq. 27) -- closed form, no oracle."""
    N = 64
    p = CFG0.with_(nx=N, ny=N)
    tf = make(p)
    x = np.arange(N)[None, :] * np.ones((N, 1))
    y = x.T
    tf.write_field(0, B.FIELD_PHI, 0.5 + 0.01 * np.cos(2 * np.pi * (3 * x + 4 * y) / N))
    S = tf.structure_factor(0)
    assert abs(S[5] - 0.5 * 0.01 ** 2) < 1e-12 and abs(S.sum() - S[5]) < 1e-12
    assert abs(tf.length_scale(0) - N / (2 * math.pi * 5)) < 1e-6


# ------------------------------------------------------- state management
def test_checkpoint_resume_bitwise(tmp_path):
    p = [CFG0.with_(nx=40, ny=24, zeta=z) for z in (0.002, 0.01)]
    a = make(p, seed=11)
    a.step(30)
    a.sync()
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(30)
    a.sync()
    b = B.TwoFluid(p)
    b.load(path)
    assert b.step_count() == 30
    b.step(30)
    b.sync()
    for inst in range(2):
        for fld in (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_F1 + 6, B.FIELD_F2 + 2):
            assert np.array_equal(a.read_field(inst, fld), b.read_field(inst, fld))
    with pytest.raises(B.TwoFluidError):
        B.TwoFluid(CFG0.with_(nx=8, ny=8)).load(path)


def test_run_to_run_determinism():
    p = CFG0.with_(nx=48, ny=48, zeta=0.01)
    a = make(p, seed=1)
    b = make(p, seed=1)
    a.step(50)
    b.step(50)
    for fld in (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_U1X):
        assert np.array_equal(a.read_field(0, fld), b.read_field(0, fld))


def test_advance_host_equals_device_steps():
    import torch
    p = CFG0.with_(nx=32, ny=32)
    a = make(p, seed=5)
    b = make(p, seed=5)
    nb = a.state_bytes()
    h_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    a.advance_host(None, 0, h_in.data_ptr())
    a.advance_host(h_in.data_ptr(), 7, h_out.data_ptr())
    b.step(7)
    assert np.array_equal(a.read_field(0, B.FIELD_PHI), b.read_field(0, B.FIELD_PHI))
    b.advance_host(None, 0, h_in.data_ptr())
    assert torch.equal(h_in, h_out)


@pytest.mark.parametrize("storage", [B.STORE_F32, B.STORE_F16], ids=["f32", "f16"])
def test_advance_host_batch_pipeline_bitwise(storage):
    """On a batch the host-buffer entry point runs pipelined per instance
    (the uploads, steps and downloads of different instances overlap on the
    context's own streams; five instances wrap around its four compute
    lanes; pinned buffers replay a captured graph, pageable ones are enqueued
    directly).  Every use of it gives bitwise the state of plain device steps:
    a download that first completes pending sub-steps, an upload alone from
    pageable memory, an upload and a download through one buffer, and an
    upload followed by steps that leave sub-steps pending."""
    import torch
    ps = [CFG0.with_(nx=40, ny=36, zeta=z, storage=storage) for z in (0.0, 0.002, 0.005, 0.01, 0.02)]
    fields = [B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_U1X, B.FIELD_U2Y] + \
             [B.FIELD_F1 + i for i in range(9)] + [B.FIELD_F2 + i for i in (0, 3, 8)]

    def same(x, y):
        for inst in range(len(ps)):
            for fld in fields:
                assert np.array_equal(x.read_field(inst, fld), y.read_field(inst, fld)), (inst, fld)

    a, b = make(ps, seed=3), make(ps, seed=3)
    h = torch.empty(a.state_bytes(), dtype=torch.uint8, pin_memory=True)
    a.step(4)
    b.step(4)
    a.advance_host(None, 3, h.data_ptr())          # pending sub-steps, 3 steps, download
    b.step(3)
    same(a, b)
    c = B.TwoFluid(ps)
    hp = h.numpy().copy()                          # pageable memory: enqueued, not captured
    c.advance_host(hp.ctypes.data, 0, None)        # upload only
    same(c, b)
    a.advance_host(h.data_ptr(), 2, h.data_ptr())  # one buffer in and out
    b.step(2)
    same(a, b)
    d = B.TwoFluid(ps)
    d.advance_host(h.data_ptr(), 5, None)          # upload, steps, sub-steps left pending
    b.step(5)
    same(d, b)
    assert a.step_count() == 9 and b.step_count() == 14 and d.step_count() == 5


@pytest.mark.parametrize("nx,ny,storage,n", [(64, 384, B.STORE_F32, 1), (48, 1000, B.STORE_F16, 1),
                                              (64, 512, B.STORE_BF16, 3), (2048, 2048, B.STORE_F32, 1)],
                         ids=["3bands", "7bands-ragged-f16", "4bands-3steps-bf16", "2048sq-16bands"])
def test_advance_host_banded_bitwise(nx, ny, storage, n):
    """A single instance through host buffers runs in row bands (uploads,
    LBM-only passes, FD-only passes and downloads of different bands overlap;
    with more than one step the middle steps are whole-grid launches).  The
    downloaded raw state and the context's fields equal plain device steps bit
    for bit, also with one buffer for input and output."""
    import torch
    p = CFG0.with_(nx=nx, ny=ny, zeta=0.01, storage=storage)
    a, b = make(p, seed=9), make(p, seed=9)
    nb = a.state_bytes()
    h_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    h_ref = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    a.advance_host(None, 0, h_in.data_ptr())                  # the plain state, downloaded
    a.advance_host(h_in.data_ptr(), n, h_out.data_ptr())      # banded: upload, n steps, download
    b.step(n)
    b.advance_host(None, 0, h_ref.data_ptr())
    assert torch.equal(h_out, h_ref)
    for fld in (B.FIELD_PHI, B.FIELD_QXY, B.FIELD_U1X, B.FIELD_F1 + 5, B.FIELD_F2 + 8):
        assert np.array_equal(a.read_field(0, fld), b.read_field(0, fld)), fld
    a.advance_host(h_out.data_ptr(), n, h_out.data_ptr())     # one buffer in and out (graph replay)
    b.step(n)
    b.advance_host(None, 0, h_ref.data_ptr())
    assert torch.equal(h_out, h_ref)
    assert a.step_count() == b.step_count() == 2 * n


def test_argument_errors():
    tf = make(CFG0.with_(nx=8, ny=8))
    for call in (lambda: tf.read_field(1, B.FIELD_PHI), lambda: tf.read_field(0, 99),
                 lambda: tf.write_field(0, B.FIELD_U1X, np.zeros((8, 8))),
                 lambda: tf.step(-1), lambda: tf.init_fields(0, inst=3)):
        with pytest.raises(B.TwoFluidError) as ei:
            call()
        assert ei.value.code == B.TF_ERR_ARG
    tf.step(0)
    assert tf.step_count() == 0
