"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against a closed form, an invariant, a textbook
identity or a special case, never against a retyped copy of its own formula.
Citations name the paper's section / equation the pinned piece implements.
"""
import math

import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import inputs

P0 = O.Params()  # the 64x64 correctness configuration's parameters


def seeded_state(p, seed=0, phi0=0.5, dphi=0.01, S0=0.01):
    up, ut = inputs.initial_draws(seed, p.nx, p.ny)
    phi = phi0 + dphi * (2.0 * up - 1.0)
    Q = O.q_from_director(S0, np.pi * ut)
    return O.state_from_fields(phi, Q[0, 0], Q[0, 1], p)


# ---------------------------------------------------------------- lattice
def test_d2q9_isotropy():
    """Sec. III D2Q9: weight moments of a lattice with c_s^2 = 1/3."""
    c = O.CI.astype(float)
    w = O.WI
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(2) / 3)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0)
    d = np.eye(2)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4)


def test_equilibrium_moments():
    """Equilibrium carries rho, rho u and rho (cs2 I + u u)."""
    rng = np.random.default_rng(1)
    rho = 1 + 0.1 * rng.random((3, 4))
    u = 0.05 * rng.standard_normal((2, 3, 4))
    feq = O.equilibrium(rho, u)
    r, m = O.moments(feq)
    assert np.allclose(r, rho, atol=1e-15)
    assert np.allclose(m, rho * u, atol=1e-15)
    c = O.CI.astype(float)
    Pi = np.einsum("ia,ib,i...->ab...", c, c, feq)
    want = rho * (np.eye(2)[:, :, None, None] / 3 + np.einsum("a...,b...->ab...", u, u))
    assert np.allclose(Pi, want, atol=1e-15)


def test_guo_source_moments():
    """Guo forcing (Sec. III): zeroth moment 0, first (1-1/2tau) F,
    second (1-1/2tau)(u F + F u)."""
    rng = np.random.default_rng(2)
    u = 0.05 * rng.standard_normal((2, 5))
    F = 1e-3 * rng.standard_normal((2, 5))
    tau = 0.8
    S = O.guo_source(u, F, tau)
    c = O.CI.astype(float)
    k = 1 - 0.5 / tau
    assert np.allclose(S.sum(0), 0, atol=1e-18)
    assert np.allclose(np.einsum("ia,i...->a...", c, S), k * F, atol=1e-18)
    second = np.einsum("ia,ib,i...->ab...", c, c, S)
    want = k * (np.einsum("a...,b...->ab...", u, F) + np.einsum("a...,b...->ab...", F, u))
    assert np.allclose(second, want, atol=1e-18)


def test_streaming_moves_along_ci():
    """A pulse in f_i at x0 sits at x0 + c_i after streaming (periodic)."""
    ny, nx = 5, 7
    for i in range(9):
        f = np.zeros((9, ny, nx))
        f[i, 0, 6] = 1.0
        g = O.stream(f)
        y, x = np.argwhere(g[i] == 1.0)[0]
        assert (x, y) == ((6 + O.CI[i, 0]) % nx, (0 + O.CI[i, 1]) % ny)
        assert g.sum() == 1.0


# ------------------------------------------------------------ invariants
def test_phi_mass_conserved():
    """Flux-form central advection and the 5-point Laplacian sum to zero on a
    periodic grid, so sum(phi) is constant (Sec. II Eq. 1, Sec. III)."""
    p = P0.with_(nx=16, ny=12, zeta=0.05)
    s = seeded_state(p, seed=3)
    m0 = s.phi.sum()
    s = O.run(s, p, 30)
    assert abs(s.phi.sum() - m0) / m0 < 1e-13


def test_fluid_mass_conserved():
    """BGK and Guo have zero zeroth moment: sum rho_k constant per fluid."""
    p = P0.with_(nx=16, ny=12, zeta=0.05)
    s = seeded_state(p, seed=4)
    c0 = O.conserved(s, p)
    s = O.run(s, p, 30)
    c1 = O.conserved(s, p)
    assert abs(c1[1] - c0[1]) < 1e-11 and abs(c1[2] - c0[2]) < 1e-11


def test_momentum_bookkeeping():
    """Guo's first moment: sum m(n+1) - sum m(n) = sum (F1 + F2) = sum (G1 + G2)
    (the drag cancels between the fluids)."""
    p = P0.with_(nx=16, ny=16, zeta=0.2, gamma=0.3)
    s = seeded_state(p, seed=5, S0=0.3, dphi=0.2)
    s = O.run(s, p, 5)
    c0 = O.conserved(s, p)
    s1 = O.step(s, p)
    c1 = O.conserved(s1, p)
    scale = np.abs(O.macro(s, p)["G1"]).max()
    assert scale > 1e-6
    assert np.allclose(c1[3:5] - c0[3:5], c0[5:7], atol=1e-12 * scale * 256, rtol=0)


def test_momentum_exact_for_uniform_phi():
    """With phi uniform the forces are pure central divergences (active and
    elastic stresses) and the capillary force vanishes, so the step conserves
    the total momentum to rounding.  (Later steps need not: the flow makes
    phi non-uniform and sum(mu grad phi) is only O(dx^2).)"""
    p = P0.with_(nx=16, ny=16, zeta=0.3, gamma=0.2)
    s = seeded_state(p, seed=6, S0=0.5, dphi=0.0)
    s = O.State(s.f1, s.f2, s.phi, s.Qxx, s.Qxy)
    c0 = O.conserved(s, p)
    G1 = O.macro(s, p)["G1"]
    assert np.abs(G1).max() > 1e-3          # the forces are not trivially zero
    assert np.all(np.abs(c0[5:7]) < 1e-15)
    s1 = O.step(s, p)
    c1 = O.conserved(s1, p)
    assert np.all(np.abs(c1[3:5] - c0[3:5]) < 1e-15)
    assert np.abs(O.macro(s1, p)["u1"]).max() > 1e-4


# ------------------------------------------------------------------ drag
def test_drag_closed_form():
    """Uniform fields, u1 != u2: no gradients, only the implicit drag.  The
    velocity difference shrinks per step by exactly (1 - g)/(1 + g) with
    g = gamma phi (1 - phi) and rho1 = rho2 = 1; total momentum is constant."""
    phi0, gamma = 0.3, 0.4
    p = P0.with_(nx=4, ny=3, gamma=gamma, zeta=0.0)
    phi = np.full((3, 4), phi0)
    Z = np.zeros((3, 4))
    u1 = np.stack([np.full((3, 4), 0.02), np.full((3, 4), -0.01)])
    u2 = np.stack([np.full((3, 4), -0.03), np.full((3, 4), 0.005)])
    s = O.state_from_fields(phi, Z, Z, p, u1, u2)
    g = gamma * phi0 * (1 - phi0)
    r = (1 - g) / (1 + g)
    mc = O.macro(s, p)
    d0 = mc["u1"] - mc["u2"]
    mt0 = (mc["m1"] + mc["m2"]).sum(axis=(1, 2))
    for n in range(1, 6):
        s = O.step(s, p)
        mc = O.macro(s, p)
        assert np.allclose(mc["u1"] - mc["u2"], d0 * r ** n, rtol=1e-12, atol=1e-17)
        assert np.allclose((mc["m1"] + mc["m2"]).sum(axis=(1, 2)), mt0, atol=1e-15)


# ------------------------------------------------------------- viscosity
def _amp_sin(field, k, axis_coord):
    return 2.0 * np.mean(field * np.sin(k * axis_coord))


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_shear_wave_decay(tau):
    """Shear wave u_x = U sin(k y): decays as exp(-nu k^2 t), nu = (tau - 1/2)/3
    (BGK viscosity), with uniform phi and Q = 0 (lambda = 0 keeps Q = 0)."""
    N = 64
    k = 2 * np.pi / N
    p = P0.with_(nx=4, ny=N, tau1=tau, tau2=tau, lam=0.0, zeta=0.0, gamma=0.0)
    y = np.arange(N)[:, None] * np.ones((1, 4))
    U = 1e-4
    u = np.stack([U * np.sin(k * y), np.zeros_like(y)])
    Z = np.zeros_like(y)
    s = O.state_from_fields(np.full_like(y, 0.5), Z, Z, p, u, u)
    nu = (tau - 0.5) / 3
    T = 400
    a0 = _amp_sin(O.macro(s, p)["u1"][0], k, y)
    s = O.run(s, p, T)
    mc = O.macro(s, p)
    a1 = _amp_sin(mc["u1"][0], k, y)
    rate = -math.log(a1 / a0) / T
    assert abs(rate / (nu * k * k) - 1) < 0.01
    assert np.all(s.Qxx == 0) and np.all(s.Qxy == 0)
    assert np.max(np.abs(s.phi - 0.5)) < 1e-14


def test_shear_wave_with_drag_two_modes():
    """Wave in fluid 1 only, drag on: the sum u1 + u2 decays at nu k^2 and the
    difference at nu k^2 - ln((1 - g)/(1 + g)) per step (g = gamma phi(1-phi))."""
    N = 64
    k = 2 * np.pi / N
    gamma = 0.08
    p = P0.with_(nx=4, ny=N, lam=0.0, zeta=0.0, gamma=gamma)
    y = np.arange(N)[:, None] * np.ones((1, 4))
    u1 = np.stack([1e-4 * np.sin(k * y), 0 * y])
    Z = np.zeros_like(y)
    s = O.state_from_fields(np.full_like(y, 0.5), Z, Z, p, u1, 0 * u1)
    mc = O.macro(s, p)
    s0 = _amp_sin((mc["u1"] + mc["u2"])[0], k, y)
    d0 = _amp_sin((mc["u1"] - mc["u2"])[0], k, y)
    T = 60
    s = O.run(s, p, T)
    mc = O.macro(s, p)
    s1 = _amp_sin((mc["u1"] + mc["u2"])[0], k, y)
    d1 = _amp_sin((mc["u1"] - mc["u2"])[0], k, y)
    nu = (p.tau1 - 0.5) / 3
    g = gamma * 0.25
    assert abs(-math.log(s1 / s0) / T / (nu * k * k) - 1) < 0.01
    want = nu * k * k - math.log((1 - g) / (1 + g))
    assert abs(-math.log(d1 / d0) / T / want - 1) < 0.01


def test_guo_kolmogorov_steady_state():
    """Guo-forced BGK (Sec. III) with F_x = F0 sin(k y): the steady velocity is
    F0 sin(k y) / (rho nu k^2) to O(k^2).  Missing the (1 - 1/2tau) factor or
    the half-force shift changes the amplitude by O(1)."""
    N = 32
    k = 2 * np.pi / N
    tau = 0.9
    nu = (tau - 0.5) / 3
    y = np.arange(N)[:, None] * np.ones((1, 2))
    F0 = 1e-6
    F = np.stack([F0 * np.sin(k * y), 0 * y])
    f = O.equilibrium(np.ones_like(y), np.zeros((2,) + y.shape))
    for _ in range(6000):
        rho, m = O.moments(f)
        u = (m + 0.5 * F) / rho
        f = O.stream(O.collide(f, rho, u, F, tau))
    rho, m = O.moments(f)
    u = (m + 0.5 * F) / rho
    amp = _amp_sin(u[0], k, y)
    assert abs(amp / (F0 / (nu * k * k)) - 1) < 0.01


# --------------------------------------------------------- Cahn-Hilliard
def test_double_well_derivative():
    """f'(phi) is the derivative of f(phi) = phi^2 (1-phi)^2 (Sec. II)."""
    x = np.linspace(-0.3, 1.3, 17)
    h = 1e-6
    num = (O.double_well(x + h) - O.double_well(x - h)) / (2 * h)
    assert np.allclose(O.double_well_prime(x), num, atol=1e-9)


@pytest.mark.parametrize("n", [1, 3, 7])
def test_spinodal_growth_discrete(n):
    """Linear Cahn-Hilliard, no flow: a single mode of amplitude 1e-7 about
    phi0 = 1/2 grows per sub-step by G = 1 - dt M kh^2 (A_ch f''(1/2) + kappa kh^2),
    kh^2 = 4 sin^2(pi n / N) the 5-point Laplacian eigenvalue, f''(1/2) = -1."""
    N = 32
    p = P0.with_(nx=N, ny=2)
    x = np.arange(N)[None, :] * np.ones((2, 1))
    a = 1e-7
    phi = 0.5 + a * np.cos(2 * np.pi * n * x / N)
    zero = np.zeros((2, 2, N))
    dt = 1.0 / p.n_sub
    kh2 = 4 * np.sin(np.pi * n / N) ** 2
    G = 1 - dt * p.M * kh2 * (-p.A_ch + p.kappa * kh2)
    for s in range(1, 11):
        phi = phi + dt * O.ch_rate(phi, zero, zero, p)
        amp = 2 * np.mean((phi - 0.5) * np.cos(2 * np.pi * n * x / N))
        assert abs(amp / (a * G ** s) - 1) < 1e-8


def test_spinodal_continuum_band():
    """Continuum growth rate omega = M k^2 (A_ch - kappa k^2): unstable band
    k^2 < A_ch / kappa, fastest k^2 = A_ch / (2 kappa).  The discrete oracle
    rate approaches it as k -> 0 (relative error O(k^2))."""
    p = P0
    N = 256
    x = np.arange(N)[None, :] * np.ones((2, 1))
    zero = np.zeros((2, 2, N))
    rates = []
    ks = 2 * np.pi * np.arange(1, 60) / N
    for k in ks:
        phi = 0.5 + 1e-8 * np.cos(k * x)
        r = O.ch_rate(phi, zero, zero, p)
        rates.append(2 * np.mean(r * np.cos(k * x)) / 1e-8)
        if k < 0.3:
            cont = p.M * k * k * (p.A_ch - p.kappa * k * k)
            scale = p.M * k * k * (p.A_ch + p.kappa * k * k)
            assert abs(rates[-1] - cont) < 0.02 * scale
    rates = np.array(rates)
    kfast = ks[int(np.argmax(rates))]
    assert abs(kfast - math.sqrt(p.A_ch / (2 * p.kappa))) < 0.03
    kh2 = 4 * np.sin(ks / 2) ** 2
    assert np.all((rates > 0) == (kh2 < p.A_ch / p.kappa))


def test_tanh_interface_profile():
    """Flat-interface equilibrium of mu = A_ch f'(phi) - kappa phi'' = 0:
    phi = [1 + tanh(x / W)] / 2 with W = sqrt(2 kappa / A_ch) (= 2 here)."""
    N = 128
    p = P0.with_(nx=N, ny=1)
    x = np.arange(N, dtype=float)[None, :]
    W0 = 4.0
    phi = 0.5 * (np.tanh((x - N / 4) / W0) - np.tanh((x - 3 * N / 4) / W0))
    zero = np.zeros((2, 1, N))
    dt = 1.0 / p.n_sub
    for _ in range(40000):
        phi = phi + dt * O.ch_rate(phi, zero, zero, p)
    # least-squares width of the left interface
    xs = x[0, N // 8: 3 * N // 8] - N / 4
    prof = phi[0, N // 8: 3 * N // 8]
    Ws = np.linspace(1.5, 2.5, 2001)
    err = [np.sum((prof - 0.5 * (1 + np.tanh(xs / w))) ** 2) for w in Ws]
    W = Ws[int(np.argmin(err))]
    assert abs(W / math.sqrt(2 * p.kappa / p.A_ch) - 1) < 0.05
    assert abs(phi.max() - 1) < 0.02 and abs(phi.min()) < 0.02


def test_advection_sign():
    """-div(phi u_c) with uniform u_c = (U, 0) transports the pattern toward +x:
    d phi/dt = -U d phi/dx (central) for M = 0 (Sec. II Eq. 1)."""
    N = 32
    p = P0.with_(nx=N, ny=3, M=0.0)
    x = np.arange(N)[None, :] * np.ones((3, 1))
    k = 2 * np.pi / N
    phi = 0.5 + 0.01 * np.sin(k * x)
    U = 0.02
    u = np.stack([np.full_like(x, U), 0 * x])
    r = O.ch_rate(phi, u, u, p)
    assert np.allclose(r, -U * 0.01 * np.sin(k) * np.cos(k * x), atol=1e-16)


# --------------------------------------------------------- Beris-Edwards
def test_b_term_drops_in_2d():
    """In 2D Q.Q = (Tr Q^2 / 2) I, so the cubic-invariant term B only adds a
    multiple of I that Eq. (7) removes: H does not depend on B."""
    rng = np.random.default_rng(7)
    Q = O.q_tensor(rng.standard_normal((6, 5)) * 0.3, rng.standard_normal((6, 5)) * 0.3)
    H0 = O.molecular_field(Q, P0.with_(B_Q=0.0))
    H1 = O.molecular_field(Q, P0.with_(B_Q=0.7))
    assert np.allclose(H0, H1, atol=1e-15)
    assert np.allclose(O.trace(H0), 0, atol=1e-15)


def test_ldg_bulk_relaxation():
    """Uniform Q, no flow: dQ/dt = Gamma_Q H with H = -(A + C q^2) Q, q^2 =
    Qxx^2 + Qxy^2 (Eq. 7-8).  The Euler sub-steps follow the scalar map
    q <- q (1 - dt Gamma (A + C q^2)) exactly, the solution approaches the
    continuum q^2(t) = qe^2 / (1 + (qe^2/q0^2 - 1) exp(-2 Gamma |A| t)) to
    O(dt), and relaxes to the bulk order qe = sqrt(-A/C)."""
    p = P0.with_(nx=3, ny=2)
    th = 0.4
    q0 = 0.05
    Qxx = np.full((2, 3), q0 * np.cos(2 * th))
    Qxy = np.full((2, 3), q0 * np.sin(2 * th))
    Z = np.zeros((2, 2, 3))
    dt = 1 / p.n_sub
    q = q0
    for n in range(1, 401):
        Q = O.q_tensor(Qxx, Qxy)
        dxx, dxy = O.traceless_symmetric(O.be_rate(Q, Z, p))
        Qxx, Qxy = Qxx + dt * dxx, Qxy + dt * dxy
        q = q * (1 - dt * p.Gamma_Q * (p.A_Q + p.C_Q * q * q))
        qn = np.hypot(Qxx, Qxy)
        assert np.allclose(qn, q, rtol=1e-13)
        assert np.allclose(np.arctan2(Qxy, Qxx), 2 * th, atol=1e-13)
    t = 400 * dt
    qe2 = -p.A_Q / p.C_Q
    cont = qe2 / (1 + (qe2 / q0 ** 2 - 1) * math.exp(-2 * p.Gamma_Q * abs(p.A_Q) * t))
    assert abs(q * q / cont - 1) < 0.02
    for _ in range(20000):
        q = q * (1 - dt * p.Gamma_Q * (p.A_Q + p.C_Q * q * q))
    assert abs(q - math.sqrt(qe2)) < 1e-10


@pytest.mark.parametrize("nx,ny,mx,my,comp", [(16, 4, 3, 0, 0), (12, 10, 2, 3, 1),
                                             (8, 8, 4, 1, 0)])
def test_frank_term_single_mode_decay(nx, ny, mx, my, comp):
    """Frank part of the molecular field (Eq. 7-8): with A_Q = C_Q = 0 and no
    flow, H = K lap(Q), so the Beris-Edwards sub-step (Eq. 11) is the explicit
    heat equation Q <- Q + dt_fd Gamma_Q K lap(Q).  A Fourier mode of the
    periodic grid is an eigenvector of the five-point Laplacian with
    eigenvalue -k2, k2 = 4 sin^2(pi m_x / nx) + 4 sin^2(pi m_y / ny), so every
    sub-step multiplies it by exactly 1 - dt_fd Gamma_Q K k2.  A wrong sign or
    factor on K lap(Q), or a Laplacian missing from one component, fails."""
    p = P0.with_(nx=nx, ny=ny, A_Q=0.0, C_Q=0.0, K=0.37, Gamma_Q=0.45, lam=0.8)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    mode = np.cos(2 * np.pi * (mx * x / nx + my * y / ny) + 0.3)
    Qxx = 0.02 * mode if comp == 0 else np.zeros_like(mode)
    Qxy = 0.02 * mode if comp == 1 else np.zeros_like(mode)
    k2 = 4 * math.sin(math.pi * mx / nx) ** 2 + 4 * math.sin(math.pi * my / ny) ** 2
    dt_fd = p.dt / p.n_sub
    g = 1 - dt_fd * p.Gamma_Q * p.K * k2
    zero = np.zeros((2, ny, nx))
    phi = np.full((ny, nx), 0.5)
    # H itself: -k2 K times the mode in the excited component, zero in the other
    H = O.molecular_field(O.q_tensor(Qxx, Qxy), p)
    exc, other = (H[0, 0], H[0, 1]) if comp == 0 else (H[0, 1], H[0, 0])
    assert np.allclose(exc, -p.K * k2 * 0.02 * mode, rtol=0, atol=1e-15)
    assert np.allclose(other, 0, atol=1e-17)
    assert np.allclose(H[1, 1], -H[0, 0], atol=1e-17) and np.allclose(H[1, 0], H[0, 1], atol=1e-17)
    # every sub-step scales the mode by g (no flow: phi stays put)
    ph, a, b = phi, Qxx, Qxy
    for s in range(1, 4 * p.n_sub + 1):
        ph, a, b = O.substeps(ph, a, b, zero, zero, p.with_(n_sub=1, dt=dt_fd))
        exc = a if comp == 0 else b
        assert np.allclose(exc, 0.02 * mode * g ** s, rtol=0, atol=1e-12 * 0.02)
        assert np.allclose(b if comp == 0 else a, 0, atol=1e-17)
    assert np.allclose(ph, 0.5, atol=1e-16)


def test_fd_time_step_scales_the_substeps():
    """dt_fd = dt / n_sub (Sec. III): with the relaxation alone (uniform Q, no
    flow) one lattice step of n_sub sub-steps follows the scalar Euler map with
    that step, for the lattice-unit reading dt = 1 and the printed dt = 0.02."""
    for dt in (1.0, 0.02):
        p = P0.with_(nx=2, ny=2, dt=dt)
        q0 = 0.05
        Qxx = np.full((2, 2), q0)
        Qxy = np.zeros((2, 2))
        zero = np.zeros((2, 2, 2))
        _, a, _ = O.substeps(np.full((2, 2), 0.5), Qxx, Qxy, zero, zero, p)
        q = q0
        for _ in range(p.n_sub):
            q = q * (1 - (dt / p.n_sub) * p.Gamma_Q * (p.A_Q + p.C_Q * q * q))
        assert np.allclose(a, q, rtol=1e-14)


def test_velocity_gradient_index_order():
    """W_ij = d_j u_i: a shear u_x(y) has only W_xy."""
    N = 16
    y = np.arange(N)[:, None] * np.ones((1, 5))
    k = 2 * np.pi / N
    u = np.stack([np.sin(k * y), 0 * y])
    Wg = O.velocity_gradient(u)
    assert np.allclose(Wg[0, 1], np.sin(k) * np.cos(k * y), atol=1e-15)
    assert np.allclose(Wg[0, 0], 0) and np.allclose(Wg[1, 0], 0) and np.allclose(Wg[1, 1], 0)


@pytest.mark.parametrize("lam", [0.0, 0.7, 2.0])
@pytest.mark.parametrize("S0,th", [(0.3, 0.2), (1.0, 1.1), (0.6, -0.7)])
def test_director_rotation_in_shear(lam, S0, th):
    """Simple shear u_x = r y (W_xy = r) acting on Q = S0 (cos 2th, sin 2th)
    through Eq. (12).  Written in director form the traceless-symmetric part of
    S rotates the director at d th/dt = r (-1/2 + lam cos(2 th) / (4 S0)) and
    changes the order at dS/dt = (lam r / 2) sin(2 th) (1 - 4 S0^2).  For
    lam = 0 it is a pure co-rotation with the fluid's angular velocity -r/2."""
    r = 0.3
    Wg = np.zeros((2, 2, 1))
    Wg[0, 1] = r
    Q = O.q_tensor(np.array([S0 * np.cos(2 * th)]), np.array([S0 * np.sin(2 * th)]))
    dxx, dxy = O.traceless_symmetric(O.corotation(Wg, Q, P0.with_(lam=lam)))
    a, b = S0 * np.cos(2 * th), S0 * np.sin(2 * th)
    dth = (-np.sin(2 * th) * dxx + np.cos(2 * th) * dxy) / (2 * S0)
    assert np.allclose(dth, r * (-0.5 + lam * np.cos(2 * th) / (4 * S0)), atol=1e-15)
    dS = np.cos(2 * th) * dxx + np.sin(2 * th) * dxy
    assert np.allclose(dS, 0.5 * lam * r * np.sin(2 * th) * (1 - 4 * S0 ** 2), atol=1e-15)
    del a, b


def test_tumbling_threshold_at_unit_lambda():
    """Sec. II: |lambda| < 1 tumbles, |lambda| > 1 flow-aligns.  At the bulk
    order S0 = sqrt(-A_Q/C_Q) of the default parameters the director rate of
    Eq. (12) under shear has a steady (aligned) angle iff lambda >= 1."""
    S0 = math.sqrt(-P0.A_Q / P0.C_Q)
    r = 0.1
    Wg = np.zeros((2, 2, 1))
    Wg[0, 1] = r
    th = np.linspace(0, np.pi, 721)
    for lam, aligns in ((0.9, False), (0.99, False), (1.01, True), (1.1, True), (2.0, True)):
        rates = []
        for t_ in th:
            Q = O.q_tensor(np.array([S0 * np.cos(2 * t_)]), np.array([S0 * np.sin(2 * t_)]))
            dxx, dxy = O.traceless_symmetric(O.corotation(Wg, Q, P0.with_(lam=lam)))
            rates.append(float((-np.sin(2 * t_) * dxx + np.cos(2 * t_) * dxy)[0]))
        rates = np.array(rates)
        has_zero = bool(np.any(rates >= 0) and np.any(rates < 0))
        assert has_zero == aligns


def test_corotation_rigid_rotation():
    """lam = 0, rigid rotation u = w (-y, x): Q rotates counter-clockwise at
    angular rate w, i.e. dQxx/dt = -2 w Qxy, dQxy/dt = 2 w Qxx."""
    w = 0.05
    Wg = np.zeros((2, 2, 1))
    Wg[0, 1] = -w   # d_y u_x
    Wg[1, 0] = w    # d_x u_y
    Q = O.q_tensor(np.array([0.3]), np.array([-0.2]))
    dxx, dxy = O.traceless_symmetric(O.corotation(Wg, Q, P0.with_(lam=0.0)))
    assert np.allclose(dxx, -2 * w * (-0.2)) and np.allclose(dxy, 2 * w * 0.3)


def test_extension_aligns_q():
    """Q = 0 under pure extension E = diag(e, -e): S = lam E, so Qxx grows at
    lam e (flow alignment along the stretching axis)."""
    e = 0.01
    Wg = np.zeros((2, 2, 1))
    Wg[0, 0], Wg[1, 1] = e, -e
    Z = np.zeros(1)
    dxx, dxy = O.traceless_symmetric(O.corotation(Wg, O.q_tensor(Z, Z), P0.with_(lam=0.7)))
    assert np.allclose(dxx, 0.7 * e) and np.allclose(dxy, 0)


# ------------------------------------------------------------ stresses
def test_elastic_stress_identities():
    """Sec. II elastic stress: (i) Q = 0 gives -lam H - T; (ii) the
    antisymmetric part is Q.H - H.Q (all other terms are symmetric);
    (iii) H parallel to Q gives a symmetric stress."""
    rng = np.random.default_rng(8)
    p = P0.with_(lam=0.9, K=0.3)
    Q = O.q_tensor(0.4 * rng.standard_normal((8, 8)), 0.4 * rng.standard_normal((8, 8)))
    H = O.q_tensor(rng.standard_normal((8, 8)), rng.standard_normal((8, 8)))
    sig = O.elastic_stress(Q, H, p)
    anti = 0.5 * (sig - O.transpose(sig))
    comm = O.matmul(Q, H) - O.matmul(H, Q)
    assert np.allclose(anti, 0.5 * (comm - O.transpose(comm)), atol=1e-14)
    assert np.allclose(anti, comm, atol=1e-14)
    sig_par = O.elastic_stress(Q, 1.7 * Q, p)
    assert np.allclose(sig_par, O.transpose(sig_par), atol=1e-14)
    Z = np.zeros((8, 8))
    Q0 = O.q_tensor(Z, Z)
    sig0 = O.elastic_stress(Q0, H, p)
    assert np.allclose(sig0, -p.lam * H, atol=1e-15)


def test_frank_stress_term():
    """(grad Q).dF/d(grad Q) with F_K = (K/2) sum_kij (d_k Q_ij)^2:
    for Qxx = a sin(k x) it is diag(2 K (d_x Qxx)^2, 0)."""
    N = 16
    x = np.arange(N)[None, :] * np.ones((4, 1))
    k = 2 * np.pi / N
    Qxx = 0.3 * np.sin(k * x)
    Q = O.q_tensor(Qxx, 0 * x)
    H = O.q_tensor(0 * x, 0 * x)
    K = 0.25
    sig = O.elastic_stress(Q, H, P0.with_(K=K, lam=0.0))
    dQ = 0.3 * np.sin(k) * np.cos(k * x)
    assert np.allclose(sig[0, 0], -2 * K * dQ ** 2, atol=1e-16)
    assert np.allclose(sig[1, 1], 0) and np.allclose(sig[0, 1], 0)


def test_active_force_single_mode():
    """F_active = div(zeta phi Q) (Sec. II) for Qxx = a sin(k x), phi uniform."""
    N = 16
    x = np.arange(N)[None, :] * np.ones((4, 1))
    k = 2 * np.pi / N
    Z = 0 * x
    p = P0.with_(zeta=0.2, lam=0.0, K=0.0, A_Q=0.0, C_Q=0.0, A_ch=0.0, kappa=0.0)
    Q = O.q_tensor(0.3 * np.sin(k * x), Z)
    G1, G2 = O.forces(np.full_like(x, 0.5), Q, p)
    assert np.allclose(G1[0], 0.2 * 0.5 * 0.3 * np.sin(k) * np.cos(k * x), atol=1e-16)
    assert np.allclose(G1[1], 0, atol=1e-16) and np.allclose(G2, 0, atol=1e-16)


def test_capillary_force_continuum_limit():
    """mu grad(phi) - grad(phi mu) = -phi grad(mu) in the continuum (Eq. 10);
    the central-difference form converges to it at second order."""
    errs = []
    for N in (32, 64, 128):
        x = np.arange(N)[None, :] * np.ones((2, 1))
        k = 2 * np.pi / N
        phi = 0.5 + 0.2 * np.sin(k * x) + 0.1 * np.cos(2 * k * x)
        mu = np.cos(k * x) + 0.3 * np.sin(3 * k * x)
        dmu = -k * np.sin(k * x) + 0.9 * k * np.cos(3 * k * x)
        F = O.capillary_force(phi, mu)[0]
        errs.append(np.max(np.abs(F + phi * dmu)) / np.max(np.abs(phi * dmu)))
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2) < 0.15 for o in order)


# ------------------------------------------------------------ observables
def test_fourier_matches_brute_dft():
    """Normalised transform (1/N) sum_x g e^{-i k.x} against an O(N^4) sum."""
    ny, nx = 6, 8
    g = np.random.default_rng(9).standard_normal((ny, nx))
    out = np.zeros((ny, nx), complex)
    for qy in range(ny):
        for qx in range(nx):
            s = 0j
            for y in range(ny):
                for x in range(nx):
                    s += g[y, x] * np.exp(-2j * np.pi * (qx * x / nx + qy * y / ny))
            out[qy, qx] = s / (nx * ny)
    assert np.allclose(O.fourier(g), out, atol=1e-14)


def test_structure_factor_parseval_and_single_mode():
    N = 32
    g = np.random.default_rng(10).standard_normal((N, N))
    ph = O.fourier(g - g.mean())
    assert abs((np.abs(ph) ** 2).sum() - np.mean((g - g.mean()) ** 2)) < 1e-13
    x = np.arange(N)[None, :] * np.ones((N, 1))
    y = x.T
    phi = 0.5 + 0.1 * np.cos(2 * np.pi * (3 * x + 4 * y) / N)
    S = O.structure_factor(phi)
    assert abs(S[5] - 2 * 0.05 ** 2) < 1e-15 and abs(S.sum() - S[5]) < 1e-15
    L = O.length_scale(phi)
    assert abs(L - N / (2 * np.pi * 5)) < 1e-12


def test_energy_spectrum_total_is_half_mean_square():
    rng = np.random.default_rng(11)
    u = rng.standard_normal((2, 16, 16))
    Ek, Etot = O.energy_spectrum(u)
    assert abs(Etot - 0.5 * np.mean((u * u).sum(0))) < 1e-13
    assert Ek.sum() <= Etot + 1e-15
    assert np.all(O.shell_counts(16, 16) >= 1)


def test_vorticity_single_mode():
    N = 16
    y = np.arange(N)[:, None] * np.ones((1, N))
    k = 2 * np.pi / N
    u = np.stack([np.sin(k * y), 0 * y])
    assert np.allclose(O.vorticity(u), -np.sin(k) * np.cos(k * y), atol=1e-15)
