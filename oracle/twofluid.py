"""Plain FP64 CPU oracle of the coupled two-fluid lattice step.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement
of what the CUDA path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library and imports nothing from the product package.

Method (Ahmed, Lin & Qu, "Phase separation dynamics and active turbulence in a
binary fluid mixture", arXiv 2511.00445):

* Sec. II, Eq. (1)-(3): Cahn-Hilliard equation for the active concentration phi
  with chemical potential mu = f'(phi) - eps^2 lap(phi), f = phi^2 (1-phi)^2.
* Sec. II, Eq. (4)-(6): one momentum equation per fluid, coupled by the drag
  F_drag = gamma phi (1-phi) (u2 - u1); fluid 1 also feels the active force
  div(zeta phi Q) and the elastic stress; both feel the capillary force.
* Sec. II, elastic-stress display (after Eq. 6), Eq. (7)-(8): elastic stress,
  molecular field H and Landau-de Gennes free energy.
* Sec. II, Eq. (10): capillary force F_ch = mu grad(phi) - grad(phi mu).
* Sec. II, Eq. (11)-(12): Beris-Edwards equation and the co-rotation term S.
* Sec. III: D2Q9 BGK lattice Boltzmann per fluid with Guo forcing, periodic
  boundaries, second-order central differences for phi and Q, five
  finite-difference sub-steps per lattice step.

Readings where the paper is silent or ambiguous:
lattice units (dt = dx = 1, tau given directly); A_ch multiplies the double
well and kappa = eps^2; the LdG coefficients A_Q, B_Q, C_Q are parameters (B_Q
drops out in 2D) and default to a bulk order S = sqrt(-A_Q/C_Q) = 1/2, the
value at which the co-rotation term puts the tumbling-to-aligning transition
at |lambda| = 1 as Sec. II states; forces enter each lattice-Boltzmann fluid per unit volume
(the phi factors on the left of Eq. 4-5 are not divided out); the elastic force
is the divergence of the elastic stress on its second index, applied to fluid 1;
the Guo half-force velocity shift includes the implicit drag, which turns the
velocity evaluation into a 2x2 solve; forces are evaluated from (phi^n, Q^n);
the five sub-steps are forward Euler with u1, u2 frozen and phi, Q updated
simultaneously; W_ij = d_j u_i, E = sym(W), Omega = antisym(W); the
Beris-Edwards increment is projected onto its traceless-symmetric part;
phi advection is the conservative central flux form, Q advection the central
non-conservative form.

Tensors are stored as arrays of shape (2, 2, ny, nx) with tensor indices
first; scalars as (ny, nx); vectors as (2, ny, nx) with component (x, y).
Array axis -1 is x, axis -2 is y.
"""
from __future__ import annotations

from dataclasses import dataclass, replace, asdict

import numpy as np

# D2Q9 velocity set and weights (Sec. III, "two-dimensional D2Q9 lattice").
# Order: rest, the four axis directions counter-clockwise from +x, then the
# four diagonals counter-clockwise from (+1, +1).
CI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
               [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
WI = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
CS2 = 1.0 / 3.0  # lattice speed of sound squared


@dataclass(frozen=True)
class Params:
    """Model and scheme parameters (Sec. III parameter list, lattice units)."""
    nx: int = 64
    ny: int = 64
    tau1: float = 1.0        # BGK relaxation time of the active fluid
    tau2: float = 1.0        # BGK relaxation time of the passive fluid
    rho1: float = 1.0        # rest density of fluid 1 (initial equilibrium)
    rho2: float = 1.0        # rest density of fluid 2
    gamma: float = 0.01      # drag (momentum transfer) coefficient, Eq. (4)-(5)
    zeta: float = 0.005      # activity, F_active = div(zeta phi Q)
    lam: float = 0.7         # tumbling / flow-alignment parameter lambda
    K: float = 0.04          # Frank elastic constant, Eq. (8)
    Gamma_Q: float = 0.2     # rotational diffusion Gamma in Eq. (11)
    A_Q: float = -0.1        # Landau-de Gennes A, Eq. (8)
    B_Q: float = 0.0         # Landau-de Gennes B (drops out in 2D)
    C_Q: float = 0.4         # Landau-de Gennes C (bulk order sqrt(-A_Q/C_Q) = 1/2)
    M: float = 0.2           # Cahn-Hilliard mobility, Eq. (1)
    A_ch: float = 0.05       # prefactor of the double well f(phi)
    kappa: float = 0.1       # eps^2 in mu = A_ch f'(phi) - eps^2 lap(phi), Eq. (2)
    n_sub: int = 5           # finite-difference sub-steps per lattice step (Sec. III)
    dt: float = 1.0          # one lattice step in the time unit of the FD rates (Sec. III:
                             # dt_fd = dt / n_sub; 1 = lattice units, the default reading)

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class State:
    """Full FP64 state: pre-collision populations at time n and phi^n, Q^n."""
    f1: np.ndarray   # (9, ny, nx) populations of the active fluid
    f2: np.ndarray   # (9, ny, nx) populations of the passive fluid
    phi: np.ndarray  # (ny, nx)
    Qxx: np.ndarray  # (ny, nx)
    Qxy: np.ndarray  # (ny, nx)

    def copy(self) -> "State":
        return State(self.f1.copy(), self.f2.copy(), self.phi.copy(),
                     self.Qxx.copy(), self.Qxy.copy())


# --------------------------------------------------------------------------
# Second-order central finite differences on the periodic grid (Sec. III).
# --------------------------------------------------------------------------
def shift(g: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """Value of g at (x + dx, y + dy), periodic."""
    return np.roll(np.roll(g, -dx, axis=-1), -dy, axis=-2)


def ddx(g):
    return 0.5 * (shift(g, 1, 0) - shift(g, -1, 0))


def ddy(g):
    return 0.5 * (shift(g, 0, 1) - shift(g, 0, -1))


def lap(g):
    """Five-point Laplacian."""
    return shift(g, 1, 0) + shift(g, -1, 0) + shift(g, 0, 1) + shift(g, 0, -1) - 4.0 * g


def grad(g):
    """Gradient; a leading axis of length 2 holds (d/dx, d/dy)."""
    return np.stack([ddx(g), ddy(g)])


def div_vector(v):
    """Divergence of a vector field v[i]."""
    return ddx(v[0]) + ddy(v[1])


def div_tensor(s):
    """Vector (div s)_i = sum_j d_j s_ij (divergence on the second index)."""
    return np.stack([ddx(s[i, 0]) + ddy(s[i, 1]) for i in range(2)])


# --------------------------------------------------------------------------
# 2x2 tensor algebra, written literally.
# --------------------------------------------------------------------------
def eye_like(ref):
    out = np.zeros((2, 2) + ref.shape)
    out[0, 0] = 1.0
    out[1, 1] = 1.0
    return out


def matmul(a, b):
    return np.einsum("ik...,kj...->ij...", a, b)


def ddot(a, b):
    """Double contraction a:b = sum_ij a_ij b_ij."""
    return np.einsum("ij...,ij...->...", a, b)


def trace(a):
    return a[0, 0] + a[1, 1]


def transpose(a):
    return np.swapaxes(a, 0, 1)


def q_tensor(Qxx, Qxy):
    """Traceless symmetric Q from its two independent components (Eq. 9)."""
    return np.stack([np.stack([Qxx, Qxy]), np.stack([Qxy, -Qxx])])


def q_from_director(S, theta):
    """Q = 2 S (p p - I/2) with p = (cos theta, sin theta)  (Sec. II, Eq. 9)."""
    p = np.stack([np.cos(theta), np.sin(theta)])
    pp = np.einsum("i...,j...->ij...", p, p)
    return 2.0 * S * (pp - 0.5 * eye_like(np.asarray(theta)))


# --------------------------------------------------------------------------
# Free energies, chemical potential, molecular field (Sec. II).
# --------------------------------------------------------------------------
def double_well(phi):
    """f(phi) = phi^2 (1 - phi)^2 (Sec. II, after Eq. 2)."""
    return phi ** 2 * (1.0 - phi) ** 2


def double_well_prime(phi):
    """f'(phi) = 2 phi (1 - phi)(1 - 2 phi), the derivative of double_well."""
    return 2.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi)


def chemical_potential(phi, p: Params):
    """mu = A_ch f'(phi) - kappa lap(phi)  (Sec. II, Eq. 2)."""
    return p.A_ch * double_well_prime(phi) - p.kappa * lap(phi)


def ldg_derivative(Q, p: Params):
    """Functional derivative dF/dQ_ij of Eq. (8), every Q_ij independent:
    A Q + B Q.Q + C Q.Q.Q - K lap(Q).  (d Tr(Q^n)/dQ_ij = n (Q^{n-1})_ji.)"""
    Q2 = matmul(Q, Q)
    Q3 = matmul(Q2, Q)
    lapQ = np.stack([np.stack([lap(Q[i, j]) for j in range(2)]) for i in range(2)])
    return p.A_Q * Q + p.B_Q * Q2 + p.C_Q * Q3 - p.K * lapQ


def molecular_field(Q, p: Params):
    """H = -dF/dQ + (I/2) Tr(dF/dQ)  (Sec. II, Eq. 7)."""
    dF = ldg_derivative(Q, p)
    return -dF + 0.5 * eye_like(Q[0, 0]) * trace(dF)


def grad_tensor(Q):
    """dQ[k, i, j] = d_k Q_ij."""
    return np.stack([np.stack([np.stack([d(Q[i, j]) for j in range(2)])
                               for i in range(2)]) for d in (ddx, ddy)])


def elastic_stress(Q, H, p: Params):
    """Elastic stress of the Sec. II display (after Eq. 6):

    sigma = -lam H.P - lam P.H + 2 lam P (Q:H) - (grad Q).dF/d(grad Q) + Q.H - H.Q,
    P = Q + I/2, with ((grad Q).dF/d(grad Q))_ij = K sum_kl d_i Q_kl d_j Q_kl
    for the Frank term (K/2)|grad Q|^2 of Eq. (8).
    """
    I = eye_like(Q[0, 0])
    P = Q + 0.5 * I
    QH = ddot(Q, H)
    dQ = grad_tensor(Q)
    T = p.K * np.einsum("ikl...,jkl...->ij...", dQ, dQ)
    return (-p.lam * matmul(H, P) - p.lam * matmul(P, H) + 2.0 * p.lam * P * QH
            - T + matmul(Q, H) - matmul(H, Q))


def capillary_force(phi, mu):
    """F_ch = mu grad(phi) - grad(phi mu)  (Sec. II, Eq. 10)."""
    return mu * grad(phi) - grad(phi * mu)


def forces(phi, Q, p: Params):
    """Non-drag body forces on each fluid (Sec. II, Eq. 4-5):
    G1 = F_active + F_elastic + phi F_ch,  G2 = (1 - phi) F_ch,
    with F_active = div(zeta phi Q) and F_elastic = div(sigma_el)."""
    mu = chemical_potential(phi, p)
    H = molecular_field(Q, p)
    sig = elastic_stress(Q, H, p)
    F_el = div_tensor(sig)
    F_act = div_tensor(p.zeta * phi * Q)
    F_ch = capillary_force(phi, mu)
    G1 = F_act + F_el + phi * F_ch
    G2 = (1.0 - phi) * F_ch
    return G1, G2


# --------------------------------------------------------------------------
# Lattice Boltzmann pieces (Sec. III).
# --------------------------------------------------------------------------
def moments(f):
    """Density rho = sum_i f_i and bare momentum m = sum_i c_i f_i."""
    rho = f.sum(axis=0)
    m = np.einsum("ia,i...->a...", CI.astype(np.float64), f)
    return rho, m


def drag_coefficient(phi, p: Params):
    """g = gamma phi (1 - phi) of F_drag = g (u2 - u1) (Sec. II)."""
    return p.gamma * phi * (1.0 - phi)


def velocities(rho1, m1, rho2, m2, G1, G2, phi, p: Params):
    """Guo velocities with the drag taken implicitly.

    Guo forcing uses u_k = (m_k + F_k/2)/rho_k with the total force
    F_1 = G1 + g (u2 - u1), F_2 = G2 - g (u2 - u1).  Written out this is, per
    site and per Cartesian component, the linear system
        [[rho1 + g/2, -g/2], [-g/2, rho2 + g/2]] [u1, u2] = [m1 + G1/2, m2 + G2/2],
    solved here with a library solver.  Returns u1, u2, F1, F2.
    """
    g = drag_coefficient(phi, p)
    a = 0.5 * g
    A = np.empty(phi.shape + (2, 2))
    A[..., 0, 0] = rho1 + a
    A[..., 0, 1] = -a
    A[..., 1, 0] = -a
    A[..., 1, 1] = rho2 + a
    rhs = np.empty(phi.shape + (2, 2))      # (..., fluid, component)
    rhs[..., 0, :] = np.moveaxis(m1 + 0.5 * G1, 0, -1)
    rhs[..., 1, :] = np.moveaxis(m2 + 0.5 * G2, 0, -1)
    sol = np.linalg.solve(A, rhs)
    u1 = np.moveaxis(sol[..., 0, :], -1, 0)
    u2 = np.moveaxis(sol[..., 1, :], -1, 0)
    F1 = G1 + g * (u2 - u1)
    F2 = G2 - g * (u2 - u1)
    return u1, u2, F1, F2


def equilibrium(rho, u):
    """Second-order D2Q9 equilibrium f_i^eq = w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs4) - u^2/(2 cs2)]."""
    cu = np.einsum("ia,a...->i...", CI.astype(np.float64), u)
    uu = (u * u).sum(axis=0)
    w = WI.reshape((9,) + (1,) * rho.ndim)
    return w * rho * (1.0 + cu / CS2 + 0.5 * cu ** 2 / CS2 ** 2 - 0.5 * uu / CS2)


def guo_source(u, F, tau):
    """Guo forcing term (1 - 1/(2 tau)) w_i [(c_i - u)/cs2 + (c_i.u) c_i/cs4].F."""
    c = CI.astype(np.float64)
    cu = np.einsum("ia,a...->i...", c, u)
    cF = np.einsum("ia,a...->i...", c, F)
    uF = (u * F).sum(axis=0)
    w = WI.reshape((9,) + (1,) * uF.ndim)
    return (1.0 - 0.5 / tau) * w * ((cF - uF) / CS2 + cu * cF / CS2 ** 2)


def collide(f, rho, u, F, tau):
    """BGK relaxation plus Guo source: f* = f - (f - f^eq)/tau + S."""
    return f - (f - equilibrium(rho, u)) / tau + guo_source(u, F, tau)


def stream(fs):
    """Periodic streaming f_i(x + c_i, t + 1) = f*_i(x, t)."""
    out = np.empty_like(fs)
    for i in range(9):
        out[i] = shift(fs[i], -CI[i, 0], -CI[i, 1])
    return out


# --------------------------------------------------------------------------
# Finite-difference sub-steps (Sec. II Eq. 3, 11, 12; Sec. III).
# --------------------------------------------------------------------------
def velocity_gradient(u):
    """W_ij = d_j u_i."""
    return np.stack([np.stack([ddx(u[i]), ddy(u[i])]) for i in range(2)])


def corotation(Wg, Q, p: Params):
    """S(grad u, Q) = (lam E + Om).P + P.(lam E - Om) - 2 lam P (Q : grad u)
    with E = (W + W^T)/2, Om = (W - W^T)/2, P = Q + I/2  (Sec. II, Eq. 12)."""
    E = 0.5 * (Wg + transpose(Wg))
    Om = 0.5 * (Wg - transpose(Wg))
    P = Q + 0.5 * eye_like(Q[0, 0])
    return (matmul(p.lam * E + Om, P) + matmul(P, p.lam * E - Om)
            - 2.0 * p.lam * P * ddot(Q, Wg))


def traceless_symmetric(a):
    """Projection onto traceless symmetric 2x2 tensors; returns (xx, xy)."""
    return 0.5 * (a[0, 0] - a[1, 1]), 0.5 * (a[0, 1] + a[1, 0])


def mixture_velocity(phi, u1, u2):
    """Barycentric velocity u_c = phi u1 + (1 - phi) u2 (Sec. II; Sec. IV, Eq. 13)."""
    return phi * u1 + (1.0 - phi) * u2


def ch_rate(phi, u1, u2, p: Params):
    """d phi/dt = -div(phi u_c) + M lap(mu)  (Sec. II, Eq. 1 and 3)."""
    uc = mixture_velocity(phi, u1, u2)
    return -div_vector(phi * uc) + p.M * lap(chemical_potential(phi, p))


def be_rate(Q, u1, p: Params):
    """d Q/dt = -(u1.grad) Q + S(grad u1, Q) + Gamma_Q H  (Sec. II, Eq. 11)."""
    dQ = grad_tensor(Q)
    adv = -(u1[0] * dQ[0] + u1[1] * dQ[1])
    S = corotation(velocity_gradient(u1), Q, p)
    return adv + S + p.Gamma_Q * molecular_field(Q, p)


def substeps(phi, Qxx, Qxy, u1, u2, p: Params):
    """n_sub forward-Euler updates of phi and Q with dt_fd = dt / n_sub and the
    velocities held fixed (Sec. III: five FD updates share one lattice step)."""
    dt = p.dt / p.n_sub
    for _ in range(p.n_sub):
        Q = q_tensor(Qxx, Qxy)
        dphi = ch_rate(phi, u1, u2, p)
        dQxx, dQxy = traceless_symmetric(be_rate(Q, u1, p))
        phi = phi + dt * dphi
        Qxx = Qxx + dt * dQxx
        Qxy = Qxy + dt * dQxy
    return phi, Qxx, Qxy


# --------------------------------------------------------------------------
# One coupled lattice time step.
# --------------------------------------------------------------------------
def macro(state: State, p: Params):
    """Densities, Guo velocities and total forces of the current state."""
    Q = q_tensor(state.Qxx, state.Qxy)
    G1, G2 = forces(state.phi, Q, p)
    rho1, m1 = moments(state.f1)
    rho2, m2 = moments(state.f2)
    u1, u2, F1, F2 = velocities(rho1, m1, rho2, m2, G1, G2, state.phi, p)
    return dict(rho1=rho1, rho2=rho2, m1=m1, m2=m2, u1=u1, u2=u2,
                F1=F1, F2=F2, G1=G1, G2=G2)


def step(state: State, p: Params) -> State:
    """Advance (f1, f2, phi, Q) from time n to n + 1.

    1. forces from (phi^n, Q^n); 2. moments and implicit-drag Guo velocities;
    3. BGK + Guo collision and periodic streaming of both fluids;
    4. n_sub Cahn-Hilliard / Beris-Edwards sub-steps with those velocities.
    """
    mc = macro(state, p)
    f1 = stream(collide(state.f1, mc["rho1"], mc["u1"], mc["F1"], p.tau1))
    f2 = stream(collide(state.f2, mc["rho2"], mc["u2"], mc["F2"], p.tau2))
    phi, Qxx, Qxy = substeps(state.phi, state.Qxx, state.Qxy, mc["u1"], mc["u2"], p)
    return State(f1, f2, phi, Qxx, Qxy)


def run(state: State, p: Params, n: int) -> State:
    for _ in range(n):
        state = step(state, p)
    return state


def state_from_fields(phi, Qxx, Qxy, p: Params, u1=None, u2=None) -> State:
    """Populations at equilibrium with rest densities rho1, rho2 and the given
    velocities (zero by default, Sec. III initial condition)."""
    z = np.zeros((2,) + phi.shape)
    u1 = z if u1 is None else u1
    u2 = z if u2 is None else u2
    f1 = equilibrium(np.full(phi.shape, p.rho1), u1)
    f2 = equilibrium(np.full(phi.shape, p.rho2), u2)
    return State(f1, f2, np.array(phi, dtype=np.float64),
                 np.array(Qxx, dtype=np.float64), np.array(Qxy, dtype=np.float64))


# --------------------------------------------------------------------------
# Conserved sums (FP64), used by the invariance checks.
# --------------------------------------------------------------------------
def conserved(state: State, p: Params):
    """[sum phi, sum rho1, sum rho2, sum (m1+m2)_x, sum (m1+m2)_y,
        sum (G1+G2)_x, sum (G1+G2)_y, number of non-finite values]."""
    rho1, m1 = moments(state.f1)
    rho2, m2 = moments(state.f2)
    G1, G2 = forces(state.phi, q_tensor(state.Qxx, state.Qxy), p)
    allv = np.concatenate([state.f1.ravel(), state.f2.ravel(), state.phi.ravel(),
                           state.Qxx.ravel(), state.Qxy.ravel()])
    return np.array([state.phi.sum(), rho1.sum(), rho2.sum(),
                     (m1 + m2)[0].sum(), (m1 + m2)[1].sum(),
                     (G1 + G2)[0].sum(), (G1 + G2)[1].sum(),
                     float(np.count_nonzero(~np.isfinite(allv)))])


# --------------------------------------------------------------------------
# Observables (Sec. IV).
# --------------------------------------------------------------------------
def shell_geometry(nx: int, ny: int):
    """Shell index of every FFT mode (Sec. IV, Eq. 27 shells k - 1/2 <= k' < k + 1/2).

    Mode (n_x, n_y) (signed integers, numpy fftfreq order) has wavevector
    k = 2 pi (n_x/nx, n_y/ny).  Shells have width k0 = 2 pi / m, m = min(nx, ny):
    with r = |k|/k0 = sqrt((n_x m/nx)^2 + (n_y m/ny)^2) the mode lies in shell
    floor(r + 1/2).  r is formed from the integer mode numbers with separately
    rounded operations so that modes exactly on a shell boundary are assigned
    reproducibly.  Shells 0 .. m/2 are kept; corner modes beyond are dropped.
    Returns (r, shell, n_shell, k0).
    """
    m = min(nx, ny)
    sx = np.rint(np.fft.fftfreq(nx) * nx)
    sy = np.rint(np.fft.fftfreq(ny) * ny)
    tx = sx * m / nx
    ty = sy * m / ny
    r = np.sqrt(tx[None, :] * tx[None, :] + ty[:, None] * ty[:, None])
    shell = np.floor(r + 0.5).astype(np.int64)
    n_shell = m // 2 + 1
    k0 = 2.0 * np.pi / m
    return r, shell, n_shell, k0


def fourier(g):
    """Normalised transform g_hat(k) = (1/N) sum_x g(x) exp(-i k.x), N = nx*ny."""
    return np.fft.fft2(g) / g.size


def shell_sum(values, nx, ny):
    _, shell, n_shell, _ = shell_geometry(nx, ny)
    out = np.zeros(n_shell)
    keep = shell < n_shell
    np.add.at(out, shell[keep], values[keep])
    return out


def shell_counts(nx, ny):
    return shell_sum(np.ones((ny, nx)), nx, ny)


def structure_factor(phi):
    """Shell sums of |phi_hat(k)|^2 of delta phi = phi - <phi> (Sec. IV, Eq. 24, 27)."""
    ny, nx = phi.shape
    ph = fourier(phi - phi.mean())
    return shell_sum(np.abs(ph) ** 2, nx, ny)


def length_scale(phi):
    """L(t) = sum_k Phi(k) / sum_k k Phi(k), Phi(k) = 1/2 shell sum |phi_hat|^2
    over shells m >= 1 with k_m = m k0 (Sec. IV, Eq. 27)."""
    ny, nx = phi.shape
    _, _, n_shell, k0 = shell_geometry(nx, ny)
    Phi = 0.5 * structure_factor(phi)
    km = k0 * np.arange(n_shell)
    num = Phi[1:].sum()
    den = (km[1:] * Phi[1:]).sum()
    return num / den if den > 0 else 0.0


def energy_spectrum(uc):
    """E_kin(k) = 1/2 shell sum of u_hat_c(k) . u_hat_c(-k) (Sec. IV, Eq. 22) and
    the total E = 1/2 sum_k |u_hat_c|^2 = <|u_c|^2>/2 over all modes (Eq. 29)."""
    ny, nx = uc.shape[1:]
    ux = fourier(uc[0])
    uy = fourier(uc[1])
    dens = 0.5 * (np.abs(ux) ** 2 + np.abs(uy) ** 2)
    return shell_sum(dens, nx, ny), dens.sum()


def vorticity(u):
    """omega = d_x u_y - d_y u_x (Sec. IV, Eq. 15)."""
    return ddx(u[1]) - ddy(u[0])


def rms(a):
    return float(np.sqrt(np.mean(a * a)))


def phase_difference(state: State, p: Params):
    """[rms|u1 - u2|, rms(w1 - w2), rms|u1|, rms|u_c|, rms w1, rms w_c] of the
    current state's Guo velocities (Sec. IV, Fig. 8 quantities)."""
    mc = macro(state, p)
    u1, u2 = mc["u1"], mc["u2"]
    uc = mixture_velocity(state.phi, u1, u2)
    du = u1 - u2
    w1, w2, wc = vorticity(u1), vorticity(u2), vorticity(uc)
    return np.array([np.sqrt(np.mean((du * du).sum(axis=0))), rms(w1 - w2),
                     np.sqrt(np.mean((u1 * u1).sum(axis=0))),
                     np.sqrt(np.mean((uc * uc).sum(axis=0))), rms(w1), rms(wc)])


def std_phi(phi):
    """Standard deviation Delta of the concentration field (Sec. IV, Fig. 3)."""
    return float(np.sqrt(np.mean((phi - phi.mean()) ** 2)))


# --------------------------------------------------------------------------
# Correlations, defects, energy densities, Reynolds number (Sec. IV).
# --------------------------------------------------------------------------
def displacement_shells(nx: int, ny: int):
    """Shell of every displacement r = (r_x, r_y) of the periodic grid, taken
    as its minimum image (signed r_x in numpy fftfreq order) in lattice
    units: floor(|r| + 1/2), shells 0 .. min(nx, ny)/2 (longer displacements
    are dropped).  Returns (shell, n_shell); shell has shape (ny, nx) indexed
    by the displacement's array position (dy, dx)."""
    sx = np.rint(np.fft.fftfreq(nx) * nx)
    sy = np.rint(np.fft.fftfreq(ny) * ny)
    r = np.sqrt(sx[None, :] * sx[None, :] + sy[:, None] * sy[:, None])
    return np.floor(r + 0.5).astype(np.int64), min(nx, ny) // 2 + 1


def autocorrelation(a):
    """R(r) = < sum_c a_c(x) a_c(x + r) >_x for every displacement r, by the
    definition (one shifted copy per displacement; small grids only).
    a: components (c, ny, nx).  Returns (ny, nx) indexed by (dy, dx)."""
    c, ny, nx = a.shape
    R = np.empty((ny, nx))
    for dy in range(ny):
        ay = np.roll(a, -dy, axis=1)
        for dx in range(nx):
            R[dy, dx] = (a * np.roll(ay, -dx, axis=2)).sum(axis=0).mean()
    return R


def spatial_correlation(a, centred: bool):
    """C(r) = <a(0) . a(r)> / <|a|^2> averaged over the displacements of each
    shell (Sec. IV, spatial correlation functions of u_c, omega_c and Q).
    centred: use delta a = a - <a> (the paper's delta u_c, delta omega_c)."""
    a = np.asarray(a, dtype=np.float64)
    if centred:
        a = a - a.mean(axis=(1, 2), keepdims=True)
    ny, nx = a.shape[1:]
    R = autocorrelation(a)
    shell, n_shell = displacement_shells(nx, ny)
    keep = shell < n_shell
    sums = np.zeros(n_shell)
    counts = np.zeros(n_shell)
    np.add.at(sums, shell[keep], R[keep])
    np.add.at(counts, shell[keep], 1.0)
    return sums / counts / R[0, 0]


def correlation_fields(state: State, p: Params):
    """The three correlated quantities of the current state: u_c (2, ny, nx),
    omega_c (1, ny, nx) and (Q_xx, Q_xy) (2, ny, nx), whose dot product is
    Q:Q / 2 for a traceless symmetric Q (the factor cancels in the ratios)."""
    mc = macro(state, p)
    uc = mixture_velocity(state.phi, mc["u1"], mc["u2"])
    return uc, vorticity(uc)[None], np.stack([state.Qxx, state.Qxy])


def spatial_correlations(state: State, p: Params):
    """[C_uu(r), C_ww(r), C_QQ(r)] shell-averaged (Sec. IV)."""
    uc, wc, q = correlation_fields(state, p)
    return [spatial_correlation(uc, True), spatial_correlation(wc, True),
            spatial_correlation(q, False)]


def time_correlations(then: State, now: State, p: Params):
    """[C_uu(t), C_ww(t), C_QQ(t)] between two states (Sec. IV, temporal
    correlation functions): <a(tau) . a(tau + t)> / <|a(tau)|^2>."""
    out = []
    for a, b in zip(correlation_fields(then, p), correlation_fields(now, p)):
        out.append(float((a * b).sum(axis=0).mean() / (a * a).sum(axis=0).mean()))
    return out


def defect_charges(Qxx, Qxy):
    """Winding-number charge of the director around every plaquette (Sec. IV,
    +-1/2 defects): the plaquette with lower-left site (x, y) is walked
    (x, y) -> (x+1, y) -> (x+1, y+1) -> (x, y+1) -> (x, y); the director angle
    theta = atan2(Q_xy, Q_xx) / 2 changes along each edge by the difference
    wrapped into [-pi/2, pi/2) (a director is a headless line); the summed
    change over 2 pi is the charge.  Returns charges (ny, nx) in halves."""
    th = 0.5 * np.arctan2(Qxy, Qxx)
    loop = [th, np.roll(th, -1, axis=1), np.roll(np.roll(th, -1, axis=1), -1, axis=0),
            np.roll(th, -1, axis=0)]
    total = np.zeros_like(th)
    for k in range(4):
        d = loop[(k + 1) % 4] - loop[k]
        total += (d + 0.5 * np.pi) % np.pi - 0.5 * np.pi
    return np.rint(2.0 * total / (2.0 * np.pi)) / 2.0


def defect_counts(Qxx, Qxy):
    """[number of +1/2, number of -1/2, number of other nonzero charges];
    the defect density of Sec. IV is (n_+ + n_-) / (nx ny)."""
    q = defect_charges(Qxx, Qxy)
    return np.array([np.count_nonzero(q == 0.5), np.count_nonzero(q == -0.5),
                     np.count_nonzero((q != 0) & (np.abs(q) != 0.5))], dtype=np.int64)


def elastic_energy_density(Qxx, Qxy, K):
    """E_elastic = K/2 |grad Q|^2 = K/2 sum_{k,i,j} (d_k Q_ij)^2 with all four
    tensor entries (Q_yy = -Q_xx, Q_yx = Q_xy) and central differences
    (Sec. IV, Fig. 6)."""
    Q = q_tensor(Qxx, Qxy)
    g = 0.0
    for i in range(2):
        for j in range(2):
            g = g + ddx(Q[i, j]) ** 2 + ddy(Q[i, j]) ** 2
    return 0.5 * K * g


def kinetic_energy_density(state: State, p: Params):
    """E_kin = 1/2 rho_c |u_c|^2 with the local total density rho_c = rho1 + rho2
    (Sec. IV, Fig. 6)."""
    mc = macro(state, p)
    uc = mixture_velocity(state.phi, mc["u1"], mc["u2"])
    return 0.5 * (mc["rho1"] + mc["rho2"]) * (uc * uc).sum(axis=0)


def reynolds(state: State, p: Params):
    """Re = rho_c u_c,rms L_a / eta_c, L_a = sqrt(K / |zeta|) (Sec. IV), with
    rho_c = rho1 + rho2 the rest densities, eta_c = eta1 + eta2 and
    eta_k = rho_k (tau_k - 1/2) / 3 in lattice units.  Returns (Re, L_a)."""
    uc_rms = phase_difference(state, p)[3]
    La = np.sqrt(p.K / abs(p.zeta)) if p.zeta != 0 else np.inf
    eta = p.rho1 * (p.tau1 - 0.5) / 3.0 + p.rho2 * (p.tau2 - 0.5) / 3.0
    return (p.rho1 + p.rho2) * uc_rms * La / eta, La
