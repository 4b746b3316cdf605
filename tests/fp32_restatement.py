"""Float32 restatement of the coupled step, independent of the CUDA library.

Test infrastructure: it shows what FP32 arithmetic alone does to the method,
so that the parity bars of the GPU tests rest on evidence a CPU reproduces.
Every array and every constant is numpy float32, so each operation rounds to
FP32 as the kernels do (the order of operations is this file's own, not the
kernels').  The state is held as the kernels hold it: phi as phi - phi_ref and
each population as its deviation d_i = f_i - w_i from the rest equilibrium.

Equations (paper Sec. II-III, with the readings of the FP64 oracle): chemical
potential mu = A_ch f'(phi) - kappa lap(phi) (Eq. 2); H = -(A_Q + C_Q q^2) Q +
K lap(Q) (Eq. 7-8, two components); elastic stress (display after Eq. 6)
reduced to -lam H + 2 lam (Q:H) Q - T + (Q.H - H.Q); active force
div(zeta phi Q); capillary force mu grad(phi) - grad(phi mu) (Eq. 10); G1, G2
(Eq. 4-5); implicit-drag Guo velocities (2x2 Cramer solve); BGK + Guo collision
and pull streaming; n_sub forward-Euler CH / BE sub-steps (Eq. 1, 11-12).
"""
import numpy as np

F = np.float32
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float32)


def _sh(g, dx, dy):
    """g at (x + dx, y + dy), periodic."""
    return np.roll(np.roll(g, -dx, axis=-1), -dy, axis=-2)


def _dx(g):
    return F(0.5) * (_sh(g, 1, 0) - _sh(g, -1, 0))


def _dy(g):
    return F(0.5) * (_sh(g, 0, 1) - _sh(g, 0, -1))


def _lap(g):
    return (_sh(g, 1, 0) + _sh(g, -1, 0)) + (_sh(g, 0, 1) + _sh(g, 0, -1)) - F(4) * g


class Fp32State:
    """d1, d2: (9, ny, nx) population deviations; dphi = phi - phi_ref; a, b = Q_xx, Q_xy."""

    def __init__(self, d1, d2, dphi, a, b):
        self.d1, self.d2, self.dphi, self.a, self.b = (np.asarray(v, dtype=np.float32)
                                                       for v in (d1, d2, dphi, a, b))


def from_oracle(state, phi_ref=0.5):
    """Round an FP64 oracle State into the FP32 deviation form."""
    w = W.astype(np.float64)[:, None, None]
    return Fp32State(state.f1 - w, state.f2 - w, state.phi - phi_ref, state.Qxx, state.Qxy)


def _mu(dphi, p, c):
    """A_ch f'(c + d) as its exact cubic in d = phi - c (coefficients rounded
    once from FP64), minus kappa lap(d)."""
    m0 = F(p.A_ch * (2 * c - 6 * c * c + 4 * c ** 3))
    m1 = F(p.A_ch * (2 - 12 * c + 12 * c * c))
    m2 = F(p.A_ch * (-6 + 12 * c))
    m3 = F(p.A_ch * 4)
    return m0 + dphi * (m1 + dphi * (m2 + dphi * m3)) - F(p.kappa) * _lap(dphi)


def _hg(a, b, p):
    cq = -(F(p.A_Q) + F(p.C_Q) * (a * a + b * b))
    return cq * a + F(p.K) * _lap(a), cq * b + F(p.K) * _lap(b)


def macro(s: Fp32State, p, c=0.5):
    """Densities, Guo velocities and total forces of the FP32 state."""
    a, b, dphi = s.a, s.b, s.dphi
    phi = F(c) + dphi
    mu = _mu(dphi, p, c)
    h, g = _hg(a, b, p)
    dxa, dya, dxb, dyb = _dx(a), _dy(a), _dx(b), _dy(b)
    k2 = F(2 * p.K)
    Txx = k2 * (dxa * dxa + dxb * dxb)
    Tyy = k2 * (dya * dya + dyb * dyb)
    Txy = k2 * (dxa * dya + dxb * dyb)
    qh2 = F(2) * (a * h + b * g)
    anti = F(2) * (a * g - b * h)
    lam = F(p.lam)
    sxx = -lam * h + F(2) * lam * qh2 * a - Txx
    syy = lam * h - F(2) * lam * qh2 * a - Tyy
    sym = -lam * g + F(2) * lam * qh2 * b - Txy
    sxy, syx = sym + anti, sym - anti
    z = F(p.zeta)
    Fel = (_dx(sxx) + _dy(sxy), _dx(syx) + _dy(syy))
    Fact = (z * (_dx(phi * a) + _dy(phi * b)), z * (_dx(phi * b) - _dy(phi * a)))
    Fch = (mu * _dx(dphi) - _dx(phi * mu), mu * _dy(dphi) - _dy(phi * mu))
    G1 = [Fact[k] + Fel[k] + phi * Fch[k] for k in range(2)]
    G2 = [(F(1) - phi) * Fch[k] for k in range(2)]
    cx, cy = CX.astype(np.float32)[:, None, None], CY.astype(np.float32)[:, None, None]
    dr1, dr2 = s.d1.sum(axis=0, dtype=np.float32), s.d2.sum(axis=0, dtype=np.float32)
    m1 = ((cx * s.d1).sum(axis=0, dtype=np.float32), (cy * s.d1).sum(axis=0, dtype=np.float32))
    m2 = ((cx * s.d2).sum(axis=0, dtype=np.float32), (cy * s.d2).sum(axis=0, dtype=np.float32))
    r1 = F(1) + dr1
    r2 = F(1) + dr2
    gd = F(p.gamma) * phi * (F(1) - phi)
    ad = F(0.5) * gd
    det = r1 * r2 + ad * (r1 + r2)
    u1, u2, F1, F2 = [], [], [], []
    for k in range(2):
        b1 = m1[k] + F(0.5) * G1[k]
        b2 = m2[k] + F(0.5) * G2[k]
        v1 = ((r2 + ad) * b1 + ad * b2) / det
        v2 = (ad * b1 + (r1 + ad) * b2) / det
        u1.append(v1)
        u2.append(v2)
        F1.append(G1[k] + gd * (v2 - v1))
        F2.append(G2[k] - gd * (v2 - v1))
    return dict(dr1=dr1, dr2=dr2, u1=np.stack(u1), u2=np.stack(u2), F1=F1, F2=F2)


def _collide_stream(d, dr, u, Fv, tau):
    om = F(1.0 / tau)
    guo = F(1.0 - 0.5 / tau)
    rho = F(1) + dr
    usq = F(1.5) * (u[0] * u[0] + u[1] * u[1])
    uF = F(3) * (u[0] * Fv[0] + u[1] * Fv[1])
    out = np.empty_like(d)
    for i in range(9):
        cx, cy = F(CX[i]), F(CY[i])
        cu = cx * u[0] + cy * u[1]
        cF = cx * Fv[0] + cy * Fv[1]
        deq = W[i] * (dr + rho * (cu * (F(3) + F(4.5) * cu) - usq))
        src = guo * W[i] * (F(3) * cF - uF + F(9) * cu * cF)
        post = d[i] - om * (d[i] - deq) + src
        out[i] = _sh(post, -int(CX[i]), -int(CY[i]))
    return out


def step(s: Fp32State, p, c=0.5) -> Fp32State:
    """One coupled step n -> n+1 in FP32 (same stages and order as the oracle)."""
    mc = macro(s, p, c)
    d1 = _collide_stream(s.d1, mc["dr1"], mc["u1"], mc["F1"], p.tau1)
    d2 = _collide_stream(s.d2, mc["dr2"], mc["u2"], mc["F2"], p.tau2)
    u1, u2 = mc["u1"], mc["u2"]
    dt = F(p.dt / p.n_sub)
    dphi, a, b = s.dphi, s.a, s.b
    Wxx, Wxy, Wyx, Wyy = _dx(u1[0]), _dy(u1[0]), _dx(u1[1]), _dy(u1[1])
    trE = Wxx + Wyy
    e1 = F(0.5) * (Wxx - Wyy)
    exy = F(0.5) * (Wxy + Wyx)
    w2 = Wxy - Wyx
    lam = F(p.lam)
    for _ in range(p.n_sub):
        phi = F(c) + dphi
        uc = [phi * u1[k] + (F(1) - phi) * u2[k] for k in range(2)]
        divJ = _dx(phi * uc[0]) + _dy(phi * uc[1])
        rphi = -divJ + F(p.M) * _lap(_mu(dphi, p, c))
        h, g = _hg(a, b, p)
        qe2 = F(4) * (a * e1 + b * exy)
        ra = (-(u1[0] * _dx(a) + u1[1] * _dy(a)) + lam * (trE * a + e1 - qe2 * a) + w2 * b
              + F(p.Gamma_Q) * h)
        rb = (-(u1[0] * _dx(b) + u1[1] * _dy(b)) + lam * (trE * b + exy - qe2 * b) - w2 * a
              + F(p.Gamma_Q) * g)
        dphi, a, b = dphi + dt * rphi, a + dt * ra, b + dt * rb
    return Fp32State(d1, d2, dphi, a, b)
