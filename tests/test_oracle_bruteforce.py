"""Brute-force cross-check of the oracle's whole step on tiny grids (CPU only).

The step is written out again here site by site with explicit periodic index
arithmetic and with the 2x2 tensor algebra reduced by hand to its two
independent components (Q = [[a, b], [b, -a]], H = [[h, g], [g, -h]]):

* Q.Q = (a^2 + b^2) I, so H = -(A_Q + C_Q q^2) Q + K lap Q (Eq. 7-8);
* H.P + P.H = H + (Q:H) I with P = Q + I/2, so the elastic stress of Sec. II
  becomes -lam H + 2 lam (Q:H) Q - T + (Q.H - H.Q), the last term being
  antisymmetric with xy entry 2 (a g - b h);
* S of Eq. (12) has traceless-symmetric part
  lam [tr(E) Q + E0 - 2 (Q:E0) Q] + (Om.Q - Q.Om).

Agreement with the oracle's literal matrix algebra pins both the oracle's
index conventions (roll directions, transposes) and this reduction.
"""
import numpy as np
import pytest

from oracle import twofluid as O
from paper_2511_00445_gb300 import inputs

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
WW = [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36]


def bf_step(f1, f2, phi, Qxx, Qxy, p):
    ny, nx = phi.shape

    def at(a, x, y):
        return a[y % ny, x % nx]

    def D(a, x, y):
        return 0.5 * (at(a, x + 1, y) - at(a, x - 1, y)), 0.5 * (at(a, x, y + 1) - at(a, x, y - 1))

    def L(a, x, y):
        return at(a, x + 1, y) + at(a, x - 1, y) + at(a, x, y + 1) + at(a, x, y - 1) - 4 * at(a, x, y)

    def mu_field(ph):
        mu = np.zeros_like(ph)
        for y in range(ny):
            for x in range(nx):
                c = ph[y, x]
                mu[y, x] = p.A_ch * 2 * c * (1 - c) * (1 - 2 * c) - p.kappa * L(ph, x, y)
        return mu

    def h_field(a, b):
        h = np.zeros_like(a)
        g = np.zeros_like(a)
        for y in range(ny):
            for x in range(nx):
                q2 = a[y, x] ** 2 + b[y, x] ** 2
                h[y, x] = -(p.A_Q + p.C_Q * q2) * a[y, x] + p.K * L(a, x, y)
                g[y, x] = -(p.A_Q + p.C_Q * q2) * b[y, x] + p.K * L(b, x, y)
        return h, g

    # ---- forces from (phi^n, Q^n)
    a, b = Qxx, Qxy
    mu = mu_field(phi)
    h, g = h_field(a, b)
    sxx, sxy, syx, syy = (np.zeros_like(a) for _ in range(4))
    for y in range(ny):
        for x in range(nx):
            dxa, dya = D(a, x, y)
            dxb, dyb = D(b, x, y)
            Txx = 2 * p.K * (dxa * dxa + dxb * dxb)
            Tyy = 2 * p.K * (dya * dya + dyb * dyb)
            Txy = 2 * p.K * (dxa * dya + dxb * dyb)
            QH = 2 * (a[y, x] * h[y, x] + b[y, x] * g[y, x])
            A = 2 * (a[y, x] * g[y, x] - b[y, x] * h[y, x])
            sxx[y, x] = -p.lam * h[y, x] + 2 * p.lam * QH * a[y, x] - Txx
            syy[y, x] = p.lam * h[y, x] - 2 * p.lam * QH * a[y, x] - Tyy
            sxy[y, x] = -p.lam * g[y, x] + 2 * p.lam * QH * b[y, x] - Txy + A
            syx[y, x] = -p.lam * g[y, x] + 2 * p.lam * QH * b[y, x] - Txy - A
    pa, pb, pm = phi * a, phi * b, phi * mu
    G1 = np.zeros((2, ny, nx))
    G2 = np.zeros((2, ny, nx))
    for y in range(ny):
        for x in range(nx):
            c = phi[y, x]
            dphi = D(phi, x, y)
            dpm = D(pm, x, y)
            Fch = [mu[y, x] * dphi[k] - dpm[k] for k in range(2)]
            Fax = p.zeta * (D(pa, x, y)[0] + D(pb, x, y)[1])
            Fay = p.zeta * (D(pb, x, y)[0] - D(pa, x, y)[1])
            Fex = D(sxx, x, y)[0] + D(sxy, x, y)[1]
            Fey = D(syx, x, y)[0] + D(syy, x, y)[1]
            G1[:, y, x] = [Fax + Fex + c * Fch[0], Fay + Fey + c * Fch[1]]
            G2[:, y, x] = [(1 - c) * Fch[0], (1 - c) * Fch[1]]

    # ---- moments, Cramer solve of the implicit drag, collide, stream
    out1 = np.zeros_like(f1)
    out2 = np.zeros_like(f2)
    U1 = np.zeros((2, ny, nx))
    U2 = np.zeros((2, ny, nx))
    for y in range(ny):
        for x in range(nx):
            r1 = sum(f1[i, y, x] for i in range(9))
            r2 = sum(f2[i, y, x] for i in range(9))
            m1 = [sum(c[i] * f1[i, y, x] for i in range(9)) for c in (CX, CY)]
            m2 = [sum(c[i] * f2[i, y, x] for i in range(9)) for c in (CX, CY)]
            gd = p.gamma * phi[y, x] * (1 - phi[y, x])
            ad = 0.5 * gd
            det = (r1 + ad) * (r2 + ad) - ad * ad
            u1, u2 = [0, 0], [0, 0]
            for k in range(2):
                b1 = m1[k] + 0.5 * G1[k, y, x]
                b2 = m2[k] + 0.5 * G2[k, y, x]
                u1[k] = ((r2 + ad) * b1 + ad * b2) / det
                u2[k] = (ad * b1 + (r1 + ad) * b2) / det
            U1[:, y, x] = u1
            U2[:, y, x] = u2
            F1 = [G1[k, y, x] + gd * (u2[k] - u1[k]) for k in range(2)]
            F2 = [G2[k, y, x] - gd * (u2[k] - u1[k]) for k in range(2)]
            for f, out, rho, u, F, tau in ((f1, out1, r1, u1, F1, p.tau1),
                                           (f2, out2, r2, u2, F2, p.tau2)):
                uu = u[0] * u[0] + u[1] * u[1]
                for i in range(9):
                    cu = CX[i] * u[0] + CY[i] * u[1]
                    feq = WW[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
                    src = (1 - 0.5 / tau) * WW[i] * (
                        3 * ((CX[i] - u[0]) * F[0] + (CY[i] - u[1]) * F[1])
                        + 9 * cu * (CX[i] * F[0] + CY[i] * F[1]))
                    out[i, (y + CY[i]) % ny, (x + CX[i]) % nx] = f[i, y, x] - (f[i, y, x] - feq) / tau + src

    # ---- sub-steps with frozen velocities
    dt = 1.0 / p.n_sub
    ph, a, b = phi.copy(), Qxx.copy(), Qxy.copy()
    for _ in range(p.n_sub):
        mu = mu_field(ph)
        h, g = h_field(a, b)
        Jx = ph * (ph * U1[0] + (1 - ph) * U2[0])
        Jy = ph * (ph * U1[1] + (1 - ph) * U2[1])
        nph, na, nb = ph.copy(), a.copy(), b.copy()
        for y in range(ny):
            for x in range(nx):
                divJ = D(Jx, x, y)[0] + D(Jy, x, y)[1]
                nph[y, x] = ph[y, x] + dt * (-divJ + p.M * L(mu, x, y))
                Wxx, Wxy = D(U1[0], x, y)
                Wyx, Wyy = D(U1[1], x, y)
                trE = Wxx + Wyy
                e1 = 0.5 * (Wxx - Wyy)
                exy = 0.5 * (Wxy + Wyx)
                w = 0.5 * (Wxy - Wyx)
                A, B = a[y, x], b[y, x]
                QE = 2 * (A * e1 + B * exy)
                ux, uy = U1[0, y, x], U1[1, y, x]
                dax, day = D(a, x, y)
                dbx, dby = D(b, x, y)
                ra = -(ux * dax + uy * day) + p.lam * (trE * A + e1 - 2 * QE * A) + 2 * B * w \
                    + p.Gamma_Q * h[y, x]
                rb = -(ux * dbx + uy * dby) + p.lam * (trE * B + exy - 2 * QE * B) - 2 * A * w \
                    + p.Gamma_Q * g[y, x]
                na[y, x] = A + dt * ra
                nb[y, x] = B + dt * rb
        ph, a, b = nph, na, nb
    return out1, out2, ph, a, b


@pytest.mark.parametrize("nx,ny,seed", [(5, 4, 0), (3, 6, 1), (4, 4, 2)])
def test_oracle_step_matches_bruteforce(nx, ny, seed):
    p = O.Params(nx=nx, ny=ny, zeta=0.3, lam=0.9, K=0.2, gamma=0.3, tau1=0.9, tau2=1.3)
    up, ut = inputs.initial_draws(seed, nx, ny)
    phi = 0.5 + 0.3 * (2 * up - 1)
    Q = O.q_from_director(0.4, np.pi * ut)
    rng = np.random.default_rng(seed)
    u1 = 0.02 * rng.standard_normal((2, ny, nx))
    u2 = 0.02 * rng.standard_normal((2, ny, nx))
    s = O.state_from_fields(phi, Q[0, 0], Q[0, 1], p, u1, u2)
    s.f1 += 1e-3 * rng.standard_normal(s.f1.shape)   # off-equilibrium parts
    s.f2 += 1e-3 * rng.standard_normal(s.f2.shape)
    want = bf_step(s.f1, s.f2, s.phi, s.Qxx, s.Qxy, p)
    got = O.step(s, p)
    for w, g_ in zip(want, (got.f1, got.f2, got.phi, got.Qxx, got.Qxy)):
        assert np.allclose(g_, w, rtol=0, atol=1e-14)
