// Device helpers shared by the step and observation kernels.
//
// Algebra used below (2D, Q = [[a, b], [b, -a]], H = [[h, g], [g, -h]]):
//  * Q.Q = (a^2 + b^2) I, hence dF/dQ of Eq. (8) is (A_Q + C_Q q^2) Q - K lap Q
//    (the B term is a multiple of I and is removed by Eq. 7):
//      H = -(A_Q + C_Q q^2) Q + K lap Q.
//  * H.P + P.H = H + (Q:H) I for P = Q + I/2, so the elastic stress of Sec. II
//    (display after Eq. 6) is
//      sigma = -lam H + 2 lam (Q:H) Q - T + (Q.H - H.Q),
//    T_ij = 2K (d_i a d_j a + d_i b d_j b), Q:H = 2(a h + b g), and Q.H - H.Q
//    antisymmetric with xy entry 2(a g - b h).
//  * The capillary force mu grad(phi) - grad(phi mu) of Eq. (10) in central
//    differences equals [phi_+ (mu_0 - mu_+) - phi_- (mu_0 - mu_-)] / 2 per
//    axis, which needs only differences of mu.
//  * The traceless-symmetric part of S (Eq. 12) with W_ij = d_j u_i,
//    E0 = traceless part of E, w = (W_xy - W_yx)/2 is
//      lam [tr(E) Q + E0 - 2 (Q:E0) Q] + 2 w [[b, -a], [-a, -b]].
#pragma once

#include "tf_internal.h"

namespace tfd {

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Fluid-1 stress (elastic + active, zeta phi Q) and chemical potential at a
// site from the 5-point neighbourhoods of d = phi - phi_ref, a = Q_xx, b = Q_xy.
struct SiteStress {
    float mu, sxx, sxy, syx, syy;
};

__device__ __forceinline__ SiteStress site_stress(
    const DevParams& P,
    float d, float de, float dw, float dn, float ds,
    float a, float ae, float aw, float an, float as,
    float b, float be, float bw, float bn, float bs) {
    SiteStress r;
    const float lapd = (de + dw) + (dn + ds) - 4.f * d;
    r.mu = P.mu0 + d * (P.mu1 + d * (P.mu2 + d * P.mu3)) - P.kappa * lapd;
    const float lapa = (ae + aw) + (an + as) - 4.f * a;
    const float lapb = (be + bw) + (bn + bs) - 4.f * b;
    const float dxa = 0.5f * (ae - aw), dya = 0.5f * (an - as);
    const float dxb = 0.5f * (be - bw), dyb = 0.5f * (bn - bs);
    const float cq = -(P.A_Q + P.C_Q * (a * a + b * b));
    const float h = cq * a + P.K * lapa;
    const float g = cq * b + P.K * lapb;
    const float k2 = 2.f * P.K;
    const float Txx = k2 * (dxa * dxa + dxb * dxb);
    const float Tyy = k2 * (dya * dya + dyb * dyb);
    const float Txy = k2 * (dxa * dya + dxb * dyb);
    const float l2qh = 4.f * P.lam * (a * h + b * g);   // 2 lam (Q:H)
    const float anti = 2.f * (a * g - b * h);
    const float phv = P.phi_ref + d;
    const float za = P.zeta * phv * a, zb = P.zeta * phv * b;
    r.sxx = -P.lam * h + l2qh * a - Txx + za;
    r.syy = P.lam * h - l2qh * a - Tyy - za;
    const float sym = -P.lam * g + l2qh * b - Txy + zb;
    r.sxy = sym + anti;
    r.syx = sym - anti;
    return r;
}

// Non-drag forces G1 (fluid 1) and G2 (fluid 2) at a site from the stress
// and mu at the four neighbours and phi around the site.
struct SiteForce {
    float G1x, G1y, G2x, G2y;
};

__device__ __forceinline__ SiteForce site_force(
    const DevParams& P, float d, float de, float dw, float dn, float ds,
    float m0, float me, float mw, float mn, float ms,
    float sxx_e, float sxx_w, float sxy_n, float sxy_s,
    float syx_e, float syx_w, float syy_n, float syy_s) {
    const float c = P.phi_ref;
    const float fchx = 0.5f * (c * (mw - me) + de * (m0 - me) - dw * (m0 - mw));
    const float fchy = 0.5f * (c * (ms - mn) + dn * (m0 - mn) - ds * (m0 - ms));
    const float phv = c + d;
    const float om = (1.f - c) - d;
    SiteForce F;
    F.G1x = 0.5f * ((sxx_e - sxx_w) + (sxy_n - sxy_s)) + phv * fchx;
    F.G1y = 0.5f * ((syx_e - syx_w) + (syy_n - syy_s)) + phv * fchy;
    F.G2x = om * fchx;
    F.G2y = om * fchy;
    return F;
}

// Moments of nine deviations d_i = f_i - w_i: density deviation and momentum.
__device__ __forceinline__ void moments(const float (&f)[9], float& drho, float& mx, float& my) {
    drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    mx = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    my = (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
}

// Implicit-drag Guo velocities: solve
//   (rho1 + g/2) u1 - g/2 u2 = m1 + G1/2,  -g/2 u1 + (rho2 + g/2) u2 = m2 + G2/2
// and return the total forces F1 = G1 + g (u2 - u1), F2 = G2 - g (u2 - u1).
struct Velocities {
    float u1x, u1y, u2x, u2y, F1x, F1y, F2x, F2y;
};

__device__ __forceinline__ Velocities drag_solve(const DevParams& P, float phv, float rho1,
                                                 float m1x, float m1y, float rho2, float m2x,
                                                 float m2y, const SiteForce& G) {
    const float gd = P.gamma * phv * (1.f - phv);
    const float ad = 0.5f * gd;
    const float inv = 1.f / (rho1 * rho2 + ad * (rho1 + rho2));
    const float r1x = m1x + 0.5f * G.G1x, r1y = m1y + 0.5f * G.G1y;
    const float r2x = m2x + 0.5f * G.G2x, r2y = m2y + 0.5f * G.G2y;
    Velocities v;
    v.u1x = ((rho2 + ad) * r1x + ad * r2x) * inv;
    v.u1y = ((rho2 + ad) * r1y + ad * r2y) * inv;
    v.u2x = (ad * r1x + (rho1 + ad) * r2x) * inv;
    v.u2y = (ad * r1y + (rho1 + ad) * r2y) * inv;
    const float dx = gd * (v.u2x - v.u1x), dy = gd * (v.u2y - v.u1y);
    v.F1x = G.G1x + dx;
    v.F1y = G.G1y + dy;
    v.F2x = G.G2x - dx;
    v.F2y = G.G2y - dy;
    return v;
}

// BGK + Guo collision of nine deviations in place (Sec. III):
//   d* = d - omega (d - d^eq) + (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i].F
// with d^eq = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)], rho = 1 + drho.
__device__ __forceinline__ void collide(float (&f)[9], float drho, float ux, float uy,
                                        float Fx, float Fy, float omega, float guo) {
    const float rho = 1.f + drho;
    const float usq15 = 1.5f * (ux * ux + uy * uy);
    const float uF3 = 3.f * (ux * Fx + uy * Fy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float cx = (float)d2q9_cx(i), cy = (float)d2q9_cy(i);
        const float w = d2q9_w(i);
        const float cu = cx * ux + cy * uy;
        const float cF = cx * Fx + cy * Fy;
        const float deq = w * (drho + rho * (cu * (3.f + 4.5f * cu) - usq15));
        const float src = guo * w * (3.f * cF - uF3 + 9.f * cu * cF);
        f[i] = f[i] - omega * (f[i] - deq) + src;
    }
}

}  // namespace tfd
