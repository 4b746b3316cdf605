// Paired FP32 arithmetic for the fused step: each lane carries two adjacent
// columns (or the two fluids of a site), and every operation returns, for
// each of the two elements, the correctly rounded IEEE result of the written
// operation.  Nothing is contracted or reassociated, so the prologue,
// epilogue, tile, strip and ensemble kernels produce bitwise the same values
// for the same inputs.
//
// Every pair operation is one packed fused multiply-add (fma.rn.f32x2, two
// FP32 lanes per instruction), which halves the FP32 instructions of a pair:
//   a * b = fma(a, b, -0),  a + b = fma(a, 1, b),  a - b = fma(b, -1, a),
//   -a = fma(a, -1, -0).
// Each is exact to the scalar operation: the product or sum is formed exactly
// and rounded once, and the signed zero added or the factor +-1 changes neither
// the value nor the sign of a zero result.  Because every operation is already
// a single FMA, the compiler has no separate multiply and add left to fuse: an
// earlier version that wrote the packed forms as separate add/sub/mul (the
// __f*2_rn intrinsics and add/sub/mul.rn.f32x2) saw a product fed unrounded into
// a following subtraction at a few sites, in places that moved with code layout.
// Compiling with -DTF_SCALAR_FP32 selects per-element scalar intrinsics
// (__fadd_rn, __fsub_rn, __fmul_rn, __fmaf_rn) with identical results.
#pragma once

#include "tf_internal.h"

namespace tfq {

typedef float2 f2;
__device__ __forceinline__ f2 S2(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 P2(float a, float b) { return make_float2(a, b); }
#ifdef TF_SCALAR_FP32
__device__ __forceinline__ f2 A2(f2 a, f2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ f2 B2(f2 a, f2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ f2 M2(f2 a, f2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
// a * b + c with a single rounding per element
__device__ __forceinline__ f2 F2(f2 a, f2 b, f2 c) {
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ f2 N2(f2 a) { return make_float2(-a.x, -a.y); }
#else
__device__ __forceinline__ unsigned long long pk(f2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ f2 upk(unsigned long long r) {
    f2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
// a * b + c with a single rounding per element
__device__ __forceinline__ f2 F2(f2 a, f2 b, f2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ f2 M2(f2 a, f2 b) { return F2(a, b, make_float2(-0.f, -0.f)); }
__device__ __forceinline__ f2 A2(f2 a, f2 b) { return F2(a, make_float2(1.f, 1.f), b); }
__device__ __forceinline__ f2 B2(f2 a, f2 b) { return F2(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ f2 N2(f2 a) { return F2(a, make_float2(-1.f, -1.f), make_float2(-0.f, -0.f)); }
#endif
__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// x-neighbour sum v(x - 1) + v(x + 1) and difference v(x + 1) - v(x - 1) of
// each column of a lane's pair (2P, 2P+1), the outer neighbours from the
// adjacent lanes.  Each is formed by one scalar operation straight into its
// pair: packed operations would first need pairs assembled from the shifted
// columns, i.e. register moves (measured: these scalar forms took the tile
// kernel's 1024^2 step from 99.6 to 97.2 us).
__device__ __forceinline__ void hsd2(f2 v, f2& s, f2& d) {
    const float up = __shfl_up_sync(0xffffffffu, v.y, 1);
    const float dn = __shfl_down_sync(0xffffffffu, v.x, 1);
    s = make_float2(__fadd_rn(up, v.y), __fadd_rn(v.x, dn));
    d = make_float2(__fsub_rn(v.y, up), __fsub_rn(dn, v.x));
}
__device__ __forceinline__ f2 hsum2(f2 v) {
    f2 s, d;
    hsd2(v, s, d);
    return s;
}
__device__ __forceinline__ f2 hdiff2(f2 v) {
    f2 s, d;
    hsd2(v, s, d);
    return d;
}

// Column pair of this lane for a neighbourhood whose columns start at shared
// column o and span w: lanes cover pairs from the one holding column o - 1 to
// the one holding column o + w (the one-column halo).  Surplus lanes repeat
// the last pair so that their loads stay in bounds, but their shuffled
// neighbours are not the pair's true neighbours: they never write.
// st: the lane owns its pair and the pair meets the neighbourhood.  Where o
// or o + w is odd, the edge pair also covers one column just outside; the
// whole pair is stored, and that outside column (one site beyond the radius
// the next stage reads) takes a value nobody reads.
struct PairCols {
    int c0;
    bool st;
    __device__ __forceinline__ PairCols(int o, int w, int lane) {
        const int pb = (o - 1) >> 1, pl = (o + w) >> 1;
        const bool own = pb + lane <= pl;
        c0 = 2 * min(pb + lane, pl);
        st = own && c0 + 1 >= o && c0 < o + w;
    }
    // st for a narrower neighbourhood [oq, oq + wq) inside this one
    __device__ __forceinline__ bool meets(int oq, int wq) const {
        return st && c0 + 1 >= oq && c0 < oq + wq;
    }
};

__device__ __forceinline__ void st_pair(float* p, f2 v, bool st) {
    if (st) *reinterpret_cast<float2*>(p) = v;
}

// Chemical potential and fluid-1 stress (elastic + active) for a column pair,
// from the pair's values (d = phi - phi_ref, a = Q_xx, b = Q_xy), their
// x-neighbour sums (dh, ah, bh) and differences (ax, bx) as hsd2 forms them,
// and their y-neighbours (s = row below, n = row above).  Same algebra as
// tfd::site_stress.
struct PairStress {
    f2 mu, sxx, sxy, syx, syy;
};

__device__ __forceinline__ PairStress stress2(const DevParams& P, f2 d, f2 dh, f2 dn, f2 ds,
                                               f2 a, f2 ah, f2 ax, f2 an, f2 as, f2 b, f2 bh,
                                               f2 bx, f2 bn, f2 bs) {
    const f2 m4 = S2(-4.f), half = S2(0.5f);
    PairStress o;
    const f2 lapd = F2(m4, d, A2(dh, A2(dn, ds)));
    const f2 poly = F2(d, F2(d, F2(d, S2(P.mu3), S2(P.mu2)), S2(P.mu1)), S2(P.mu0));
    o.mu = F2(S2(-P.kappa), lapd, poly);
    const f2 lapa = F2(m4, a, A2(ah, A2(an, as)));
    const f2 lapb = F2(m4, b, A2(bh, A2(bn, bs)));
    const f2 dxa = M2(half, ax), dya = M2(half, B2(an, as));
    const f2 dxb = M2(half, bx), dyb = M2(half, B2(bn, bs));
    const f2 cq = F2(S2(-P.C_Q), F2(a, a, M2(b, b)), S2(-P.A_Q));
    const f2 K = S2(P.K), k2 = S2(2.f * P.K), lam = S2(P.lam);
    const f2 h = F2(cq, a, M2(K, lapa));
    const f2 g = F2(cq, b, M2(K, lapb));
    const f2 Txx = M2(k2, F2(dxa, dxa, M2(dxb, dxb)));
    const f2 Tyy = M2(k2, F2(dya, dya, M2(dyb, dyb)));
    const f2 Txy = M2(k2, F2(dxa, dya, M2(dxb, dyb)));
    const f2 l2qh = M2(S2(4.f * P.lam), F2(a, h, M2(b, g)));     // 2 lam (Q:H)
    const f2 anti = M2(S2(2.f), B2(M2(a, g), M2(b, h)));
    const f2 phv = A2(S2(P.phi_ref), d);
    const f2 zp = M2(S2(P.zeta), phv);
    const f2 za = M2(zp, a), zb = M2(zp, b);
    o.sxx = A2(B2(F2(l2qh, a, N2(M2(lam, h))), Txx), za);
    o.syy = B2(B2(F2(lam, h, N2(M2(l2qh, a))), Tyy), za);
    const f2 sym = A2(B2(F2(l2qh, b, N2(M2(lam, g))), Txy), zb);
    o.sxy = A2(sym, anti);
    o.syx = B2(sym, anti);
    return o;
}

// One interior site of the LBM stage with the two fluids paired:
// forces G from the stress / mu / phi neighbourhood (same algebra as
// tfd::site_force), moments, implicit-drag Guo velocities (tfd::drag_solve)
// and the BGK + Guo collision of both fluids (tfd::collide).  f[i] holds
// (fluid 1, fluid 2) deviations of direction i and is updated in place; the
// Guo velocities are returned as u1 = (u1x, u1y), u2 = (u2x, u2y).
__device__ __forceinline__ void lbm_site2(const DevParams& P, float d, f2 dlr_x /*(dw, de)*/,
                                          f2 dns_y /*(ds, dn)*/, float m0, f2 mwe, f2 msn,
                                          f2 sxx_we, f2 sxy_sn, f2 syx_we, f2 syy_sn,
                                          f2 (&f)[9], f2& u1, f2& u2) {
    const f2 half = S2(0.5f);
    const float c = P.phi_ref;
    // capillary force F_ch = [phi_+ (mu_0 - mu_+) - phi_- (mu_0 - mu_-)] / 2 per axis,
    // components paired as (x, y)
    const f2 mm = P2(mwe.x, msn.x), mp = P2(mwe.y, msn.y);     // (mu_w, mu_s), (mu_e, mu_n)
    const f2 dm = P2(dlr_x.x, dns_y.x), dp = P2(dlr_x.y, dns_y.y);
    const f2 M0 = S2(m0);
    const f2 fch = M2(half, B2(F2(S2(c), B2(mm, mp), M2(dp, B2(M0, mp))), M2(dm, B2(M0, mm))));
    const f2 divs = M2(half, P2(__fadd_rn(__fsub_rn(sxx_we.y, sxx_we.x), __fsub_rn(sxy_sn.y, sxy_sn.x)),
                                __fadd_rn(__fsub_rn(syx_we.y, syx_we.x), __fsub_rn(syy_sn.y, syy_sn.x))));
    const float phv = __fadd_rn(c, d);
    const float om = __fsub_rn(__fsub_rn(1.f, c), d);
    const f2 G1 = F2(S2(phv), fch, divs);
    const f2 G2 = M2(S2(om), fch);
    // moments of both fluids: (drho1, drho2), (m1x, m2x), (m1y, m2y)
    const f2 dr = A2(A2(A2(A2(f[0], f[1]), A2(f[2], f[3])), A2(A2(f[4], f[5]), A2(f[6], f[7]))), f[8]);
    const f2 mx = A2(B2(f[1], f[3]), A2(B2(f[5], f[6]), B2(f[8], f[7])));
    const f2 my = A2(B2(f[2], f[4]), B2(A2(f[5], f[6]), A2(f[7], f[8])));
    // implicit drag: (rho1 + g/2) u1 - g/2 u2 = m1 + G1/2, -g/2 u1 + (rho2 + g/2) u2 = m2 + G2/2
    const float gd = __fmul_rn(__fmul_rn(P.gamma, phv), __fsub_rn(1.f, phv));
    const float ad = __fmul_rn(0.5f, gd);
    const f2 rho = A2(S2(1.f), dr);
    const float det = __fmaf_rn(rho.x, rho.y, __fmul_rn(ad, __fadd_rn(rho.x, rho.y)));
    const float inv = __frcp_rn(det);
    const f2 r1 = F2(half, G1, P2(mx.x, my.x));                 // (r1x, r1y)
    const f2 r2 = F2(half, G2, P2(mx.y, my.y));                 // (r2x, r2y)
    u1 = M2(F2(S2(__fadd_rn(rho.y, ad)), r1, M2(S2(ad), r2)), S2(inv));
    u2 = M2(F2(S2(ad), r1, M2(S2(__fadd_rn(rho.x, ad)), r2)), S2(inv));
    const f2 du = M2(S2(gd), B2(u2, u1));
    const f2 F1 = A2(G1, du), Fv2 = B2(G2, du);
    // collision, fluids paired: components as (fluid 1, fluid 2).
    // d* = (1 - omega) d + omega d^eq + S_i with the BGK + Guo terms split into
    // the parts even and odd in c_i, so that a direction and its opposite
    // (c.u and c.F change sign) share every product:
    //   omega d^eq + S = w [omega Z + G (9 (c.u)(c.F) - 3 u.F)]
    //                  +/- 3 w [omega rho (c.u) + G (c.F)],
    //   Z = drho + rho (4.5 (c.u)^2 - 1.5 u^2),  G = 1 - omega/2.
    const f2 UX = P2(u1.x, u2.x), UY = P2(u1.y, u2.y);
    const f2 FX = P2(F1.x, Fv2.x), FY = P2(F1.y, Fv2.y);
    const f2 OM = P2(P.omega1, P.omega2), GU = P2(P.guo1, P.guo2);
    const f2 omc = P2(__fsub_rn(1.f, P.omega1), __fsub_rn(1.f, P.omega2));
    const f2 nusq = M2(S2(-1.5f), F2(UX, UX, M2(UY, UY)));     // -1.5 u^2
    const f2 nuF3 = M2(S2(-3.f), F2(UX, FX, M2(UY, FY)));      // -3 u.F
    const f2 orho = M2(OM, rho);
    {
        const f2 Z = F2(rho, nusq, dr);
        f[0] = F2(omc, f[0], M2(S2(d2q9_w(0)), F2(OM, Z, M2(GU, nuF3))));
    }
    auto pair = [&](int i, int j, f2 cu, f2 cF) {
        const float w = d2q9_w(i);
        const f2 Z = F2(rho, F2(M2(S2(4.5f), cu), cu, nusq), dr);
        const f2 ev = M2(S2(w), F2(OM, Z, M2(GU, F2(S2(9.f), M2(cu, cF), nuF3))));
        const f2 od = M2(S2(3.f * w), F2(orho, cu, M2(GU, cF)));
        f[i] = F2(omc, f[i], A2(ev, od));
        f[j] = F2(omc, f[j], B2(ev, od));
    };
    pair(1, 3, UX, FX);                         // c = (+1, 0) and (-1, 0)
    pair(2, 4, UY, FY);                         // (0, +1) and (0, -1)
    pair(5, 7, A2(UX, UY), A2(FX, FY));         // (+1, +1) and (-1, -1)
    pair(6, 8, B2(UY, UX), B2(FY, FX));         // (-1, +1) and (+1, -1)
}

}  // namespace tfq
