// Coupled two-fluid lattice step: kernels and launch sequence.
//
// One lattice step n -> n+1 (Sec. II model, Sec. III scheme):
//   k_fields : mu(phi^n) and the fluid-1 stress sigma_el + zeta phi Q (Q^n)
//   k_lbm    : forces, pull-streaming, moments, implicit-drag Guo velocities,
//              BGK + Guo collision of both D2Q9 fluids; stores u1, u2
//   k_sub x n_sub : Cahn-Hilliard + Beris-Edwards forward-Euler sub-step with
//              the stored velocities
//
// Storage: populations as deviations d_i = f_i - w_i (FP32, or a 16-bit mode
// widened to FP32 on load, see PopF16 / PopBF16) in the pull layout
// (the buffer holds post-collision values of the previous step; the
// pre-collision f_i(x) is read from x - c_i); phi as d = phi - phi_ref.
#include "tf_device.cuh"
#include "tf_internal.h"

namespace {

constexpr int BX = 32, BY = 8;

__global__ void __launch_bounds__(BX* BY)
k_fields(const float* __restrict__ phi, const float* __restrict__ Q, float* __restrict__ mu,
         float* __restrict__ tau, const DevParams* __restrict__ prm, int nx, int ny) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int b = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const DevParams P = prm[b];
    const float* ph = phi + b * N;
    const float* qa = Q + 2 * b * N;
    const float* qb = qa + N;
    const int xp = x + 1 < nx ? x + 1 : 0, xm = x > 0 ? x - 1 : nx - 1;
    const int yp = y + 1 < ny ? y + 1 : 0, ym = y > 0 ? y - 1 : ny - 1;
    const long long c = (long long)y * nx + x, e = (long long)y * nx + xp,
                    w = (long long)y * nx + xm, n = (long long)yp * nx + x,
                    s = (long long)ym * nx + x;
    const tfd::SiteStress r = tfd::site_stress(P, ph[c], ph[e], ph[w], ph[n], ph[s], qa[c], qa[e],
                                               qa[w], qa[n], qa[s], qb[c], qb[e], qb[w], qb[n], qb[s]);
    mu[b * N + c] = r.mu;
    float* t = tau + 4 * b * N;
    t[c] = r.sxx;
    t[N + c] = r.sxy;
    t[2 * N + c] = r.syx;
    t[3 * N + c] = r.syy;
}

// MODE 0: full collide (writes fdst and u).  MODE 1: macro only (writes u,
// rho1, rho2 and G1 + G2 into `macro` planes: u1x u1y u2x u2y rho1 rho2 Gx Gy).
template <int MODE>
__global__ void __launch_bounds__(BX* BY)
k_lbm(const void* __restrict__ fsrc, void* __restrict__ fdst, const float* __restrict__ phi,
      const float* __restrict__ mu, const float* __restrict__ tau, float* __restrict__ u,
      const DevParams* __restrict__ prm, int nx, int ny, int storage) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int b = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const DevParams P = prm[b];
    const float* ph = phi + b * N;
    const float* mm = mu + b * N;
    const float* t = tau + 4 * b * N;
    const int xp = x + 1 < nx ? x + 1 : 0, xm = x > 0 ? x - 1 : nx - 1;
    const int yp = y + 1 < ny ? y + 1 : 0, ym = y > 0 ? y - 1 : ny - 1;
    const long long c = (long long)y * nx + x, e = (long long)y * nx + xp,
                    w = (long long)y * nx + xm, n = (long long)yp * nx + x,
                    s = (long long)ym * nx + x;
    const float d = ph[c];
    const tfd::SiteForce G =
        tfd::site_force(P, d, ph[e], ph[w], ph[n], ph[s], mm[c], mm[e], mm[w], mm[n], mm[s],
                        t[e], t[w], t[N + n], t[N + s], t[2 * N + e], t[2 * N + w], t[3 * N + n],
                        t[3 * N + s]);
    float f1[9], f2[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = d2q9_cx(i) == 0 ? x : (d2q9_cx(i) > 0 ? xm : xp);
        const int sy = d2q9_cy(i) == 0 ? y : (d2q9_cy(i) > 0 ? ym : yp);
        const long long src = (long long)sy * nx + sx;
        f1[i] = pop_load(fsrc, pop_index(b, 0, i, src, N), storage);
        f2[i] = pop_load(fsrc, pop_index(b, 1, i, src, N), storage);
    }
    float dr1, m1x, m1y, dr2, m2x, m2y;
    tfd::moments(f1, dr1, m1x, m1y);
    tfd::moments(f2, dr2, m2x, m2y);
    const float phv = P.phi_ref + d;
    const tfd::Velocities v =
        tfd::drag_solve(P, phv, 1.f + dr1, m1x, m1y, 1.f + dr2, m2x, m2y, G);
    if (MODE == 0) {
        float* u0 = u + 4 * b * N;
        u0[c] = v.u1x;
        u0[N + c] = v.u1y;
        u0[2 * N + c] = v.u2x;
        u0[3 * N + c] = v.u2y;
        tfd::collide(f1, dr1, v.u1x, v.u1y, v.F1x, v.F1y, P.omega1, P.guo1);
        tfd::collide(f2, dr2, v.u2x, v.u2y, v.F2x, v.F2y, P.omega2, P.guo2);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            pop_store(fdst, pop_index(b, 0, i, c, N), f1[i], storage);
            pop_store(fdst, pop_index(b, 1, i, c, N), f2[i], storage);
        }
    } else {
        float* u0 = u + 8 * b * N;
        u0[c] = v.u1x;
        u0[N + c] = v.u1y;
        u0[2 * N + c] = v.u2x;
        u0[3 * N + c] = v.u2y;
        u0[4 * N + c] = 1.f + dr1;
        u0[5 * N + c] = 1.f + dr2;
        u0[6 * N + c] = G.G1x + G.G2x;
        u0[7 * N + c] = G.G1y + G.G2y;
    }
}

// One forward-Euler finite-difference sub-step of phi (Cahn-Hilliard, Eq. 1-3)
// and Q (Beris-Edwards, Eq. 11-12) with frozen velocities u.
__global__ void __launch_bounds__(BX* BY)
k_sub(const float* __restrict__ phi, const float* __restrict__ Q, float* __restrict__ phi_out,
      float* __restrict__ Q_out, const float* __restrict__ u, const DevParams* __restrict__ prm,
      int nx, int ny) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const int b = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const DevParams P = prm[b];
    const float* ph = phi + b * N;
    const float* qa = Q + 2 * b * N;
    const float* qb = qa + N;
    const float* u1x = u + 4 * b * N;
    const float* u1y = u1x + N;
    const float* u2x = u1x + 2 * N;
    const float* u2y = u1x + 3 * N;
    auto at = [&](int dx, int dy) -> long long {
        return (long long)tfd::wrap(y + dy, ny) * nx + tfd::wrap(x + dx, nx);
    };
    const long long c = at(0, 0), e = at(1, 0), w = at(-1, 0), n = at(0, 1), s = at(0, -1);
    // ---- Cahn-Hilliard: d(phi)/dt = -div(phi u_c) + M lap(mu)
    auto mu_at = [&](long long p0, long long pe, long long pw, long long pn, long long ps) {
        const float dd = ph[p0];
        const float lapd = (ph[pe] + ph[pw]) + (ph[pn] + ph[ps]) - 4.f * dd;
        return P.mu0 + dd * (P.mu1 + dd * (P.mu2 + dd * P.mu3)) - P.kappa * lapd;
    };
    const float mu0 = mu_at(c, e, w, n, s);
    const float mue = mu_at(e, at(2, 0), c, at(1, 1), at(1, -1));
    const float muw = mu_at(w, c, at(-2, 0), at(-1, 1), at(-1, -1));
    const float mun = mu_at(n, at(1, 1), at(-1, 1), at(0, 2), c);
    const float mus = mu_at(s, at(1, -1), at(-1, -1), c, at(0, -2));
    const float lapmu = (mue + muw) + (mun + mus) - 4.f * mu0;
    auto jx = [&](long long p) {
        const float pv = P.phi_ref + ph[p];
        return pv * (u2x[p] + pv * (u1x[p] - u2x[p]));
    };
    auto jy = [&](long long p) {
        const float pv = P.phi_ref + ph[p];
        return pv * (u2y[p] + pv * (u1y[p] - u2y[p]));
    };
    const float divJ = 0.5f * ((jx(e) - jx(w)) + (jy(n) - jy(s)));
    phi_out[b * N + c] = ph[c] + P.dt_fd * (P.M * lapmu - divJ);
    // ---- Beris-Edwards: dQ/dt = -(u1.grad) Q + S(grad u1, Q) + Gamma_Q H
    const float a = qa[c], bb = qb[c];
    const float lapa = (qa[e] + qa[w]) + (qa[n] + qa[s]) - 4.f * a;
    const float lapb = (qb[e] + qb[w]) + (qb[n] + qb[s]) - 4.f * bb;
    const float cq = -(P.A_Q + P.C_Q * (a * a + bb * bb));
    const float h = cq * a + P.K * lapa;
    const float g = cq * bb + P.K * lapb;
    const float Wxx = 0.5f * (u1x[e] - u1x[w]), Wxy = 0.5f * (u1x[n] - u1x[s]);
    const float Wyx = 0.5f * (u1y[e] - u1y[w]), Wyy = 0.5f * (u1y[n] - u1y[s]);
    const float trE = Wxx + Wyy;
    const float e1 = 0.5f * (Wxx - Wyy);
    const float exy = 0.5f * (Wxy + Wyx);
    const float om = Wxy - Wyx;  // 2 w
    const float QE2 = 4.f * (a * e1 + bb * exy);  // 2 (Q:E0)
    const float ux = u1x[c], uy = u1y[c];
    const float adv_a = ux * 0.5f * (qa[e] - qa[w]) + uy * 0.5f * (qa[n] - qa[s]);
    const float adv_b = ux * 0.5f * (qb[e] - qb[w]) + uy * 0.5f * (qb[n] - qb[s]);
    const float ra = -adv_a + P.lam * (trE * a + e1 - QE2 * a) + om * bb + P.GammaQ * h;
    const float rb = -adv_b + P.lam * (trE * bb + exy - QE2 * bb) - om * a + P.GammaQ * g;
    Q_out[2 * b * N + c] = a + P.dt_fd * ra;
    Q_out[(2 * b + 1) * N + c] = bb + P.dt_fd * rb;
}

dim3 site_grid(const tf_ctx* ctx) {
    return dim3((ctx->nx + BX - 1) / BX, (ctx->ny + BY - 1) / BY, ctx->batch);
}

}  // namespace

cudaError_t tf_launch_steps(tf_ctx* ctx, int64_t n) {
    if (tf_fused_supported(ctx)) return tf_fused_steps(ctx, n);
    return tf_unfused_steps(ctx, n);
}

cudaError_t tf_launch_flush(tf_ctx* ctx) { return tf_fused_flush(ctx); }

cudaError_t tf_unfused_steps(tf_ctx* ctx, int64_t n) {
    const dim3 grid = site_grid(ctx), block(BX, BY);
    DevBuffers& d = ctx->d;
    for (int64_t it = 0; it < n; ++it) {
        const int fc = ctx->fcur, pc = ctx->pcur;
        k_fields<<<grid, block, 0, ctx->stream>>>(d.phi[pc], d.Q[pc], d.mu, d.tau, d.prm, ctx->nx,
                                                  ctx->ny);
        k_lbm<0><<<grid, block, 0, ctx->stream>>>(d.f[fc], d.f[fc ^ 1], d.phi[pc], d.mu, d.tau,
                                                  d.u[0], d.prm, ctx->nx, ctx->ny, ctx->storage);
        ctx->fcur ^= 1;
        int p = pc;
        for (int s = 0; s < ctx->n_sub; ++s) {
            k_sub<<<grid, block, 0, ctx->stream>>>(d.phi[p], d.Q[p], d.phi[p ^ 1], d.Q[p ^ 1],
                                                   d.u[0], d.prm, ctx->nx, ctx->ny);
            p ^= 1;
        }
        ctx->pcur = p;
        ctx->steps += 1;
        ctx->launches += 2 + ctx->n_sub;
    }
    return cudaGetLastError();
}

cudaError_t tf_launch_macro(tf_ctx* ctx, float* macro_out) {
    const dim3 grid = site_grid(ctx), block(BX, BY);
    DevBuffers& d = ctx->d;
    k_fields<<<grid, block, 0, ctx->stream>>>(d.phi[ctx->pcur], d.Q[ctx->pcur], d.mu, d.tau, d.prm,
                                              ctx->nx, ctx->ny);
    k_lbm<1><<<grid, block, 0, ctx->stream>>>(d.f[ctx->fcur], nullptr, d.phi[ctx->pcur], d.mu,
                                              d.tau, macro_out, d.prm, ctx->nx, ctx->ny,
                                              ctx->storage);
    ctx->launches += 2;
    return cudaGetLastError();
}
