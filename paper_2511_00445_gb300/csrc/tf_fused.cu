// Fused coupled step: one kernel launch per lattice step in steady state.
//
// The lattice step n -> n+1 is regrouped as
//     LBM(0) | FD(0) + LBM(1) | FD(1) + LBM(2) | ... | FD(n-1)
// where LBM(k) = forces from (phi^k, Q^k), pull streaming, implicit-drag Guo
// velocities and BGK+Guo collision (Sec. III), and FD(k) = the n_sub
// Cahn-Hilliard / Beris-Edwards forward-Euler sub-steps with the velocities
// u^k of LBM(k).  Between launches the device holds f*^k (pull layout),
// phi^k, Q^k and u^k with FD(k) pending; the first launch of a run is the
// LBM-only prologue and an FD-only epilogue restores the plain state
// (f*, phi^{k+1}, Q^{k+1}) before any read.
//
// One CTA owns a TX x TY interior tile of one instance.  FD(k) is evaluated
// in shared memory on shrinking neighbourhoods of the tile (phi loses two
// sites of halo per sub-step through lap(mu), Q one site through lap(Q) and
// grad(Q)), ending with phi, Q valid two sites around the tile -- what the
// forces of LBM(k+1) need.  Each sub-step computes mu, then the new phi and Q
// into registers, then writes them back in place, separated by barriers.
#include "tf_device.cuh"
#include "tf_internal.h"

namespace {

constexpr int TX = 32, TY = 32;
constexpr int NT = 256;        // threads per CTA: 32 x 8
constexpr int NS_FUSED = 5;    // sub-steps handled by the fused kernel (Sec. III)

__device__ __forceinline__ int wrapc(int v, int n) {
    // v may lie several periods outside [0, n) for tiny grids
    v %= n;
    return v < 0 ? v + n : v;
}

template <bool DO_FD, bool DO_LBM>
struct Geo {
    static constexpr int R_END = DO_LBM ? 2 : 0;                // phi/Q radius after FD
    static constexpr int RH = R_END + (DO_FD ? 2 * NS_FUSED : 0);   // phi halo loaded
    static constexpr int RQ = R_END + (DO_FD ? NS_FUSED : 0);       // Q halo loaded
    static constexpr int RU = DO_FD ? R_END + 2 * NS_FUSED - 1 : 0; // u halo loaded
    static constexpr int W = TX + 2 * RH;
    static constexpr int H = TY + 2 * RH;
    static constexpr int A = W * H;                              // floats per smem plane
    static constexpr int NPLANES = 8;                            // phi mu u1x u1y u2x u2y qa qb
    static constexpr size_t SMEM = (size_t)NPLANES * A * sizeof(float);
};

// Iterate the sites of the square neighbourhood of radius r around the tile
// (local coordinates offset by the halo RH).  F(ly, lx, k) with k the
// per-thread slot index (static after unrolling).
template <int RH, int r, int SLOTS, typename F>
__device__ __forceinline__ void for_region(F&& f) {
    constexpr int w = TX + 2 * r, h = TY + 2 * r, cnt = w * h;
    static_assert(SLOTS * NT >= cnt, "register slots too few for region");
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
        const int idx = threadIdx.x + k * NT;
        if (idx < cnt) {
            const int ly = RH - r + idx / w;
            const int lx = RH - r + idx % w;
            f(ly, lx, k);
        }
    }
}

template <int RH, int W>
struct Sm {
    float* phi;
    float* mu;
    float* u1x;
    float* u1y;
    float* u2x;
    float* u2y;
    float* qa;
    float* qb;
    __device__ __forceinline__ static int at(int ly, int lx) { return ly * W + lx; }
};

// One forward-Euler sub-step on the neighbourhood of radius rp (phi) / rq (Q).
template <int RH, int W, int rp, int rq>
__device__ __forceinline__ void fd_substep(const DevParams& P, Sm<RH, W>& s) {
    // (a) chemical potential on radius rp + 1 (needs phi on rp + 2)
    constexpr int SL_MU = ((TX + 2 * (rp + 1)) * (TY + 2 * (rp + 1)) + NT - 1) / NT;
    for_region<RH, rp + 1, SL_MU>([&](int ly, int lx, int) {
        const int c = ly * W + lx;
        const float d = s.phi[c];
        const float lapd = (s.phi[c + 1] + s.phi[c - 1]) + (s.phi[c + W] + s.phi[c - W]) - 4.f * d;
        s.mu[c] = P.mu0 + d * (P.mu1 + d * (P.mu2 + d * P.mu3)) - P.kappa * lapd;
    });
    __syncthreads();
    // (b) new phi on radius rp and new Q on radius rq, into registers
    constexpr int SL = ((TX + 2 * rp) * (TY + 2 * rp) + NT - 1) / NT;
    float nphi[SL], na[SL], nb[SL];
    for_region<RH, rp, SL>([&](int ly, int lx, int k) {
        const int c = ly * W + lx;
        const int e = c + 1, w = c - 1, n = c + W, so = c - W;
        auto jx = [&](int p) {
            const float pv = P.phi_ref + s.phi[p];
            return pv * (s.u2x[p] + pv * (s.u1x[p] - s.u2x[p]));
        };
        auto jy = [&](int p) {
            const float pv = P.phi_ref + s.phi[p];
            return pv * (s.u2y[p] + pv * (s.u1y[p] - s.u2y[p]));
        };
        const float lapmu = (s.mu[e] + s.mu[w]) + (s.mu[n] + s.mu[so]) - 4.f * s.mu[c];
        const float divJ = 0.5f * ((jx(e) - jx(w)) + (jy(n) - jy(so)));
        nphi[k] = s.phi[c] + P.dt_fd * (P.M * lapmu - divJ);
        const int dy = ly - RH, dx = lx - RH;   // rq-region test (rq <= rp)
        if (dx >= -rq && dx < TX + rq && dy >= -rq && dy < TY + rq) {
            const float a = s.qa[c], bq = s.qb[c];
            const float lapa = (s.qa[e] + s.qa[w]) + (s.qa[n] + s.qa[so]) - 4.f * a;
            const float lapb = (s.qb[e] + s.qb[w]) + (s.qb[n] + s.qb[so]) - 4.f * bq;
            const float cq = -(P.A_Q + P.C_Q * (a * a + bq * bq));
            const float h = cq * a + P.K * lapa;
            const float g = cq * bq + P.K * lapb;
            const float Wxx = 0.5f * (s.u1x[e] - s.u1x[w]), Wxy = 0.5f * (s.u1x[n] - s.u1x[so]);
            const float Wyx = 0.5f * (s.u1y[e] - s.u1y[w]), Wyy = 0.5f * (s.u1y[n] - s.u1y[so]);
            const float trE = Wxx + Wyy;
            const float e1 = 0.5f * (Wxx - Wyy);
            const float exy = 0.5f * (Wxy + Wyx);
            const float om = Wxy - Wyx;
            const float QE2 = 4.f * (a * e1 + bq * exy);
            const float ux = s.u1x[c], uy = s.u1y[c];
            const float adv_a = ux * 0.5f * (s.qa[e] - s.qa[w]) + uy * 0.5f * (s.qa[n] - s.qa[so]);
            const float adv_b = ux * 0.5f * (s.qb[e] - s.qb[w]) + uy * 0.5f * (s.qb[n] - s.qb[so]);
            const float ra = -adv_a + P.lam * (trE * a + e1 - QE2 * a) + om * bq + P.GammaQ * h;
            const float rb = -adv_b + P.lam * (trE * bq + exy - QE2 * bq) - om * a + P.GammaQ * g;
            na[k] = a + P.dt_fd * ra;
            nb[k] = bq + P.dt_fd * rb;
        }
    });
    __syncthreads();
    // (c) write back in place
    for_region<RH, rp, SL>([&](int ly, int lx, int k) {
        const int c = ly * W + lx;
        s.phi[c] = nphi[k];
        const int dy = ly - RH, dx = lx - RH;
        if (dx >= -rq && dx < TX + rq && dy >= -rq && dy < TY + rq) {
            s.qa[c] = na[k];
            s.qb[c] = nb[k];
        }
    });
    __syncthreads();
}

template <int RH, int W, int R_END, int S>
__device__ __forceinline__ void fd_all(const DevParams& P, Sm<RH, W>& s) {
    if constexpr (S < NS_FUSED) {
        constexpr int rp = R_END + 2 * (NS_FUSED - 1 - S);
        constexpr int rq = R_END + (NS_FUSED - 1 - S);
        fd_substep<RH, W, rp, rq>(P, s);
        fd_all<RH, W, R_END, S + 1>(P, s);
    }
}

template <bool DO_FD, bool DO_LBM>
__global__ void __launch_bounds__(NT, 2)
k_fused(const float* __restrict__ fsrc, float* __restrict__ fdst,
        const float* __restrict__ phi_in, float* __restrict__ phi_out,
        const float* __restrict__ Q_in, float* __restrict__ Q_out,
        const float* __restrict__ u_in, float* __restrict__ u_out,
        const DevParams* __restrict__ prm, int nx, int ny) {
    using G = Geo<DO_FD, DO_LBM>;
    constexpr int RH = G::RH, W = G::W, H = G::H, A = G::A;
    extern __shared__ float smem[];
    Sm<RH, W> s{smem, smem + A, smem + 2 * A, smem + 3 * A, smem + 4 * A, smem + 5 * A,
                smem + 6 * A, smem + 7 * A};
    const int b = blockIdx.z;
    const long long N = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const DevParams P = prm[b];
    const float* gphi = phi_in + b * N;
    const float* gqa = Q_in + 2 * b * N;
    const float* gqb = gqa + N;

    // ---- load phi (radius RH), Q (radius RQ) and, for FD, u (radius RU)
    for (int i = threadIdx.x; i < A; i += NT) {
        const int ly = i / W, lx = i - ly * W;
        const int dy = ly - RH, dx = lx - RH;
        const int gy = wrapc(y0 + dy, ny), gx = wrapc(x0 + dx, nx);
        const long long g = (long long)gy * nx + gx;
        s.phi[i] = gphi[g];
        if (dx >= -G::RQ && dx < TX + G::RQ && dy >= -G::RQ && dy < TY + G::RQ) {
            s.qa[i] = gqa[g];
            s.qb[i] = gqb[g];
        }
        if constexpr (DO_FD) {
            if (dx >= -G::RU && dx < TX + G::RU && dy >= -G::RU && dy < TY + G::RU) {
                const float* gu = u_in + 4 * b * N;
                s.u1x[i] = gu[g];
                s.u1y[i] = gu[N + g];
                s.u2x[i] = gu[2 * N + g];
                s.u2y[i] = gu[3 * N + g];
            }
        }
    }
    __syncthreads();

    if constexpr (DO_FD) fd_all<RH, W, G::R_END, 0>(P, s);

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if constexpr (DO_LBM) {
        // ---- chemical potential and fluid-1 stress on radius 1 (u planes reused)
        constexpr int SL1 = ((TX + 2) * (TY + 2) + NT - 1) / NT;
        for_region<RH, 1, SL1>([&](int ly, int lx, int) {
            const int c = ly * W + lx;
            const tfd::SiteStress r = tfd::site_stress(
                P, s.phi[c], s.phi[c + 1], s.phi[c - 1], s.phi[c + W], s.phi[c - W], s.qa[c],
                s.qa[c + 1], s.qa[c - 1], s.qa[c + W], s.qa[c - W], s.qb[c], s.qb[c + 1],
                s.qb[c - 1], s.qb[c + W], s.qb[c - W]);
            s.mu[c] = r.mu;
            s.u1x[c] = r.sxx;
            s.u1y[c] = r.sxy;
            s.u2x[c] = r.syx;
            s.u2y[c] = r.syy;
        });
        __syncthreads();
        // ---- interior: forces, pull, moments, drag, collide, store
        const float* F1 = fsrc + 18 * b * N;
        const float* F2 = F1 + 9 * N;
        float* D1 = fdst + 18 * b * N;
        float* D2 = D1 + 9 * N;
        float* uo = u_out + 4 * b * N;
#pragma unroll 1
        for (int r = ty; r < TY; r += NT / 32) {
            const int x = x0 + tx, y = y0 + r;
            if (x >= nx || y >= ny) continue;
            const int c = (RH + r) * W + RH + tx;
            const float d = s.phi[c];
            const tfd::SiteForce Fo = tfd::site_force(
                P, d, s.phi[c + 1], s.phi[c - 1], s.phi[c + W], s.phi[c - W], s.mu[c],
                s.mu[c + 1], s.mu[c - 1], s.mu[c + W], s.mu[c - W], s.u1x[c + 1], s.u1x[c - 1],
                s.u1y[c + W], s.u1y[c - W], s.u2x[c + 1], s.u2x[c - 1], s.u2y[c + W],
                s.u2y[c - W]);
            const int xp = x + 1 < nx ? x + 1 : 0, xm = x > 0 ? x - 1 : nx - 1;
            const int yp = y + 1 < ny ? y + 1 : 0, ym = y > 0 ? y - 1 : ny - 1;
            float f1[9], f2[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sx = d2q9_cx(i) == 0 ? x : (d2q9_cx(i) > 0 ? xm : xp);
                const int sy = d2q9_cy(i) == 0 ? y : (d2q9_cy(i) > 0 ? ym : yp);
                const long long src = (long long)sy * nx + sx;
                f1[i] = F1[i * N + src];
                f2[i] = F2[i * N + src];
            }
            float dr1, m1x, m1y, dr2, m2x, m2y;
            tfd::moments(f1, dr1, m1x, m1y);
            tfd::moments(f2, dr2, m2x, m2y);
            const tfd::Velocities v = tfd::drag_solve(P, P.phi_ref + d, 1.f + dr1, m1x, m1y,
                                                      1.f + dr2, m2x, m2y, Fo);
            tfd::collide(f1, dr1, v.u1x, v.u1y, v.F1x, v.F1y, P.omega1, P.guo1);
            tfd::collide(f2, dr2, v.u2x, v.u2y, v.F2x, v.F2y, P.omega2, P.guo2);
            const long long g = (long long)y * nx + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                D1[i * N + g] = f1[i];
                D2[i * N + g] = f2[i];
            }
            uo[g] = v.u1x;
            uo[N + g] = v.u1y;
            uo[2 * N + g] = v.u2x;
            uo[3 * N + g] = v.u2y;
        }
    }
    if constexpr (DO_FD) {
        // ---- store phi^{k+1}, Q^{k+1} of the interior
        float* po = phi_out + b * N;
        float* qo = Q_out + 2 * b * N;
        for (int r = ty; r < TY; r += NT / 32) {
            const int x = x0 + tx, y = y0 + r;
            if (x >= nx || y >= ny) continue;
            const int c = (RH + r) * W + RH + tx;
            const long long g = (long long)y * nx + x;
            po[g] = s.phi[c];
            qo[g] = s.qa[c];
            qo[N + g] = s.qb[c];
        }
    }
}

template <bool DO_FD, bool DO_LBM>
cudaError_t configure() {
    return cudaFuncSetAttribute(k_fused<DO_FD, DO_LBM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<DO_FD, DO_LBM>::SMEM);
}

template <bool DO_FD, bool DO_LBM>
cudaError_t launch(tf_ctx* ctx) {
    using G = Geo<DO_FD, DO_LBM>;
    DevBuffers& d = ctx->d;
    const dim3 grid((ctx->nx + TX - 1) / TX, (ctx->ny + TY - 1) / TY, ctx->batch);
    const int fc = ctx->fcur, pc = ctx->pcur, uc = ctx->ucur;
    k_fused<DO_FD, DO_LBM><<<grid, NT, G::SMEM, ctx->stream>>>(
        d.f[fc], d.f[fc ^ 1], d.phi[pc], d.phi[pc ^ 1], d.Q[pc], d.Q[pc ^ 1], d.u[uc],
        d.u[uc ^ 1], d.prm, ctx->nx, ctx->ny);
    if (DO_LBM) {
        ctx->fcur ^= 1;
        ctx->ucur ^= 1;
    }
    if (DO_FD) ctx->pcur ^= 1;
    ctx->launches += 1;
    return cudaGetLastError();
}

}  // namespace

bool tf_fused_supported(const tf_ctx* ctx) { return ctx->n_sub == NS_FUSED; }

cudaError_t tf_configure_fused_kernels() {
    cudaError_t e = configure<true, true>();
    if (e == cudaSuccess) e = configure<false, true>();
    if (e == cudaSuccess) e = configure<true, false>();
    return e;
}

cudaError_t tf_fused_steps(tf_ctx* ctx, int64_t n) {
    for (int64_t it = 0; it < n; ++it) {
        cudaError_t e = ctx->fd_pending ? launch<true, true>(ctx) : launch<false, true>(ctx);
        if (e != cudaSuccess) return e;
        ctx->fd_pending = true;
        ctx->steps += 1;
    }
    return cudaSuccess;
}

cudaError_t tf_fused_flush(tf_ctx* ctx) {
    if (!ctx->fd_pending) return cudaSuccess;
    cudaError_t e = launch<true, false>(ctx);
    ctx->fd_pending = false;
    return e;
}
