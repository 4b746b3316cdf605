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
// One CTA owns a TX x TY interior tile of one instance:
//  1. the phi, Q and u planes of the tile plus a halo are brought into shared
//     memory by bulk copies (one per row segment, periodic wrap handled by
//     splitting segments), and the population rows the tile will pull are
//     bulk-prefetched into L2 so that they stream from HBM during step 2;
//  2. FD(k) runs in shared memory on shrinking neighbourhoods of the tile
//     (phi loses two sites of halo per sub-step through lap(mu), Q one site);
//     each sub-step computes mu, then the new phi and Q into registers, then
//     writes them back in place, separated by barriers;
//  3. mu and the fluid-1 stress on radius 1, then per interior site the
//     forces, pulled populations, drag solve, collision and stores.
#include "tf_device.cuh"
#include "tf_internal.h"
#include "tf_ptx.cuh"

namespace {

constexpr int TX = 32, TY = 32;
constexpr int NT = 256;        // threads per CTA: 32 x 8
constexpr int NS_FUSED = 5;    // sub-steps handled by the fused kernel (Sec. III)
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ int wrapc(int v, int n) {
    // v may lie several periods outside [0, n) for tiny grids
    v %= n;
    return v < 0 ? v + n : v;
}

constexpr int round4(int v) { return (v + 3) & ~3; }

template <bool DO_FD, bool DO_LBM>
struct Geo {
    static constexpr int R_END = DO_LBM ? 2 : 0;                  // phi/Q radius after FD
    static constexpr int RH_NEED = R_END + (DO_FD ? 2 * NS_FUSED : 0);
    static constexpr int RH = round4(RH_NEED < 4 ? 4 : RH_NEED);  // loaded halo, 16-byte aligned
    static constexpr int W = TX + 2 * RH;
    static constexpr int H = TY + 2 * RH;
    static constexpr int A = W * H;                              // floats per smem plane
    static constexpr int NPLANES = 8;                            // phi mu u1x u1y u2x u2y qa qb
    static constexpr int NLOAD = DO_FD ? 7 : 3;                  // planes read from global
    static constexpr size_t SMEM = (size_t)NPLANES * A * sizeof(float);
    static constexpr int RP_MAX = R_END + 2 * (NS_FUSED - 1);    // largest phi update radius
    static constexpr int SLOTS = ((TX + 2 * RP_MAX) * (TY + 2 * RP_MAX) + NT - 1) / NT;
};

struct Sm {
    float* p[8];   // phi mu u1x u1y u2x u2y qa qb
};
enum { P_PHI = 0, P_MU, P_U1X, P_U1Y, P_U2X, P_U2Y, P_QA, P_QB };

// One forward-Euler sub-step: phi on the neighbourhood of radius rp, Q on rq.
// Sites of a neighbourhood are numbered row-major and dealt to the threads
// in order; each thread keeps its updated values in registers until all
// threads have read the old ones.
template <int RH, int W, int SLOTS>
__device__ __forceinline__ void fd_substep(const DevParams& P, const Sm& s, int rp, int rq) {
    float* __restrict__ phi = s.p[P_PHI];
    float* __restrict__ mu = s.p[P_MU];
    const float* __restrict__ u1x = s.p[P_U1X];
    const float* __restrict__ u1y = s.p[P_U1Y];
    const float* __restrict__ u2x = s.p[P_U2X];
    const float* __restrict__ u2y = s.p[P_U2Y];
    float* __restrict__ qa = s.p[P_QA];
    float* __restrict__ qb = s.p[P_QB];
    // (a) chemical potential on radius rp + 1 (needs phi on rp + 2)
    {
        const int r = rp + 1, w = TX + 2 * r, cnt = w * (TY + 2 * r);
        int ly = threadIdx.x / w, lx = threadIdx.x - ly * w;
        const int dly = NT / w, dlx = NT - dly * w;
#pragma unroll 4
        for (int idx = threadIdx.x; idx < cnt; idx += NT) {
            const int c = (RH - r + ly) * W + RH - r + lx;
            const float d = phi[c];
            const float lapd = (phi[c + 1] + phi[c - 1]) + (phi[c + W] + phi[c - W]) - 4.f * d;
            mu[c] = P.mu0 + d * (P.mu1 + d * (P.mu2 + d * P.mu3)) - P.kappa * lapd;
            lx += dlx;
            ly += dly;
            if (lx >= w) {
                lx -= w;
                ly += 1;
            }
        }
    }
    __syncthreads();
    // (b) new phi on radius rp and new Q on radius rq, into registers
    const int w = TX + 2 * rp, cnt = w * (TY + 2 * rp);
    const int ly0 = threadIdx.x / w, lx0 = threadIdx.x - ly0 * w;
    const int dly = NT / w, dlx = NT - dly * w;
    float nphi[SLOTS], na[SLOTS], nb[SLOTS];
    {
        int ly = ly0, lx = lx0;
#pragma unroll
        for (int k = 0; k < SLOTS; ++k) {
            if (threadIdx.x + k * NT < cnt) {
                const int c = (RH - rp + ly) * W + RH - rp + lx;
                const int e = c + 1, wv = c - 1, n = c + W, so = c - W;
                const float pe = P.phi_ref + phi[e], pw = P.phi_ref + phi[wv];
                const float pn = P.phi_ref + phi[n], ps = P.phi_ref + phi[so];
                const float jxe = pe * (u2x[e] + pe * (u1x[e] - u2x[e]));
                const float jxw = pw * (u2x[wv] + pw * (u1x[wv] - u2x[wv]));
                const float jyn = pn * (u2y[n] + pn * (u1y[n] - u2y[n]));
                const float jys = ps * (u2y[so] + ps * (u1y[so] - u2y[so]));
                const float lapmu = (mu[e] + mu[wv]) + (mu[n] + mu[so]) - 4.f * mu[c];
                const float divJ = 0.5f * ((jxe - jxw) + (jyn - jys));
                nphi[k] = phi[c] + P.dt_fd * (P.M * lapmu - divJ);
                const int dy = ly - rp, dx = lx - rp;   // rq-region test (rq <= rp)
                if (dx >= -rq && dx < TX + rq && dy >= -rq && dy < TY + rq) {
                    const float a = qa[c], bq = qb[c];
                    const float ae = qa[e], aw = qa[wv], an = qa[n], as = qa[so];
                    const float be = qb[e], bw = qb[wv], bn = qb[n], bs = qb[so];
                    const float lapa = (ae + aw) + (an + as) - 4.f * a;
                    const float lapb = (be + bw) + (bn + bs) - 4.f * bq;
                    const float cq = -(P.A_Q + P.C_Q * (a * a + bq * bq));
                    const float h = cq * a + P.K * lapa;
                    const float g = cq * bq + P.K * lapb;
                    const float Wxx = 0.5f * (u1x[e] - u1x[wv]), Wxy = 0.5f * (u1x[n] - u1x[so]);
                    const float Wyx = 0.5f * (u1y[e] - u1y[wv]), Wyy = 0.5f * (u1y[n] - u1y[so]);
                    const float trE = Wxx + Wyy;
                    const float e1 = 0.5f * (Wxx - Wyy);
                    const float exy = 0.5f * (Wxy + Wyx);
                    const float om = Wxy - Wyx;
                    const float QE2 = 4.f * (a * e1 + bq * exy);
                    const float ux = u1x[c], uy = u1y[c];
                    const float adv_a = ux * 0.5f * (ae - aw) + uy * 0.5f * (an - as);
                    const float adv_b = ux * 0.5f * (be - bw) + uy * 0.5f * (bn - bs);
                    const float ra = -adv_a + P.lam * (trE * a + e1 - QE2 * a) + om * bq + P.GammaQ * h;
                    const float rb = -adv_b + P.lam * (trE * bq + exy - QE2 * bq) - om * a + P.GammaQ * g;
                    na[k] = a + P.dt_fd * ra;
                    nb[k] = bq + P.dt_fd * rb;
                }
            }
            lx += dlx;
            ly += dly;
            if (lx >= w) {
                lx -= w;
                ly += 1;
            }
        }
    }
    __syncthreads();
    // (c) write back in place
    {
        int ly = ly0, lx = lx0;
#pragma unroll
        for (int k = 0; k < SLOTS; ++k) {
            if (threadIdx.x + k * NT < cnt) {
                const int c = (RH - rp + ly) * W + RH - rp + lx;
                phi[c] = nphi[k];
                const int dy = ly - rp, dx = lx - rp;
                if (dx >= -rq && dx < TX + rq && dy >= -rq && dy < TY + rq) {
                    qa[c] = na[k];
                    qb[c] = nb[k];
                }
            }
            lx += dlx;
            ly += dly;
            if (lx >= w) {
                lx -= w;
                ly += 1;
            }
        }
    }
    __syncthreads();
}

// Copy `len` floats of row gy starting at column xs (periodic in x) from a
// global plane into shared memory, splitting the segment at the wrap.
__device__ __forceinline__ void bulk_row(float* dst, const float* plane, int gy, int xs, int len,
                                         int nx, uint64_t* bar) {
    int off = 0;
    while (off < len) {
        const int gx = wrapc(xs + off, nx);
        const int n = min(len - off, nx - gx);
        tfp::bulk_g2s(dst + off, plane + (long long)gy * nx + gx, (uint32_t)n * 4u, bar);
        off += n;
    }
}

__device__ __forceinline__ void prefetch_row(const float* plane, int gy, int xs, int len, int nx) {
    int off = 0;
    while (off < len) {
        const int gx = wrapc(xs + off, nx);
        const int n = min(len - off, nx - gx);
        tfp::prefetch_l2(plane + (long long)gy * nx + gx, (uint32_t)n * 4u);
        off += n;
    }
}

template <bool DO_FD, bool DO_LBM>
__global__ void __launch_bounds__(NT, 2)
k_fused(const float* __restrict__ fsrc, float* __restrict__ fdst,
        const float* __restrict__ phi_in, float* __restrict__ phi_out,
        const float* __restrict__ Q_in, float* __restrict__ Q_out,
        const float* __restrict__ u_in, float* __restrict__ u_out,
        const DevParams* __restrict__ prm, int nx, int ny, int* __restrict__ err) {
    using G = Geo<DO_FD, DO_LBM>;
    constexpr int RH = G::RH, W = G::W, H = G::H, A = G::A;
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(8) uint64_t bar;
    Sm s;
#pragma unroll
    for (int k = 0; k < 8; ++k) s.p[k] = smem + k * A;
    const int b = blockIdx.z;
    const long long N = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const DevParams& P = prm[b];
    // 16-byte bulk copies need every row start on a 16-byte boundary.
    const bool bulk = (nx & 3) == 0;

    // ---- stage 1: tile loads (and population prefetch)
    const float* gsrc[G::NLOAD];
    int sdst[G::NLOAD];
    gsrc[0] = phi_in + b * N;
    sdst[0] = P_PHI;
    gsrc[1] = Q_in + 2 * b * N;
    sdst[1] = P_QA;
    gsrc[2] = Q_in + (2 * b + 1) * N;
    sdst[2] = P_QB;
    if constexpr (DO_FD) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gsrc[3 + k] = u_in + (4 * b + k) * N;
            sdst[3 + k] = P_U1X + k;
        }
    }
    if (bulk) {
        if (threadIdx.x == 0) {
            tfp::mbar_init(&bar, 1);
            tfp::fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0)
            tfp::mbar_arrive_expect_tx(&bar, (uint32_t)(G::NLOAD * A * sizeof(float)));
        for (int t = threadIdx.x; t < G::NLOAD * H; t += NT) {
            const int pl = t / H, ly = t - pl * H;
            const int gy = wrapc(y0 - RH + ly, ny);
            bulk_row(s.p[sdst[pl]] + ly * W, gsrc[pl], gy, x0 - RH, W, nx, &bar);
        }
        if constexpr (DO_LBM) {
            const float* F = fsrc + 18 * b * N;
            for (int t = threadIdx.x; t < 18 * (TY + 2); t += NT) {
                const int i = t / (TY + 2), r = t - i * (TY + 2);
                prefetch_row(F + (long long)i * N, wrapc(y0 - 1 + r, ny), x0 - 4, TX + 8, nx);
            }
        }
        const bool ok = tfp::wait_bounded(&bar, 0, kWaitPolls);
        if (__syncthreads_or(!ok)) {
            // A bulk copy did not complete: report, give in-flight copies a
            // bounded chance to land in this CTA's shared memory, and leave.
            if (threadIdx.x == 0) atomicExch(err, TF_ERR_TIMEOUT);
            tfp::wait_bounded(&bar, 0, kWaitPolls);
            return;
        }
    } else {
        for (int i = threadIdx.x; i < A; i += NT) {
            const int ly = i / W, lx = i - ly * W;
            const long long g = (long long)wrapc(y0 - RH + ly, ny) * nx + wrapc(x0 - RH + lx, nx);
#pragma unroll
            for (int pl = 0; pl < G::NLOAD; ++pl) s.p[sdst[pl]][i] = gsrc[pl][g];
        }
        __syncthreads();
    }

    // ---- stage 2: sub-steps of the pending FD
    if constexpr (DO_FD) {
#pragma unroll 1
        for (int st = 0; st < NS_FUSED; ++st) {
            const int rp = G::R_END + 2 * (NS_FUSED - 1 - st);
            const int rq = G::R_END + (NS_FUSED - 1 - st);
            fd_substep<RH, W, G::SLOTS>(P, s, rp, rq);
        }
    }

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if constexpr (DO_LBM) {
        // ---- stage 3a: chemical potential and fluid-1 stress on radius 1
        {
            const float* phi = s.p[P_PHI];
            const float* qa = s.p[P_QA];
            const float* qb = s.p[P_QB];
            constexpr int w = TX + 2, cnt = w * (TY + 2);
            for (int idx = threadIdx.x; idx < cnt; idx += NT) {
                const int ly = idx / w, lx = idx - ly * w;
                const int c = (RH - 1 + ly) * W + RH - 1 + lx;
                const tfd::SiteStress r = tfd::site_stress(
                    P, phi[c], phi[c + 1], phi[c - 1], phi[c + W], phi[c - W], qa[c], qa[c + 1],
                    qa[c - 1], qa[c + W], qa[c - W], qb[c], qb[c + 1], qb[c - 1], qb[c + W],
                    qb[c - W]);
                s.p[P_MU][c] = r.mu;
                s.p[P_U1X][c] = r.sxx;
                s.p[P_U1Y][c] = r.sxy;
                s.p[P_U2X][c] = r.syx;
                s.p[P_U2Y][c] = r.syy;
            }
        }
        __syncthreads();
        // ---- stage 3b: interior forces, pull, moments, drag, collide, store
        const float* phi = s.p[P_PHI];
        const float* mu = s.p[P_MU];
        const float* sxx = s.p[P_U1X];
        const float* sxy = s.p[P_U1Y];
        const float* syx = s.p[P_U2X];
        const float* syy = s.p[P_U2Y];
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
            const float d = phi[c];
            const tfd::SiteForce Fo = tfd::site_force(
                P, d, phi[c + 1], phi[c - 1], phi[c + W], phi[c - W], mu[c], mu[c + 1],
                mu[c - 1], mu[c + W], mu[c - W], sxx[c + 1], sxx[c - 1], sxy[c + W], sxy[c - W],
                syx[c + 1], syx[c - 1], syy[c + W], syy[c - W]);
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
            po[g] = s.p[P_PHI][c];
            qo[g] = s.p[P_QA][c];
            qo[N + g] = s.p[P_QB][c];
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
        d.u[uc ^ 1], d.prm, ctx->nx, ctx->ny, d.flags);
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
