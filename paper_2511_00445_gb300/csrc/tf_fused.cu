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
};

// Dynamic shared memory: eight planes of A floats each, in this order.
extern __shared__ __align__(16) float tf_smem[];
enum { P_PHI = 0, P_MU, P_U1X, P_U1Y, P_U2X, P_U2Y, P_QA, P_QB };

// One forward-Euler sub-step: phi on the neighbourhood of radius rp, Q on rq.
//
// Each warp owns a band of consecutive rows of the neighbourhood across its
// whole width: lane l holds the column slots q = l and q = l + 32, where slot
// q is neighbourhood column q - 1 (slots 0 and w + 1 are the one-site halo).
// A warp walks its band top to bottom keeping the previous, current and next
// rows of the fields it needs in registers, so y-neighbours come from
// registers, x-neighbours of read-only planes from shared memory and the
// x-neighbours of the flux J_x by warp shuffles.  Rows are written back in
// place as soon as they are computed; the rows just above and below a band
// belong to other warps and are captured in registers before a barrier.
__device__ __forceinline__ void shfl_lr(float v1, float v2, int lane, float& l1, float& r1,
                                        float& l2, float& r2) {
    const unsigned FULL = 0xffffffffu;
    const float up1 = __shfl_up_sync(FULL, v1, 1), up2 = __shfl_up_sync(FULL, v2, 1);
    const float dn1 = __shfl_down_sync(FULL, v1, 1), dn2 = __shfl_down_sync(FULL, v2, 1);
    const float q31 = __shfl_sync(FULL, v1, 31), q32 = __shfl_sync(FULL, v2, 0);
    l1 = up1;
    r1 = lane == 31 ? q32 : dn1;
    l2 = lane == 0 ? q31 : up2;
    r2 = dn2;
}

template <int RH, int W, int A>
__device__ __forceinline__ void fd_substep(const DevParams& P, int rp, int rq) {
    float* __restrict__ phi = tf_smem + P_PHI * A;
    float* __restrict__ mu = tf_smem + P_MU * A;
    const float* __restrict__ u1x = tf_smem + P_U1X * A;
    const float* __restrict__ u1y = tf_smem + P_U1Y * A;
    const float* __restrict__ u2x = tf_smem + P_U2X * A;
    const float* __restrict__ u2y = tf_smem + P_U2Y * A;
    float* __restrict__ qa = tf_smem + P_QA * A;
    float* __restrict__ qb = tf_smem + P_QB * A;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;

    // (a) chemical potential on radius ra = rp + 1 (reads phi on ra + 1)
    {
        const int ra = rp + 1, w = TX + 2 * ra, h = TY + 2 * ra, o = RH - ra;
        const int bh = (h + NW - 1) / NW, y0 = warp * bh, y1 = min(h, y0 + bh);
        for (int y = y0; y < y1; ++y) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int x = lane + 32 * k;
                if (x < w) {
                    const int c = (o + y) * W + o + x;
                    const float d = phi[c];
                    const float lapd = (phi[c + 1] + phi[c - 1]) + (phi[c + W] + phi[c - W]) - 4.f * d;
                    mu[c] = P.mu0 + d * (P.mu1 + d * (P.mu2 + d * P.mu3)) - P.kappa * lapd;
                }
            }
        }
    }
    __syncthreads();

    // (b) phi on radius rp, Q on radius rq
    const int w = TX + 2 * rp, h = TY + 2 * rp, o = RH - rp;
    const int bh = (h + NW - 1) / NW, y0 = warp * bh, y1 = min(h, y0 + bh);
    const int dq = rp - rq;                       // Q neighbourhood inside the phi one
    int col[2];                                   // shared-memory column of each slot
    bool cmp[2], cq[2];                           // slot computed for phi / for Q
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int q = lane + 32 * k;
        col[k] = o - 1 + min(q, w + 1);           // clamp idle slots onto the halo
        cmp[k] = q >= 1 && q <= w;
        cq[k] = cmp[k] && q - 1 >= dq && q - 1 < dq + TX + 2 * rq;
    }
    auto flux = [&](float pv, float v1, float v2) { return pv * (v2 + pv * (v1 - v2)); };
    // Row state of the rolling window (two column slots each).
    struct Row {
        float mu[2], ax[2], ay[2], qa[2], qb[2], jy[2], ph[2], jx[2];
    };
    Row r0, r1, r2;                               // three rows: roles rotate by renaming
    float e_ph[2], e_qa[2], e_qb[2];              // row y1 (below the band), captured early
    auto load_row = [&](Row& R, int y, bool edge) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = (o + y) * W + col[k];
            R.mu[k] = mu[c];
            R.ax[k] = u1x[c];
            R.ay[k] = u1y[c];
            if (edge) {
                R.ph[k] = e_ph[k];
                R.qa[k] = e_qa[k];
                R.qb[k] = e_qb[k];
            } else {
                R.ph[k] = phi[c];
                R.qa[k] = qa[c];
                R.qb[k] = qb[c];
            }
            const float pv = P.phi_ref + R.ph[k];
            R.jy[k] = flux(pv, R.ay[k], u2y[c]);
            R.jx[k] = flux(pv, R.ax[k], u2x[c]);
        }
    };
    // Compute row y from (Pr, Cr, Nr) = rows y-1, y, y+1 and write it back.
    auto do_row = [&](int y, const Row& Pr, const Row& Cr, const Row& Nr) {
        float jl[2], jr[2];
        shfl_lr(Cr.jx[0], Cr.jx[1], lane, jl[0], jr[0], jl[1], jr[1]);
        const bool qrow = y >= dq && y < dq + TY + 2 * rq;
        float nph[2], nqa[2], nqb[2];
        bool wq[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = (o + y) * W + col[k];
            const float lapmu = (mu[c + 1] + mu[c - 1]) + (Nr.mu[k] + Pr.mu[k]) - 4.f * Cr.mu[k];
            const float divJ = 0.5f * ((jr[k] - jl[k]) + (Nr.jy[k] - Pr.jy[k]));
            nph[k] = Cr.ph[k] + P.dt_fd * (P.M * lapmu - divJ);
            wq[k] = qrow && cq[k];
            nqa[k] = 0.f;
            nqb[k] = 0.f;
            if (wq[k]) {
                const float a = Cr.qa[k], bq = Cr.qb[k];
                const float ae = qa[c + 1], aw = qa[c - 1], be = qb[c + 1], bw = qb[c - 1];
                const float lapa = (ae + aw) + (Nr.qa[k] + Pr.qa[k]) - 4.f * a;
                const float lapb = (be + bw) + (Nr.qb[k] + Pr.qb[k]) - 4.f * bq;
                const float cqf = -(P.A_Q + P.C_Q * (a * a + bq * bq));
                const float hh = cqf * a + P.K * lapa;
                const float g = cqf * bq + P.K * lapb;
                const float Wxx = 0.5f * (u1x[c + 1] - u1x[c - 1]), Wxy = 0.5f * (Nr.ax[k] - Pr.ax[k]);
                const float Wyx = 0.5f * (u1y[c + 1] - u1y[c - 1]), Wyy = 0.5f * (Nr.ay[k] - Pr.ay[k]);
                const float trE = Wxx + Wyy;
                const float e1 = 0.5f * (Wxx - Wyy);
                const float exy = 0.5f * (Wxy + Wyx);
                const float om = Wxy - Wyx;
                const float QE2 = 4.f * (a * e1 + bq * exy);
                const float ux = Cr.ax[k], uy = Cr.ay[k];
                const float adv_a = ux * 0.5f * (ae - aw) + uy * 0.5f * (Nr.qa[k] - Pr.qa[k]);
                const float adv_b = ux * 0.5f * (be - bw) + uy * 0.5f * (Nr.qb[k] - Pr.qb[k]);
                const float ra = -adv_a + P.lam * (trE * a + e1 - QE2 * a) + om * bq + P.GammaQ * hh;
                const float rb = -adv_b + P.lam * (trE * bq + exy - QE2 * bq) - om * a + P.GammaQ * g;
                nqa[k] = a + P.dt_fd * ra;
                nqb[k] = bq + P.dt_fd * rb;
            }
        }
        __syncwarp();   // every lane has read row y (x-neighbours) before it is overwritten
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = (o + y) * W + col[k];
            if (cmp[k]) phi[c] = nph[k];
            if (wq[k]) {
                qa[c] = nqa[k];
                qb[c] = nqb[k];
            }
        }
    };
    if (y0 < y1) {
        load_row(r0, y0 - 1, false);
        load_row(r1, y0, false);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int ce = (o + y1) * W + col[k];
            e_ph[k] = phi[ce];
            e_qa[k] = qa[ce];
            e_qb[k] = qb[ce];
        }
    }
    __syncthreads();   // band edges captured before any row is overwritten
    int y = y0;
    for (; y + 3 <= y1; y += 3) {
        load_row(r2, y + 1, false);
        do_row(y, r0, r1, r2);
        load_row(r0, y + 2, false);
        do_row(y + 1, r1, r2, r0);
        load_row(r1, y + 3, y + 3 == y1);
        do_row(y + 2, r2, r0, r1);
    }
    if (y < y1) {
        load_row(r2, y + 1, y + 1 == y1);
        do_row(y, r0, r1, r2);
        ++y;
        if (y < y1) {
            load_row(r0, y + 1, y + 1 == y1);
            do_row(y, r1, r2, r0);
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
    __shared__ __align__(8) uint64_t bar;
    const int b = blockIdx.z;
    const long long N = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const DevParams P = prm[b];
    // 16-byte bulk copies need every row start on a 16-byte boundary.
    const bool bulk = (nx & 3) == 0;

    // ---- stage 1: tile loads (and population prefetch)
    // Load task pl: 0 phi, 1 Q_xx, 2 Q_xy, 3..6 u1x u1y u2x u2y.
    auto src_plane = [&](int pl) -> const float* {
        return pl == 0 ? phi_in + b * N
                       : (pl < 3 ? Q_in + (2 * b + pl - 1) * N : u_in + (4 * b + pl - 3) * N);
    };
    auto dst_plane = [&](int pl) -> float* {
        return tf_smem + (pl == 0 ? P_PHI : (pl < 3 ? P_QA + pl - 1 : P_U1X + pl - 3)) * A;
    };
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
            bulk_row(dst_plane(pl) + ly * W, src_plane(pl), gy, x0 - RH, W, nx, &bar);
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
            for (int pl = 0; pl < G::NLOAD; ++pl) dst_plane(pl)[i] = src_plane(pl)[g];
        }
        __syncthreads();
    }

    // ---- stage 2: sub-steps of the pending FD
    if constexpr (DO_FD) {
#pragma unroll 1
        for (int st = 0; st < NS_FUSED; ++st) {
            const int rp = G::R_END + 2 * (NS_FUSED - 1 - st);
            const int rq = G::R_END + (NS_FUSED - 1 - st);
            fd_substep<RH, W, A>(P, rp, rq);
        }
    }

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if constexpr (DO_LBM) {
        // ---- stage 3a: chemical potential and fluid-1 stress on radius 1
        {
            const float* phi = tf_smem + P_PHI * A;
            const float* qa = tf_smem + P_QA * A;
            const float* qb = tf_smem + P_QB * A;
            constexpr int w = TX + 2, cnt = w * (TY + 2);
            for (int idx = threadIdx.x; idx < cnt; idx += NT) {
                const int ly = idx / w, lx = idx - ly * w;
                const int c = (RH - 1 + ly) * W + RH - 1 + lx;
                const tfd::SiteStress r = tfd::site_stress(
                    P, phi[c], phi[c + 1], phi[c - 1], phi[c + W], phi[c - W], qa[c], qa[c + 1],
                    qa[c - 1], qa[c + W], qa[c - W], qb[c], qb[c + 1], qb[c - 1], qb[c + W],
                    qb[c - W]);
                tf_smem[P_MU * A + c] = r.mu;
                tf_smem[P_U1X * A + c] = r.sxx;
                tf_smem[P_U1Y * A + c] = r.sxy;
                tf_smem[P_U2X * A + c] = r.syx;
                tf_smem[P_U2Y * A + c] = r.syy;
            }
        }
        __syncthreads();
        // ---- stage 3b: interior forces, pull, moments, drag, collide, store
        const float* phi = tf_smem + P_PHI * A;
        const float* mu = tf_smem + P_MU * A;
        const float* sxx = tf_smem + P_U1X * A;
        const float* sxy = tf_smem + P_U1Y * A;
        const float* syx = tf_smem + P_U2X * A;
        const float* syy = tf_smem + P_U2Y * A;
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
            po[g] = tf_smem[P_PHI * A + c];
            qo[g] = tf_smem[P_QA * A + c];
            qo[N + g] = tf_smem[P_QB * A + c];
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
