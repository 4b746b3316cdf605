// Device code of the fused coupled step, shared by the per-context kernel
// (tf_fused.cu) and the persistent ensemble kernel (tf_ensemble.cu).
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
// One CTA owns an interior tile of tw x th sites of one instance (tw <= 32 or
// 40 columns, th <= 32 or 30 rows, fixed per launch by the host; see Geo):
//  1. the phi, Q and u planes of the tile plus a halo are brought into shared
//     memory by bulk copies (one per row segment, periodic wrap handled by
//     splitting segments), and the population rows the tile will pull are
//     prefetched into L2 so that they stream from HBM during step 2;
//  2. FD(k) runs in shared memory on shrinking neighbourhoods of the tile
//     (phi loses two sites of halo per sub-step through lap(mu), Q one site);
//     each sub-step computes mu, then the new phi and Q into registers, then
//     writes them back in place, separated by barriers;
//  3. mu and the fluid-1 stress on radius 1, then per interior site the
//     forces, pulled populations, drag solve, collision and stores.
#pragma once

#include "tf_check.cuh"
#include "tf_device.cuh"
#include "tf_internal.h"
#include "tf_pair.cuh"
#include "tf_ptx.cuh"

namespace {

constexpr int TX = 32;              // width of the narrow tiles (per-context and ensemble)
constexpr int TY_DEFAULT = 32;      // height of the narrow per-context tiles
// Wide per-context tiles for grids of several waves (see Geo): 40 x 30 fills
// the 32 column-pair lanes at the widest sub-step in 108 KB of shared memory.
constexpr int TX_WIDE = 40;
constexpr int TY_WIDE = 30;
constexpr int NT = 256;        // threads per CTA: 32 x 8
constexpr int NS_FUSED = 5;    // sub-steps handled by the fused kernel (Sec. III)
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ int wrapc(int v, int n) {
    if ((unsigned)v < (unsigned)n) return v;
    if (v < 0 && v >= -n) return v + n;
    if (v >= n && v < 2 * n) return v - n;
    v %= n;     // several periods outside [0, n): tiny grids only
    return v < 0 ? v + n : v;
}

constexpr int round4(int v) { return (v + 3) & ~3; }

// First column of tile column k of ntx (k = ntx gives nx): when nx is a
// multiple of 4 every tile starts on a multiple of 4 (16-byte rows for the
// bulk copies); widths differ by at most 4.
__host__ __device__ inline int tile_col(int k, int ntx, int nx) {
    return nx % 4 == 0 ? 4 * (int)((long long)k * (nx / 4) / ntx) : (int)((long long)k * nx / ntx);
}

// TXM: the widest tile.  A warp row of a sub-step costs the same however
// many of its 32 column pairs are used, so sub-step work per site falls with
// the tile width; 40 columns plus the widest neighbourhood (2 x 11) plus the
// one-column halo of each side fill exactly 64 columns.
template <bool DO_FD, bool DO_LBM, int TY, int TXM = TX>
struct Geo {
    static constexpr int R_END = DO_LBM ? 2 : 0;                  // phi/Q radius after FD
    static constexpr int RH_NEED = R_END + (DO_FD ? 2 * NS_FUSED : 0);
    static constexpr int RH = round4(RH_NEED < 4 ? 4 : RH_NEED);  // loaded halo, 16-byte aligned
    static constexpr int W = TXM + 2 * RH;
    // lanes of the widest paired row (PairCols): the chemical potential of the
    // first sub-step on radius RH_NEED - 1, or the stress stage on radius 1
    static constexpr int RA = DO_FD ? RH_NEED - 1 : 1;
    static constexpr int LANES = ((RH - RA + TXM + 2 * RA) >> 1) - ((RH - RA - 1) >> 1) + 1;
    static_assert(LANES <= 32, "widest paired row within the 32 lanes of a warp");
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
// whole width; lane l holds one pair of adjacent columns (64-bit shared loads,
// paired FP32 arithmetic).  A warp walks its band top to bottom keeping rows
// y-1, y, y+1 in registers (roles rotate by renaming), so y-neighbours come
// from registers and x-neighbours from warp shuffles.  Rows are written back
// in place (a lane touches only its own columns in shared memory); the rows
// just above and below a band belong to other warps and are captured in
// registers before a barrier.
template <int RH, int W, int A>
__device__ __forceinline__ void fd_substep(const DevParams& P, int tw, int th, int rp, int rq) {
    using namespace tfq;
    float* __restrict__ phi = tf_smem + P_PHI * A;
    float* __restrict__ mu = tf_smem + P_MU * A;
    const float* __restrict__ u1x = tf_smem + P_U1X * A;
    const float* __restrict__ u1y = tf_smem + P_U1Y * A;
    const float* __restrict__ u2x = tf_smem + P_U2X * A;
    const float* __restrict__ u2y = tf_smem + P_U2Y * A;
    float* __restrict__ qa = tf_smem + P_QA * A;
    float* __restrict__ qb = tf_smem + P_QB * A;
    // warp index shuffled from lane 0, so that the compiler keeps the
    // warp-uniform row arithmetic in uniform registers (2048^2: 315 -> 307 us)
    const int lane = threadIdx.x & 31, warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
    constexpr int NW = NT / 32;
    const f2 mu0 = S2(P.mu0), mu1 = S2(P.mu1), mu2 = S2(P.mu2), mu3 = S2(P.mu3);
    const f2 kap = S2(-P.kappa), m4 = S2(-4.f), half = S2(0.5f), cref = S2(P.phi_ref);

    // (a) chemical potential on radius ra = rp + 1 (reads phi on ra + 1)
    {
        const int ra = rp + 1, w = tw + 2 * ra, h = th + 2 * ra, o = RH - ra;
        const PairCols pc(o, w, lane);
        const int bh = (h + NW - 1) / NW, y0 = warp * bh, y1 = min(h, y0 + bh);
        if (y0 < y1) {
            constexpr int H = A / W;
            const float* col = phi + TF_BC(pc.c0, W - 1);
            f2 pp = ld2(col + TF_BC(o + y0 - 1, H) * W), pcur = ld2(col + TF_BC(o + y0, H) * W);
            for (int y = y0; y < y1; ++y) {
                const f2 pn = ld2(col + TF_BC(o + y + 1, H) * W);
                const f2 lap = F2(m4, pcur, A2(hsum2(pcur), A2(pp, pn)));
                const f2 poly = F2(pcur, F2(pcur, F2(pcur, mu3, mu2), mu1), mu0);
                st_pair(mu + TF_BC((o + y) * W + pc.c0, A - 1), F2(kap, lap, poly), pc.st);
                pp = pcur;
                pcur = pn;
            }
        }
    }
    __syncthreads();

    // (b) phi on radius rp, Q on radius rq
    const int w = tw + 2 * rp, h = th + 2 * rp, o = RH - rp;
    const PairCols pc(o, w, lane);
    const int bh = (h + NW - 1) / NW, y0 = warp * bh, y1 = min(h, y0 + bh);
    const int oq = RH - rq, wq = tw + 2 * rq;     // Q neighbourhood (shared coordinates)
    const bool qs = pc.meets(oq, wq);
    // Forward Euler with dt and the factors 1/2 of the central differences
    // folded into the coefficients (Eq. 1 and Eqs. 11-12):
    //   phi' = phi + (dt/2) [2M lap(mu) - (J_x(+x) - J_x(-x) + J_y(+y) - J_y(-y))]
    //   a'   = a + [c a + dt Gamma K lap(a) + (dt lam / 4) E1 + (dt/2) O b - (dt/2) u1.D a]
    //   b'   = b + [c b + dt Gamma K lap(b) + (dt lam / 4) EX - (dt/2) O a - (dt/2) u1.D b]
    // with D the undivided central differences (D_x v = v(+x) - v(-x)) and
    //   E1 = D_x u_x - D_y u_y, EX = D_y u_x + D_x u_y, O = D_y u_x - D_x u_y,
    //   c  = -dt Gamma (A_Q + C_Q q^2) + dt lam ((D_x u_x + D_y u_y)/2 - (a E1 + b EX)).
    // The bracket is dt [Gamma H + S - u1.grad Q] with H and S as in the
    // device helpers: tr E = (D_x u_x + D_y u_y)/2, E0 = (E1, EX)/4,
    // 4 (Q:E0)/2 = a E1 + b EX, and the rotation part om (b, -a), om = O/2.
    // Each field takes its increment in one final addition: a constant such as
    // 1 - dt Gamma A_Q, rounded once and applied to the field every sub-step,
    // would bias the field itself, not just its increment.
    const float dt = P.dt_fd, dG = __fmul_rn(dt, P.GammaQ), hdt = 0.5f * dt;
    const f2 M2x = S2(2.f * P.M), nhdt = S2(-hdt), hdt2 = S2(hdt);
    const f2 cGA = S2(-__fmul_rn(dG, P.A_Q)), cGC = S2(-__fmul_rn(dG, P.C_Q));
    const f2 cGK = S2(__fmul_rn(dG, P.K)), lamd = S2(__fmul_rn(dt, P.lam));
    const f2 lamq = S2(0.25f * __fmul_rn(dt, P.lam));
    auto flux = [&](f2 pv, f2 v1, f2 v2) { return M2(pv, F2(pv, B2(v1, v2), v2)); };
    struct Row {
        f2 mu, ax, ay, qa, qb, jy, ph, jx;
    };
    Row r0, r1, r2;                               // three rows: roles rotate by renaming
    f2 e_ph, e_qa, e_qb;                          // row y1 (below the band), captured early
    auto load_row = [&](Row& R, int y, bool edge) {
        const int c = TF_BC((o + y) * W + pc.c0, A - 1);
        R.mu = ld2(mu + c);
        R.ax = ld2(u1x + c);
        R.ay = ld2(u1y + c);
        if (edge) {
            R.ph = e_ph;
            R.qa = e_qa;
            R.qb = e_qb;
        } else {
            R.ph = ld2(phi + c);
            R.qa = ld2(qa + c);
            R.qb = ld2(qb + c);
        }
        const f2 pv = A2(cref, R.ph);
        R.jy = flux(pv, R.ay, ld2(u2y + c));
        R.jx = flux(pv, R.ax, ld2(u2x + c));
    };
    // Compute row y from (Pr, Cr, Nr) = rows y-1, y, y+1 and write it back.
    auto do_row = [&](int y, const Row& Pr, const Row& Cr, const Row& Nr) {
        const f2 dJ = A2(hdiff2(Cr.jx), B2(Nr.jy, Pr.jy));
        const f2 lapmu = F2(m4, Cr.mu, A2(hsum2(Cr.mu), A2(Nr.mu, Pr.mu)));
        const f2 nph = F2(hdt2, F2(M2x, lapmu, N2(dJ)), Cr.ph);
        const int row = o + y;
        const bool qrow = row >= oq && row < oq + th + 2 * rq;
        // A lane reads and writes only its own columns (x-neighbours come by
        // shuffle), so row y is overwritten in place without a warp barrier.
        const int c = TF_BC(row * W + pc.c0, A - 1);
        st_pair(phi + c, nph, pc.st);
        // Q on every row, stored only inside its neighbourhood (the rows read
        // lie inside phi's): the row stays one basic block, so the phi and Q
        // chains of consecutive rows interleave.
        {
            f2 ah, ax, bh, bx;
            hsd2(Cr.qa, ah, ax);
            hsd2(Cr.qb, bh, bx);
            const f2 a = Cr.qa, bq = Cr.qb;
            const f2 lapa = F2(m4, a, A2(ah, A2(Nr.qa, Pr.qa)));
            const f2 lapb = F2(m4, bq, A2(bh, A2(Nr.qb, Pr.qb)));
            const f2 cg = F2(cGC, F2(a, a, M2(bq, bq)), cGA);      // -dt Gamma (A_Q + C_Q q^2)
            const f2 Dxx = hdiff2(Cr.ax), Dyy = B2(Nr.ay, Pr.ay);
            const f2 Dxy = B2(Nr.ax, Pr.ax), Dyx = hdiff2(Cr.ay);
            const f2 E1 = B2(Dxx, Dyy), EX = A2(Dxy, Dyx);
            const f2 t1 = F2(half, A2(Dxx, Dyy), N2(F2(a, E1, M2(bq, EX))));
            const f2 cc = F2(lamd, t1, cg);
            const f2 hO = M2(hdt2, B2(Dxy, Dyx));
            const f2 nux = M2(nhdt, Cr.ax), nuy = M2(nhdt, Cr.ay);
            const f2 nqa = A2(a, F2(cc, a, F2(cGK, lapa, F2(lamq, E1, F2(hO, bq,
                                  F2(nux, ax, M2(nuy, B2(Nr.qa, Pr.qa))))))));
            const f2 nqb = A2(bq, F2(cc, bq, F2(cGK, lapb, F2(lamq, EX, F2(N2(hO), a,
                                  F2(nux, bx, M2(nuy, B2(Nr.qb, Pr.qb))))))));
            st_pair(qa + c, nqa, qs && qrow);
            st_pair(qb + c, nqb, qs && qrow);
        }
    };
    if (y0 < y1) {
        load_row(r0, y0 - 1, false);
        load_row(r1, y0, false);
        const int ce = TF_BC((o + y1) * W + pc.c0, A - 1);
        e_ph = ld2(phi + ce);
        e_qa = ld2(qa + ce);
        e_qb = ld2(qb + ce);
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
        const int gx = TF_BC(wrapc(xs + off, nx), nx);
        const int n = min(len - off, nx - gx);
        tfp::bulk_g2s(dst + off, plane + (long long)gy * nx + gx, (uint32_t)n * 4u, bar);
        off += n;
    }
}

// L2 prefetch hint for elements [c0, c1] (c0 <= c1) of one row: one
// per-thread prefetch per 128-byte line, every address inside the range.
// (Bulk prefetches through the copy engine were slower: it handles many
// small requests slowly.)
template <typename T>
__device__ __forceinline__ void prefetch_span(const T* row, int c0, int c1) {
    const char* const p0 = reinterpret_cast<const char*>(row + c0);
    const char* const p1 = reinterpret_cast<const char*>(row + c1);
    for (const char* q = p0; q < p1; q += 128) tfp::prefetch_l2_line(q);
    tfp::prefetch_l2_line(p1);
}

// Device pointers and sizes of one stepping launch (one group of instances
// with one grid size); src/in buffers hold the current state, dst/out the next.
template <class S>
struct TileArgs {
    const typename S::T* fsrc;
    typename S::T* fdst;
    const float* phi_in;
    float* phi_out;
    const float* Q_in;
    float* Q_out;
    const float* u_in;
    float* u_out;
    const DevParams* prm;
    int nx, ny;
    int* err;
};

// One tile of tw <= TXM columns and th <= TY rows (origin x0, y0) of instance b:
// loads, pending sub-steps, LBM, stores.  Every value a tile stores depends
// only on the state inside its dependency cone, so results do not depend on
// how the grid is cut into tiles.  `bar` is this CTA's initialised mbarrier and `phase` the
// number of tiles the CTA has already loaded with it (the wait parity).  A CTA
// that processes several tiles must pass through __syncthreads() between
// them (each thread ends a tile with a generic-to-async proxy fence).
// Returns false after a bulk-copy timeout (reported in *err).
// MULTI: the launch runs several steps, so the population source was written
// by other CTAs earlier in the same launch; it is then read through L2 only.
template <bool DO_FD, bool DO_LBM, class S, int TY, bool MULTI = false, int TXM = TX>
__device__ __forceinline__ bool fused_tile(const TileArgs<S>& a, int b, int x0, int y0, int tw,
                                           int th, uint64_t* bar, uint32_t phase) {
    using G = Geo<DO_FD, DO_LBM, TY, TXM>;
    constexpr int RH = G::RH, W = G::W, H = G::H, A = G::A;
    const typename S::T* __restrict__ fsrc = a.fsrc;
    typename S::T* __restrict__ fdst = a.fdst;
    const float* __restrict__ phi_in = a.phi_in;
    float* __restrict__ phi_out = a.phi_out;
    const float* __restrict__ Q_in = a.Q_in;
    float* __restrict__ Q_out = a.Q_out;
    const float* __restrict__ u_in = a.u_in;
    float* __restrict__ u_out = a.u_out;
    const int nx = a.nx, ny = a.ny;
    const long long N = (long long)nx * ny;
    const DevParams P = a.prm[b];
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
    const int hr = th + 2 * RH;     // loaded rows (<= H)
    const int wr = tw + 2 * RH;     // loaded columns (<= W; a multiple of 4 whenever bulk)
    if (bulk) {
        if (threadIdx.x == 0)
            tfp::mbar_arrive_expect_tx(bar, (uint32_t)(G::NLOAD * hr * wr * sizeof(float)));
        for (int t = threadIdx.x; t < G::NLOAD * H; t += NT) {
            const int pl = t / H, ly = t - pl * H;
            if (ly >= hr) continue;
            const int gy = wrapc(y0 - RH + ly, ny);
            bulk_row(dst_plane(pl) + ly * W, src_plane(pl), gy, x0 - RH, wr, nx, bar);
        }
        if (DO_LBM) {
            // the population rows the tile pulls (the fluid pairs of columns
            // x0 - 1 .. x0 + tw) into L2, so that they stream from HBM during
            // the sub-steps
            for (int t = threadIdx.x; t < 9 * (TY + 2); t += NT) {
                const int i = t / (TY + 2), r = t - i * (TY + 2);
                if (r >= th + 2) continue;
                prefetch_span(fsrc + pop_index(b, 0, i, (long long)wrapc(y0 - 1 + r, ny) * nx, N),
                              2 * max(x0 - 1, 0), 2 * min(x0 + tw, nx - 1) + 1);
            }
        }
        const bool ok = tfp::wait_bounded(bar, phase & 1u, kWaitPolls);
        if (__syncthreads_or(!ok)) {
            // A bulk copy did not complete: report, give in-flight copies a
            // bounded chance to land in this CTA's shared memory, and leave.
            if (threadIdx.x == 0) atomicExch(a.err, TF_ERR_TIMEOUT);
            tfp::wait_bounded(bar, phase & 1u, kWaitPolls);
            return false;
        }
    } else {
        for (int i = threadIdx.x; i < hr * wr; i += NT) {
            const int ly = i / wr, lx = i - ly * wr;
            const long long g = (long long)wrapc(y0 - RH + ly, ny) * nx + wrapc(x0 - RH + lx, nx);
#pragma unroll
            for (int pl = 0; pl < G::NLOAD; ++pl)
                dst_plane(pl)[ly * W + lx] = MULTI ? __ldcg(src_plane(pl) + g) : src_plane(pl)[g];
        }
        __syncthreads();
    }

    // ---- stage 2: sub-steps of the pending FD (unrolled: the radii are
    // constants in each copy)
    if constexpr (DO_FD) {
#pragma unroll
        for (int st = 0; st < NS_FUSED; ++st) {
            const int rp = G::R_END + 2 * (NS_FUSED - 1 - st);
            const int rq = G::R_END + (NS_FUSED - 1 - st);
            fd_substep<RH, W, A>(P, tw, th, rp, rq);
        }
    }

    const int tx = threadIdx.x & 31, ty = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
    if constexpr (DO_LBM) {
        using namespace tfq;
        // ---- stage 3a: chemical potential and fluid-1 stress on radius 1
        // (paired column walk like the sub-steps; results go to the mu plane
        // and to the four u planes, free after the sub-steps)
        {
            const float* phi = tf_smem + P_PHI * A;
            const float* qa = tf_smem + P_QA * A;
            const float* qb = tf_smem + P_QB * A;
            constexpr int o = RH - 1, NW = NT / 32;
            const int w = tw + 2, h = th + 2;
            const PairCols pc(o, w, tx);
            const int bh = (h + NW - 1) / NW;
            const int y0 = ty * bh, y1 = min(h, y0 + bh);
            if (y0 < y1) {
                const int col = pc.c0;
                f2 dp = ld2(phi + (o + y0 - 1) * W + col), dc = ld2(phi + (o + y0) * W + col);
                f2 ap = ld2(qa + (o + y0 - 1) * W + col), ac = ld2(qa + (o + y0) * W + col);
                f2 bp = ld2(qb + (o + y0 - 1) * W + col), bc = ld2(qb + (o + y0) * W + col);
                for (int y = y0; y < y1; ++y) {
                    const int cn = TF_BC((o + y + 1) * W + col, A - 1), cc = TF_BC((o + y) * W + col, A - 1);
                    const f2 dn = ld2(phi + cn), an = ld2(qa + cn), bn = ld2(qb + cn);
                    f2 ah, ax, bh, bx;
                    hsd2(ac, ah, ax);
                    hsd2(bc, bh, bx);
                    const PairStress r =
                        stress2(P, dc, hsum2(dc), dn, dp, ac, ah, ax, an, ap, bc, bh, bx, bn, bp);
                    st_pair(tf_smem + P_MU * A + cc, r.mu, pc.st);
                    st_pair(tf_smem + P_U1X * A + cc, r.sxx, pc.st);
                    st_pair(tf_smem + P_U1Y * A + cc, r.sxy, pc.st);
                    st_pair(tf_smem + P_U2X * A + cc, r.syx, pc.st);
                    st_pair(tf_smem + P_U2Y * A + cc, r.syy, pc.st);
                    dp = dc;
                    dc = dn;
                    ap = ac;
                    ac = an;
                    bp = bc;
                    bc = bn;
                }
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
        using T2 = typename S::T2;
        const T2* F1 = reinterpret_cast<const T2*>(fsrc + pop_index(b, 0, 0, 0, N));
        T2* D1 = reinterpret_cast<T2*>(fdst + pop_index(b, 0, 0, 0, N));
        float* uo = u_out + 4 * b * N;
        // the LBM update of site (r, cx) of the tile
        auto lbm_site = [&](int r, int cx) {
            const int x = x0 + cx, y = y0 + r;
            if (x >= nx || y >= ny) return;
            const int c = TF_BC((RH + r) * W + RH + cx - W - 1, A - 2 * W - 2) + W + 1;
            const int xp = x + 1 < nx ? x + 1 : 0, xm = x > 0 ? x - 1 : nx - 1;
            const int yp = y + 1 < ny ? y + 1 : 0, ym = y > 0 ? y - 1 : ny - 1;
            f2 f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sx = d2q9_cx(i) == 0 ? x : (d2q9_cx(i) > 0 ? xm : xp);
                const int sy = d2q9_cy(i) == 0 ? y : (d2q9_cy(i) > 0 ? ym : yp);
                const long long src = TF_BC64((long long)sy * nx + sx, N);
                if constexpr (MULTI)
                    f[i] = S::load2_cg(F1 + i * N + src);
                else
                    f[i] = S::load2(F1 + i * N + src);
            }
            f2 u1, u2;
            lbm_site2(P, phi[c], P2(phi[c - 1], phi[c + 1]), P2(phi[c - W], phi[c + W]), mu[c],
                      P2(mu[c - 1], mu[c + 1]), P2(mu[c - W], mu[c + W]), P2(sxx[c - 1], sxx[c + 1]),
                      P2(sxy[c - W], sxy[c + W]), P2(syx[c - 1], syx[c + 1]),
                      P2(syy[c - W], syy[c + W]), f, u1, u2);
            const long long g = TF_BC64((long long)y * nx + x, N);
#pragma unroll
            for (int i = 0; i < 9; ++i) S::store2(D1 + i * N + g, f[i]);
            uo[g] = u1.x;
            uo[N + g] = u1.y;
            uo[2 * N + g] = u2.x;
            uo[3 * N + g] = u2.y;
        };
        if (tw == 32) {
            // one tile row per warp pass, one column per lane (y uniform in a warp)
#pragma unroll 1
            for (int r = ty; r < th; r += NT / 32) lbm_site(r, tx);
        } else {
            // the tile's tw x th sites in row-major order, one per thread (a warp
            // may span two rows); (r, cx) advance by NT sites per pass
            int r = threadIdx.x / tw, cx = threadIdx.x - r * tw;
            const int dr = NT / tw, dc = NT - dr * tw;
#pragma unroll 1
            for (int site = threadIdx.x; site < tw * th; site += NT) {
                lbm_site(r, cx);
                cx += dc;
                r += dr;
                if (cx >= tw) {
                    cx -= tw;
                    ++r;
                }
            }
        }
    }
    if constexpr (DO_FD) {
        // ---- store phi^{k+1}, Q^{k+1} of the interior
        float* po = phi_out + b * N;
        float* qo = Q_out + 2 * b * N;
        for (int site = threadIdx.x; site < tw * th; site += NT) {
            const int r = site / tw, cx = site - r * tw;
            const int x = x0 + cx, y = y0 + r;
            if (x >= nx || y >= ny) continue;
            const int c = TF_BC((RH + r) * W + RH + cx, A);
            const long long g = TF_BC64((long long)y * nx + x, N);
            po[g] = tf_smem[P_PHI * A + c];
            qo[g] = tf_smem[P_QA * A + c];
            qo[N + g] = tf_smem[P_QB * A + c];
        }
    }
    // The next tile's bulk copies (async proxy) overwrite this tile's shared
    // memory: order this thread's generic accesses before them.
    tfp::fence_proxy_async_smem();
    return true;
}

}  // namespace
