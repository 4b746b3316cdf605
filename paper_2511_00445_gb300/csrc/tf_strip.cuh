// Steady-state coupled step on large grids: the strip-streaming kernel.
//
// Same step as k_fused<1, 1> (tf_fused.cuh): the pending five Cahn-Hilliard /
// Beris-Edwards sub-steps FD(k) (Sec. III; Eq. 1, 11-12) with the stored
// velocities u^k, then LBM(k+1) (forces, pull streaming, implicit-drag Guo
// velocities, BGK + Guo collision of both D2Q9 fluids) from phi^{k+1},
// Q^{k+1}.  Every value is computed with the same correctly rounded scalar
// operations in the same order as k_fused (tfq helpers), so the two kernels
// give bitwise the same state; only the schedule differs.
//
// Schedule.  One CTA owns a strip of tw <= 96 columns and a segment of S rows
// of one instance.  Its window is the strip plus 12 columns on each side (120
// columns: 30 lanes x 4 columns), and it walks down the segment in blocks of
// R = 8 rows.  Per block every stage advances by R rows, each stage lagging
// two rows behind the one it reads:
//   input rows of phi^(0), Q^(0), u  : [L - R, L)            (asynchronous copies issued
//                                       one block ahead: phi / Q at the block's start,
//                                       u once the fifth sub-step has read its rows)
//   sub-step s = 1..5 (phi^(s), Q^(s)): [L - 2s - R, L - 2s)  (each warp one row; it
//                                       evaluates mu^(s) on its row and the two beside it)
//   stress and mu of phi^(5), Q^(5)   : [L - 11 - R, L - 11)
//   LBM, stores of the new state      : [L - 12 - R, L - 12)
// Sub-step s overwrites phi^(s-1), Q^(s-1) in place in one ring of rows; the
// rows just above its block that the next block still needs as neighbours
// (two of phi, one of Q) are saved first into per-stage shadow rows.  The
// halo shrinks with the stage (phi^(s) is exact on rows and columns within
// 12 - 2s of the segment / strip, Q^(s) within 7 - s), so nothing outside the
// window or the segment is ever needed; rows outside a stage's exact range
// are skipped, columns outside it are computed and never read.
//
// The LBM pulls its populations straight from global memory.  At the start
// of a block every CTA asks L2 for the population rows its LBM phase will pull
// (per-thread prefetch instructions, ~3 per thread; 343 -> 325 us per 2048^2
// step), each thread issues its first site's pulls before waiting for the
// stress rows its LBM row reads and the next site's pulls before computing the
// current one.  Measured and removed (2048^2, per step): bulk L2 prefetches
// through the copy engine (525 -> 442 us without them), prefetching one block
// further ahead (340 us), and loading the window rows with one bulk copy per
// row (the copy engine handles small copies slowly; per-thread 16-byte
// asynchronous copies took 399 -> 381 us for the u rows, and issuing them
// without per-row index divisions 374 -> 348 us).
#pragma once

#include "tf_check.cuh"
#include "tf_fused.cuh"

namespace {

namespace ts {
constexpr int R = 8;                    // rows per block: one per warp in the FD phases
constexpr int NW = NT / 32;
static_assert(NW == R, "one row per warp");
constexpr int HALO = 12;                // window columns on each side of the strip
constexpr int TWMAX = 96;               // widest strip
constexpr int WW = TWMAX + 2 * HALO;    // window row (floats)
constexpr int LANES = WW / 4;           // lanes holding window columns (4 each)
static_assert(WW % 4 == 0 && LANES <= 32, "window row within one warp");
constexpr int DP = 2 * R + 13;          // phi / Q ring rows
constexpr int DU = R + 11;              // u ring rows
constexpr int DS = R + 2;               // stress ring rows
constexpr int SC0 = 8;                  // first window column kept in the stress ring
constexpr int SW = 104;                 // stress ring columns [SC0, SC0 + SW)
static_assert(SC0 + SW >= HALO + TWMAX + 1 + 1 && SC0 <= HALO - 1 - 3, "stress columns cover the LBM's");
constexpr int NSUB = NS_FUSED;
// phi, Q_xx and Q_xy each have DP ring rows followed by two shadow rows per
// sub-step, at one common field stride, so a row index addresses all three.
constexpr int SH0 = DP;                              // first shadow row index
constexpr int FROWS = DP + 2 * NSUB;
constexpr int FS = FROWS * WW;                       // field stride
constexpr int OFF_PHI = 0;
constexpr int OFF_QA = OFF_PHI + FS;
constexpr int OFF_QB = OFF_QA + FS;
constexpr int OFF_U = OFF_QB + FS;                   // u1x, u1y, u2x, u2y: DU rows each
constexpr int OFF_ST = OFF_U + 4 * DU * WW;          // mu, sxx, sxy, syx, syy: DS rows x SW
constexpr int NFLOAT = OFF_ST + 5 * DS * SW;
constexpr size_t SMEM = (size_t)NFLOAT * sizeof(float);
}  // namespace ts

// Four adjacent columns of a lane as two pairs (columns 0,1 and 2,3).
struct V4 {
    tfq::f2 lo, hi;
};

__device__ __forceinline__ V4 ld4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

__device__ __forceinline__ void st4(float* p, const V4& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.lo.x, v.lo.y, v.hi.x, v.hi.y);
}

// x-neighbour sums v(x - 1) + v(x + 1) and differences v(x + 1) - v(x - 1) of
// a lane's four columns (the outer neighbours from the adjacent lanes), each
// formed by one scalar operation straight into its pair, as hsd2 does for a
// column pair (2048^2: 318 -> 301 us with the sub-step and stress phases on
// these forms).
__device__ __forceinline__ void hsd4(const V4& v, V4& s, V4& d) {
    const float up = __shfl_up_sync(0xffffffffu, v.hi.y, 1);
    const float dn = __shfl_down_sync(0xffffffffu, v.lo.x, 1);
    s = {make_float2(__fadd_rn(up, v.lo.y), __fadd_rn(v.lo.x, v.hi.x)),
         make_float2(__fadd_rn(v.lo.y, v.hi.y), __fadd_rn(v.hi.x, dn))};
    d = {make_float2(__fsub_rn(v.lo.y, up), __fsub_rn(v.hi.x, v.lo.x)),
         make_float2(__fsub_rn(v.hi.y, v.lo.y), __fsub_rn(dn, v.hi.x))};
}
__device__ __forceinline__ V4 hsum4(const V4& v) {
    V4 s, d;
    hsd4(v, s, d);
    return s;
}
__device__ __forceinline__ V4 hdiff4(const V4& v) {
    V4 s, d;
    hsd4(v, s, d);
    return d;
}

// Ring slots of segment row t (any t >= -3 DP; rows below -HALO, or -1 for
// the stress ring, are only touched by rows that are skipped).  One modulo
// per phase; neighbouring rows step from it with a conditional wrap.
__device__ __forceinline__ int pslot(int t) { return (t + ts::HALO + 3 * ts::DP) % ts::DP; }
__device__ __forceinline__ int uslot(int t) { return (t + ts::HALO + 3 * ts::DU) % ts::DU; }
__device__ __forceinline__ int sslot(int t) { return (t + 1 + 3 * ts::DS) % ts::DS; }
template <int D>
__device__ __forceinline__ int step_slot(int base, int k) {   // (base + k) mod D, 0 <= k < D
    const int v = base + k;
    return v >= D ? v - D : v;
}

template <class S>
__global__ void __launch_bounds__(NT, 2) k_strip(const TileArgs<S> a) {
    using namespace tfq;
    using ts::R;
    using ts::WW;
    float* const sm = tf_smem;
    const int b = blockIdx.z;
    const int nx = a.nx, ny = a.ny;
    const long long N = (long long)nx * ny;
    const int x0 = tile_col(blockIdx.x, gridDim.x, nx);
    const int tw = tile_col(blockIdx.x + 1, gridDim.x, nx) - x0;
    const int y0 = (int)((long long)blockIdx.y * ny / gridDim.y);
    const int SG = (int)((long long)(blockIdx.y + 1) * ny / gridDim.y) - y0;
    const DevParams P = a.prm[b];
    // The warp index through a shuffle from lane 0: the compiler then treats
    // it, and every row index and ring slot derived from it, as uniform across
    // the warp and keeps that arithmetic in uniform registers (2048^2: 276 ->
    // 269 us; 128 registers with a 24-byte spill -> 122 without).
    const int lane = threadIdx.x & 31, warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
    const int col = 4 * min(lane, ts::LANES - 1);   // this lane's first window column
    const bool own = lane < ts::LANES;
    const int nblk = (SG + 2 * ts::HALO + R - 1) / R;   // blocks (= iterations)
    TF_BC_BEGIN();
    // Warp k's stress row of the current block is stored: one mbarrier per
    // warp, all 32 lanes arrive once per block.  A warp's LBM row reads the
    // stress rows of warps k - 2 .. k only (the rows above the block came with
    // the previous one), so it waits for those three instead of the whole CTA
    // (2048^2: 266.3 -> 264.7 us).
    __shared__ __align__(8) uint64_t stress_bar[ts::NW];
    if (threadIdx.x < ts::NW) tfp::mbar_init(&stress_bar[threadIdx.x], 32);
    __syncthreads();


    // Window copies: 16-byte per-thread asynchronous copies.  Warp w copies
    // row t0 + w of an input block (all its planes), lanes 0..29 one 4-column
    // chunk each; with nx and x0 multiples of 4 no chunk straddles the
    // periodic wrap.  The rows past the segment's lower halo are not copied.
    // (Many small bulk copies are slow on the copy engine: issued as row-sized
    // bulk copies the u rows alone cost 28 us per 2048^2 step.)
    const int gx = TF_BC(wrapc(x0 - ts::HALO + col, nx), nx - 3);
    const float* const phi_src = a.phi_in + b * N + gx;
    const float* const qa_src = a.Q_in + 2 * b * N + gx;
    const float* const u_src = a.u_in + 4 * b * N + gx;
    // the phi, Q_xx, Q_xy rows of input block `blk` into their ring slots
    auto issue_pq = [&](int blk) {
        const int t = -ts::HALO + blk * R + warp;
        if (own && t < SG + ts::HALO) {
            const long long ro = (long long)TF_BC(wrapc(y0 + t, ny), ny) * nx;
            float* const d = sm + TF_BC(pslot(t), ts::DP) * WW + col;
            tfp::cp_async16(d, phi_src + ro);
            tfp::cp_async16(d + ts::FS, qa_src + ro);
            tfp::cp_async16(d + 2 * ts::FS, qa_src + N + ro);
        }
        tfp::cp_async_commit();
    };
    // the u rows of input block `blk`
    auto issue_u = [&](int blk) {
        const int t = -ts::HALO + blk * R + warp;
        if (own && t < SG + ts::HALO) {
            const float* const src = u_src + (long long)TF_BC(wrapc(y0 + t, ny), ny) * nx;
            float* const d = sm + ts::OFF_U + TF_BC(uslot(t), ts::DU) * WW + col;
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) tfp::cp_async16(d + pl * ts::DU * WW, src + pl * N);
        }
        tfp::cp_async_commit();
    };
    issue_pq(0);
    issue_u(0);

    const float m4f = -4.f;
    const f2 m4 = S2(m4f), half = S2(0.5f);
    const f2 mu0 = S2(P.mu0), mu1 = S2(P.mu1), mu2 = S2(P.mu2), mu3 = S2(P.mu3);
    const f2 kap = S2(-P.kappa), cref = S2(P.phi_ref);
    // sub-step coefficients, exactly as fd_substep forms them
    const float dt = P.dt_fd, dG = __fmul_rn(dt, P.GammaQ), hdt = 0.5f * dt;
    const f2 M2x = S2(2.f * P.M), nhdt = S2(-hdt), hdt2 = S2(hdt);
    const f2 cGA = S2(-__fmul_rn(dG, P.A_Q)), cGC = S2(-__fmul_rn(dG, P.C_Q));
    const f2 cGK = S2(__fmul_rn(dG, P.K)), lamd = S2(__fmul_rn(dt, P.lam));
    const f2 lamq = S2(0.25f * __fmul_rn(dt, P.lam));
    auto flux = [&](f2 pv, f2 v1, f2 v2) { return M2(pv, F2(pv, B2(v1, v2), v2)); };

#pragma unroll 1
    for (int j = 0; j < nblk; ++j) {
        const int L = -ts::HALO + (j + 1) * R;     // input rows < L are resident after the wait
        tfp::cp_async_wait_all();      // this block's input rows (this thread's copies)
        __syncthreads();               // ... and every other thread's
        // the next block's phi / Q rows (their ring slots were last read by
        // the previous block's LBM)
        if (j + 1 < nblk) issue_pq(j + 1);
        // L2 prefetch of the population rows [L - 19, L - 11) that this block's
        // LBM phase pulls (rows L - 21, L - 20 came with the previous block):
        // thread (direction, row) touches every 128-byte line of the fluid
        // pairs of columns [x0 - 1, x0 + tw] of its row; each address lies
        // inside the row.
        if (threadIdx.x < 9 * R) {
            const int pl = threadIdx.x / R, t = L - 19 + threadIdx.x % R;
            if (t >= -1 && t < SG + 1) {
                prefetch_span(a.fsrc + pop_index(b, 0, pl, (long long)TF_BC(wrapc(y0 + t, ny), ny) * nx, N),
                              2 * max(x0 - 1, 0), 2 * min(x0 + tw, nx - 1) + 1);
            }
        }

        // Ring row offsets of rows L - R + warp - 12 + m, m = 0 .. 12: every
        // phi / Q row this warp's sub-steps read or write in this block, each
        // slot found once per block instead of once per sub-step (uniform;
        // 269 -> 268 us)
        int offs[13];
        {
            int sl = pslot(L - R + warp - 12);
#pragma unroll
            for (int m = 0; m < 13; ++m) {
                offs[m] = sl * WW;
                sl = sl + 1 == ts::DP ? 0 : sl + 1;
            }
        }
        // ---- the five sub-steps, unrolled so that every row bound, shadow row
        // and ring offset that depends on s is a constant (2048^2: 301 -> 292
        // us; unrolling the LBM site loop as well made the code too large)
#pragma unroll
        for (int s = 1; s <= ts::NSUB; ++s) {
            const int E = L - 2 * s;                       // block rows [E - R, E)
            const int lo = -(12 - 2 * s), hi = SG + 12 - 2 * s;     // exact rows of phi^(s)
            const int qlo = -(7 - s), qhi = SG + 7 - s;             // exact rows of Q^(s)
            // the stage touches rows [E - R - 2, E + 2) of phi / Q and [E - R - 1,
            // E + 1) of u; the two rows below the block are this stage's shadows
            const int tb = E - R - 2, ub = uslot(tb + 1);
            const int shr = ts::SH0 + 2 * (s - 1);
            auto urow = [&](int t) { return TF_BC(step_slot<ts::DU>(ub, t - tb - 1), ts::DU) * WW; };
            // row offset (shadow row or ring slot, times the row length) of row
            // t = y - 2 + j of phi^(s-1), Q^(s-1); j = 0 .. 4 is a constant
            // once the sub-steps are unrolled
            auto rof = [&](int t) {
                const int j = t - tb - warp;
                const int k = warp + j;
                return TF_BC(k < 2 ? (shr + k) * WW : offs[10 - 2 * s + j], ts::FROWS * WW);
            };
            auto phi_row = [&](int t) -> const float* { return sm + ts::OFF_PHI + rof(t); };
            auto qa_row = [&](int t) -> const float* { return sm + ts::OFF_QA + rof(t); };
            auto qb_row = [&](int t) -> const float* { return sm + ts::OFF_QB + rof(t); };
            // (a) phi^(s), Q^(s) of this warp's row into registers, with mu^(s)
            // of rows y-1, y, y+1 evaluated here from phi^(s-1) rows y-2 .. y+2
            const int y = E - R + warp;
            const bool vp = y >= lo && y < hi, vq = y >= qlo && y < qhi;
            V4 nph, nqa, nqb, oph, oqa, oqb;   // new and old (phi, Q) of row y
            if (vp) {
                const float* u1x = sm + ts::OFF_U + 0 * ts::DU * WW + col;
                const float* u1y = sm + ts::OFF_U + 1 * ts::DU * WW + col;
                const float* u2x = sm + ts::OFF_U + 2 * ts::DU * WW + col;
                const float* u2y = sm + ts::OFF_U + 3 * ts::DU * WW + col;
                const int us = urow(y - 1), uc = urow(y), un = urow(y + 1);
                const V4 phss = ld4(phi_row(y - 2) + col), phs = ld4(phi_row(y - 1) + col),
                         phc = ld4(phi_row(y) + col), phn = ld4(phi_row(y + 1) + col),
                         phnn = ld4(phi_row(y + 2) + col);
                oph = phc;
                // mu = -kappa lap(phi) + A_ch f'(phi) (Eq. 2) of the middle row
                auto mu_row = [&](const V4& pp, const V4& pc, const V4& pn) {
                    V4 mu;
                    const V4 h = hsum4(pc);
                    {
                        const f2 lap = F2(m4, pc.lo, A2(h.lo, A2(pp.lo, pn.lo)));
                        const f2 poly = F2(pc.lo, F2(pc.lo, F2(pc.lo, mu3, mu2), mu1), mu0);
                        mu.lo = F2(kap, lap, poly);
                    }
                    {
                        const f2 lap = F2(m4, pc.hi, A2(h.hi, A2(pp.hi, pn.hi)));
                        const f2 poly = F2(pc.hi, F2(pc.hi, F2(pc.hi, mu3, mu2), mu1), mu0);
                        mu.hi = F2(kap, lap, poly);
                    }
                    return mu;
                };
                const V4 mus = mu_row(phss, phs, phc), muc = mu_row(phs, phc, phn),
                         mun = mu_row(phc, phn, phnn);
                const V4 axc = ld4(u1x + uc), ays = ld4(u1y + us), ayn = ld4(u1y + un);
                const V4 bxc = ld4(u2x + uc), bys = ld4(u2y + us), byn = ld4(u2y + un);
                // fluxes J_x at row y, J_y at rows y -/+ 1
                V4 jx, jys, jyn;
                jx.lo = flux(A2(cref, phc.lo), axc.lo, bxc.lo);
                jx.hi = flux(A2(cref, phc.hi), axc.hi, bxc.hi);
                jys.lo = flux(A2(cref, phs.lo), ays.lo, bys.lo);
                jys.hi = flux(A2(cref, phs.hi), ays.hi, bys.hi);
                jyn.lo = flux(A2(cref, phn.lo), ayn.lo, byn.lo);
                jyn.hi = flux(A2(cref, phn.hi), ayn.hi, byn.hi);
                const V4 djx = hdiff4(jx), hm = hsum4(muc);
                {
                    const f2 dJ = A2(djx.lo, B2(jyn.lo, jys.lo));
                    const f2 lapmu = F2(m4, muc.lo, A2(hm.lo, A2(mun.lo, mus.lo)));
                    nph.lo = F2(hdt2, F2(M2x, lapmu, N2(dJ)), phc.lo);
                }
                {
                    const f2 dJ = A2(djx.hi, B2(jyn.hi, jys.hi));
                    const f2 lapmu = F2(m4, muc.hi, A2(hm.hi, A2(mun.hi, mus.hi)));
                    nph.hi = F2(hdt2, F2(M2x, lapmu, N2(dJ)), phc.hi);
                }
                // Q^(s) of the row, also where only phi^(s) is exact (vp && !vq:
                // computed from in-range rows, not stored): one basic block with
                // the phi update, so the two chains interleave (2048^2: 326 -> 318 us)
                {
                    const V4 as = ld4(qa_row(y - 1) + col), ac = ld4(qa_row(y) + col),
                             an = ld4(qa_row(y + 1) + col);
                    const V4 bs = ld4(qb_row(y - 1) + col), bc = ld4(qb_row(y) + col),
                             bn = ld4(qb_row(y + 1) + col);
                    oqa = ac;
                    oqb = bc;
                    const V4 axs = ld4(u1x + us), axn = ld4(u1x + un), ayc = ld4(u1y + uc);
                    V4 ah, ax, bh, bx;
                    hsd4(ac, ah, ax);
                    hsd4(bc, bh, bx);
                    const V4 dux = hdiff4(axc), duy = hdiff4(ayc);
                    auto qpair = [&](f2 a, f2 bq, f2 ah_, f2 ax_, f2 an_, f2 as_, f2 bh_, f2 bx_, f2 bn_,
                                     f2 bs_, f2 dux_, f2 duy_, f2 axn_, f2 axs_,
                                     f2 ayn_, f2 ays_, f2 axc_, f2 ayc_, f2& oa, f2& ob) {
                        const f2 lapa = F2(m4, a, A2(ah_, A2(an_, as_)));
                        const f2 lapb = F2(m4, bq, A2(bh_, A2(bn_, bs_)));
                        const f2 cg = F2(cGC, F2(a, a, M2(bq, bq)), cGA);
                        const f2 Dxx = dux_, Dyy = B2(ayn_, ays_);
                        const f2 Dxy = B2(axn_, axs_), Dyx = duy_;
                        const f2 E1 = B2(Dxx, Dyy), EX = A2(Dxy, Dyx);
                        const f2 t1 = F2(half, A2(Dxx, Dyy), N2(F2(a, E1, M2(bq, EX))));
                        const f2 cc = F2(lamd, t1, cg);
                        const f2 hO = M2(hdt2, B2(Dxy, Dyx));
                        const f2 nux = M2(nhdt, axc_), nuy = M2(nhdt, ayc_);
                        oa = A2(a, F2(cc, a, F2(cGK, lapa, F2(lamq, E1, F2(hO, bq,
                                F2(nux, ax_, M2(nuy, B2(an_, as_))))))));
                        ob = A2(bq, F2(cc, bq, F2(cGK, lapb, F2(lamq, EX, F2(N2(hO), a,
                                F2(nux, bx_, M2(nuy, B2(bn_, bs_))))))));
                    };
                    qpair(ac.lo, bc.lo, ah.lo, ax.lo, an.lo, as.lo, bh.lo, bx.lo, bn.lo, bs.lo,
                          dux.lo, duy.lo, axn.lo, axs.lo, ayn.lo, ays.lo, axc.lo,
                          ayc.lo, nqa.lo, nqb.lo);
                    qpair(ac.hi, bc.hi, ah.hi, ax.hi, an.hi, as.hi, bh.hi, bx.hi, bn.hi, bs.hi,
                          dux.hi, duy.hi, axn.hi, axs.hi, ayn.hi, ays.hi, axc.hi,
                          ayc.hi, nqa.hi, nqb.hi);
                }
            }
            __syncthreads();
            // the last sub-step has read this block's u rows: the next block's
            // u rows go into their slots
            if (s == ts::NSUB && j + 1 < nblk) issue_u(j + 1);
            // (b) save the rows the next block reads below its own (phi^(s-1)
            // of rows E - 2, E - 1 and Q^(s-1) of row E - 1), then write in place
            if (own) {
                const int py = TF_BC(offs[12 - 2 * s], ts::DP * WW) + col;   // row y
                if (warp >= R - 2 && y >= lo - 2) {
                    const int sh = TF_BC(shr + warp - (R - 2), ts::FROWS) * WW + col;
                    if (!vp) {   // row not computed: its old values are not in registers
                        oph = ld4(sm + ts::OFF_PHI + py);
                        oqa = ld4(sm + ts::OFF_QA + py);
                        oqb = ld4(sm + ts::OFF_QB + py);
                    }
                    st4(sm + ts::OFF_PHI + sh, oph);
                    if (warp == R - 1) {   // Q is read one row outside a block, phi two
                        st4(sm + ts::OFF_QA + sh, oqa);
                        st4(sm + ts::OFF_QB + sh, oqb);
                    }
                }
                if (vp) st4(sm + ts::OFF_PHI + py, nph);
                if (vq) {
                    st4(sm + ts::OFF_QA + py, nqa);
                    st4(sm + ts::OFF_QB + py, nqb);
                }
            }
            __syncthreads();
        }

        // ---- mu and the fluid-1 stress of phi^(5), Q^(5) on rows [L - 11 - R, L - 11)
        {
            const int y = L - 11 - R + warp;
            if (y >= -1 && y < SG + 1) {
                const int sb = TF_BC(pslot(y - 1), ts::DP);
                const float* ps = sm + ts::OFF_PHI + sb * WW + col;
                const float* pc = sm + ts::OFF_PHI + step_slot<ts::DP>(sb, 1) * WW + col;
                const float* pn = sm + ts::OFF_PHI + step_slot<ts::DP>(sb, 2) * WW + col;
                const int dqa = ts::OFF_QA - ts::OFF_PHI, dqb = ts::OFF_QB - ts::OFF_PHI;
                const V4 dp = ld4(ps), dc = ld4(pc), dn = ld4(pn);
                const V4 ap = ld4(ps + dqa), ac = ld4(pc + dqa), an = ld4(pn + dqa);
                const V4 bp = ld4(ps + dqb), bc = ld4(pc + dqb), bn = ld4(pn + dqb);
                const V4 dh = hsum4(dc);
                V4 ah, ax, bh, bx;
                hsd4(ac, ah, ax);
                hsd4(bc, bh, bx);
                const PairStress r0 = stress2(P, dc.lo, dh.lo, dn.lo, dp.lo, ac.lo, ah.lo, ax.lo,
                                               an.lo, ap.lo, bc.lo, bh.lo, bx.lo, bn.lo, bp.lo);
                const PairStress r1 = stress2(P, dc.hi, dh.hi, dn.hi, dp.hi, ac.hi, ah.hi, ax.hi,
                                               an.hi, ap.hi, bc.hi, bh.hi, bx.hi, bn.hi, bp.hi);
                // the row's final phi, Q (strip columns): 16-byte stores
                if (y >= 0 && y < SG && col >= ts::HALO && col < ts::HALO + tw) {
                    const int g = TF_BC((y0 + y) * nx + x0 + col - ts::HALO, (int)N - 3);
                    st4(a.phi_out + b * N + g, dc);
                    st4(a.Q_out + 2 * b * N + g, ac);
                    st4(a.Q_out + (2 * b + 1) * N + g, bc);
                }
                if (lane >= ts::SC0 / 4 && lane < (ts::SC0 + ts::SW) / 4) {
                    float* st = sm + ts::OFF_ST + TF_BC(sslot(y), ts::DS) * ts::SW +
                                TF_BC(col - ts::SC0, ts::SW - 3);
                    constexpr int PL = ts::DS * ts::SW;
                    st4(st, {r0.mu, r1.mu});
                    st4(st + PL, {r0.sxx, r1.sxx});
                    st4(st + 2 * PL, {r0.sxy, r1.sxy});
                    st4(st + 3 * PL, {r0.syx, r1.syx});
                    st4(st + 4 * PL, {r0.syy, r1.syy});
                }
            }
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tfp::smem_addr(&stress_bar[warp]))
                         : "memory");
        }
        // ---- LBM of rows [L - 12 - R, L - 12) and stores of the new state
        {
            const int eL = L - 12;
            const int r0 = max(eL - R, 0) - (eL - R), r1 = min(eL, SG) - (eL - R);   // block rows
            // 32-bit pair indices within one instance's nine direction planes
            // (9 N < 2^31, checked by the host); the instance offset is in the
            // 64-bit bases
            const int Ni = (int)N;
            using T2 = typename S::T2;
            const T2* __restrict__ F1 = reinterpret_cast<const T2*>(a.fsrc + pop_index(b, 0, 0, 0, N));
            T2* __restrict__ D1 = reinterpret_cast<T2*>(a.fdst + pop_index(b, 0, 0, 0, N));
            float* __restrict__ uo = a.u_out + 4 * b * N;
            const float* stb = sm + ts::OFF_ST - ts::SC0;   // stress ring, window columns
            constexpr int PL = ts::DS * ts::SW;
            // One block row per warp (its ring slots, row wraps and row bases are
            // warp-uniform), columns lane, lane + 32, lane + 64 of the strip, the
            // next site's pulls in flight while this site is computed (the first
            // site's before the wait for the stress rows).  2048^2: 268.9 -> 266.5 us against
            // the block's sites dealt out to all threads in row-major order.
            const int tb = eL - R + r0 - 1;                // the row below the block's first
            const int pb = pslot(tb), sb = sslot(tb);
            const bool wrow = warp >= r0 && warp < r1;     // this warp's block row is in the segment
            const int t = eL - R + warp;                   // its segment row
            const int k = t - tb;                          // 1 .. R when wrow
            const float* ph = sm + ts::OFF_PHI + step_slot<ts::DP>(pb, k) * WW;
            const float* phs = sm + ts::OFF_PHI + step_slot<ts::DP>(pb, k - 1) * WW;
            const float* phn = sm + ts::OFF_PHI + step_slot<ts::DP>(pb, k + 1) * WW;
            const float* sc = stb + step_slot<ts::DS>(sb, k) * ts::SW;
            const float* ss = stb + step_slot<ts::DS>(sb, k - 1) * ts::SW;
            const float* sn = stb + step_slot<ts::DS>(sb, k + 1) * ts::SW;
            const int gy = y0 + t;
            const int ry = gy * nx;
            const int ryp = (gy + 1 < ny ? gy + 1 : 0) * nx, rym = (gy > 0 ? gy - 1 : ny - 1) * nx;
            // pulled populations of strip column cx of the warp's row: f_i(x - c_i)
            auto pull = [&](f2 (&f)[9], int cx) {
                const int x = x0 + cx;
                const int xp = x + 1 < nx ? x + 1 : 0, xm = x > 0 ? x - 1 : nx - 1;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int sx = d2q9_cx(i) == 0 ? x : (d2q9_cx(i) > 0 ? xm : xp);
                    const int sy = d2q9_cy(i) == 0 ? ry : (d2q9_cy(i) > 0 ? rym : ryp);
                    const int idx = TF_BC(i * Ni + sy + sx, 9 * Ni);
                    f[i] = S::load2(F1 + idx);
                }
            };
            f2 f[9], fn[9];
            if (wrow && lane < tw) pull(f, lane);
            {
                // stress rows t - 1 .. t + 1 of this warp's LBM row: those of
                // warps warp - 2 .. warp; every wait is bounded
                bool ok = true;
                for (int k = max(warp - 2, 0); k <= warp; ++k)
                    ok = tfp::wait_bounded(&stress_bar[k], (uint32_t)(j & 1), kWaitPolls) && ok;
                if (!ok) atomicExch(a.err, TF_ERR_TIMEOUT);
            }
            if (wrow) {
#pragma unroll 1
                for (int cx = lane; cx < tw; cx += 32) {
                    if (cx + 32 < tw) pull(fn, cx + 32);
                    const int c = TF_BC(ts::HALO + cx, ts::SC0 + ts::SW - 1);   // window column
                    f2 u1, u2;
                    lbm_site2(P, ph[c], P2(ph[c - 1], ph[c + 1]), P2(phs[c], phn[c]), sc[c],
                              P2(sc[c - 1], sc[c + 1]), P2(ss[c], sn[c]),
                              P2(sc[PL + c - 1], sc[PL + c + 1]), P2(ss[2 * PL + c], sn[2 * PL + c]),
                              P2(sc[3 * PL + c - 1], sc[3 * PL + c + 1]),
                              P2(ss[4 * PL + c], sn[4 * PL + c]), f, u1, u2);
                    const int g = TF_BC(ry + x0 + cx, Ni);
#pragma unroll
                    for (int i = 0; i < 9; ++i) S::store2_stream(D1 + (i * Ni + g), f[i]);
                    uo[g] = u1.x;
                    uo[N + g] = u1.y;
                    uo[2 * N + g] = u2.x;
                    uo[3 * N + g] = u2.y;
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = fn[i];
                }
            }
        }
        // No barrier at the end of a block: the next block writes shared
        // memory first through its copies, issued after its first barrier.
    }
    TF_BC_END(a.err);
}

template <class S>
cudaError_t configure_strip() {
    return cudaFuncSetAttribute(k_strip<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ts::SMEM);
}

template <class S>
void launch_strip(const TileArgs<S>& a, dim3 grid, cudaStream_t stream) {
    k_strip<S><<<grid, NT, ts::SMEM, stream>>>(a);
}

}  // namespace
