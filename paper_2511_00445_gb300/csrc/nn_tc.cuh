// Tensor-core GEMM core for the surrogate network (sm_103a, tcgen05).
//
// D[m][n] = sum_k A[m][k] B[n][k] with BF16 operands and FP32 accumulation in
// tensor memory.  One CTA (4 warps) owns a 128 x BN tile of D and walks K in
// chunks of 64: every thread gathers 16-byte pieces (8 consecutive k) of A
// and B through the operation's loaders and stores them in shared memory in
// the canonical no-swizzle K-major layout (8-row x 16-byte core matrices);
// one thread issues four tcgen05.mma (K = 16 each) per chunk and commits them
// to the stage's mbarrier.  Two stages: the gather of chunk j+1 overlaps the
// MMAs of chunk j.  Epilogue: each thread owns one row of the tile, reads its
// accumulators 16 columns at a time (tcgen05.ld) and hands them to the
// operation.  Every mbarrier wait is bounded; a wait that runs out writes
// TF_ERR_TIMEOUT to the status word and the CTA finishes without trapping.
//
// An operation Op provides
//   int M, N, K;                                   GEMM sizes (K a multiple of 8)
//   uint4 a_chunk(int m, int k8) const;            A[m][8 k8 .. 8 k8 + 7] (zero outside)
//   uint4 b_chunk(int n, int k8) const;            B[n][8 k8 .. 8 k8 + 7] (zero outside)
//   void epilogue(int m, int n0, const float (&v)[16]) const;  D[m][n0 .. n0 + 15]
//   int* err;                                      device status word
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tf_ptx.cuh"
#include "twofluid.h"

namespace tcg {

constexpr int BM = 128, BK = 64, NTHREADS = 128;
constexpr uint32_t kPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of an R-row K-major tile (BK columns) in the
// canonical no-swizzle layout: core matrix (r/8, k/8) holds 8 rows of 16 bytes.
// Core matrices adjacent in K are R*16 bytes apart (leading byte offset), row
// groups 128 bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t tile_off(int r, int k, int R) {
    return (uint32_t)(((k >> 3) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// One tcgen05.mma (kind::f16, cta_group::1) accumulating into tensor memory
// when acc is nonzero, overwriting it otherwise.
__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Round two floats to BF16 (nearest even) and pack them, the first in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int BN>
constexpr int smem_bytes() {
    return 2 * (BM * BK * 2 + BN * BK * 2);
}

// grid: (ceil(M / 128), ceil(N / BN), splits); split z covers K chunks
// [z * chunks_per_split, (z + 1) * chunks_per_split).
template <int BN, class Op>
__global__ void __launch_bounds__(NTHREADS) k_gemm(const Op op, int chunks_per_split) {
    static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128, "tile width");
    constexpr int TCOLS = BN < 32 ? 32 : BN;                  // tensor-memory columns
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nchunks_all = (op.K + BK - 1) / BK;
    const int c_begin = blockIdx.z * chunks_per_split;
    const int c_end = min(nchunks_all, c_begin + chunks_per_split);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    uint32_t phase[2] = {0, 0};
    bool ok = true;
    int used = 0;
    for (int c = c_begin; c < c_end; ++c, ++used) {
        const int s = used & 1;
        unsigned char* As = tc_smem + s * (A_BYTES + B_BYTES);
        unsigned char* Bs = As + A_BYTES;
        if (used >= 2) {   // the MMAs of chunk used-2 read this stage
            ok = ok && mbar_wait(&bars[s], phase[s]);
            phase[s] ^= 1;
        }
        const int k8_0 = c * (BK / 8);
        for (int q = tid; q < BM * (BK / 8); q += NTHREADS) {
            const int r = q >> 3, kc = q & 7;
            *reinterpret_cast<uint4*>(As + tile_off(r, kc * 8, BM)) = op.a_chunk(m0 + r, k8_0 + kc);
        }
        for (int q = tid; q < BN * (BK / 8); q += NTHREADS) {
            const int r = q >> 3, kc = q & 7;
            *reinterpret_cast<uint4*>(Bs + tile_off(r, kc * 8, BN)) = op.b_chunk(n0 + r, k8_0 + kc);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                const uint64_t ad = smem_desc(smem_u32(As) + k * 2 * (BM / 8) * 128, BM * 16, 128);
                const uint64_t bd = smem_desc(smem_u32(Bs) + k * 2 * (BN / 8) * 128, BN * 16, 128);
                const uint32_t acc = (used > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tbase),
                    "l"(ad), "l"(bd), "r"(instr_desc(BM, BN)), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bars[s])));
        }
    }
    // The last commit covers every MMA issued before it.
    if (used > 0) {
        const int s = (used - 1) & 1;
        ok = ok && mbar_wait(&bars[s], phase[s]);
    }
    // tcgen05.ld below is warp-collective: decide for the whole CTA
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0) atomicExch(op.err, TF_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (used > 0 && ok) {
        const int m = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            if (m < op.M && n0 + c0 < op.N) op.epilogue(m, n0 + c0, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(TCOLS));
}

// ---------------------------------------------------------------------------
// Row-segment 3x3 convolution on the tensor cores.
//
// One CTA computes output pixels (b, y, x0 .. x0 + T - 1), T = min(W - x0, 128),
// for output channels n0 .. n0 + BN - 1.  For each chunk of up to 64 source
// channels it stages the three source rows y - 1, y, y + 1 (columns x0 - 1 ..
// x0 + T, periodic) in shared memory as 16-byte pixel rows (8 channels each,
// one block per 8-channel group), and the weights of all nine taps for those
// channels.  In that layout the A operand of tap (dy, dx) is the same tile
// read from a start address shifted by whole pixel rows, so the nine taps
// need no further loads: 9 x (channels / 16) MMAs per chunk.  Rows of A past
// the T valid pixels read staged data of other rows; their results are
// discarded by the epilogue.
//   GRAD = false: out[p][n] = relu?(bias[n] + sum_{tap, c} w[n][tap][c] src[p + d(tap)][c])
//   GRAD = true : dx[p][n] += sum_{tap, c} w[n][tap][c] src[p - d(tap)][c]
// (the input gradient with w the transposed weights wt[cin][tap][cout]).
// Short rows (one segment, T = W < 128) pack several output rows into the
// MMA tile in the forward direction: R + 2 source rows are staged with pitch
// Tp = T + 2, output row r takes tile rows r Tp .. r Tp + T - 1 (its two halo
// positions are discarded), and every tap is still one start-address shift.
// NACC tensor-memory accumulators extend the tile to NACC x 128 rows (the
// second accumulator's A operand starts 128 staged rows further), so
// up to (NACC * 128 - T) / Tp + 1 output rows per CTA (the launcher may pick
// fewer to keep the grid wide).
// ---------------------------------------------------------------------------
struct ConvRowArgs {
    const __nv_bfloat16* src;   // NHWC, Cs channels
    const __nv_bfloat16* w;     // pre-tiled weights, see row_wtile_index
    const float* bias;          // forward only
    __nv_bfloat16* out;         // forward: NHWC BF16, Nout channels
    float* dx;                  // gradient: NHWC FP32, Nout channels (accumulated)
    int B, H, W, Cs, Nout, relu;
    int* err;
    int rows;                   // output rows per CTA, 1 .. row_group(W, NACC, GRAD) (set by the launcher)
    // Forward only: with src2 set, the source is the concatenation of src
    // upsampled 2x by repetition (H/2 x W/2, C1 channels) and src2 (H x W,
    // Cs - C1 channels), read in place instead of from a materialised copy.
    const __nv_bfloat16* src2 = nullptr;
    int C1 = 0;
    int bn = 32;                // forward weight layout: 32 (x 64 source channels) or 64 (x 32)
};

// Address of the 16-byte piece of channels c .. c + 7 (c < Cs, a multiple
// of 8) of source pixel (b, yy, xx), for a plain or a concatenated source.
__device__ __forceinline__ const __nv_bfloat16* src_piece(const __nv_bfloat16* src,
                                                          const __nv_bfloat16* src2, int C1, int H,
                                                          int W, int Cs, int b, int yy, int xx, int c) {
    if (src2 == nullptr) return src + ((size_t)(b * H + yy) * W + xx) * Cs + c;
    if (c < C1) return src + ((size_t)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C1 + c;
    return src2 + ((size_t)(b * H + yy) * W + xx) * (Cs - C1) + (c - C1);
}

constexpr int ROW_T = 128;      // output pixels per CTA
constexpr int ROW_CC = 64;      // source channels per chunk
constexpr int ROW_NT = 256;     // threads: all stage operands; warps w and w + 4 share
                                // tensor-memory lanes 32 (w % 4) .. in the epilogue

__host__ __device__ constexpr int row_halo_rows(int T) {
    return 3 * (T + 2) > 2 * (T + 2) + 2 + ROW_T ? 3 * (T + 2) : 2 * (T + 2) + 2 + ROW_T;
}

// Bytes of one pre-tiled weight block: BN output channels x CC source
// channels x 9 taps (BF16); the same 36 KB for 32 x 64 and 64 x 32.
template <int BN, int CC>
constexpr int wtile_bytes_of() {
    return 9 * (CC / 16) * BN * 32;
}

template <int BN, int CC = 64>
constexpr int row_smem_bytes() {
    return (CC / 8) * row_halo_rows(ROW_T) * 16 + wtile_bytes_of<BN, CC>();
}

// Weights pre-tiled in the shared-memory image k_conv_rows stages: for output
// tile t (channels 32 t ..) and source chunk ch (channels 64 ch ..), one block
// of 36 slices (tap, 16-channel step) of 32 x 16 K-major core matrices,
// ROW_WTILE bytes, blocks ordered (t, ch).  Byte offset of weight (n, tap, c)
// for a layer with Cs source channels:
constexpr int ROW_BN = 32;
constexpr int ROW_WTILE = 36 * ROW_BN * 32;
// General layout for a tile of BNt output channels and chunks of CCt source
// channels (blocks of 9 * CCt / 16 slices of BNt x 16 K-major core matrices).
template <int BNt, int CCt>
__host__ __device__ inline long long wtile_index(int n, int tap, int c, int Cs) {
    const int nch = (Cs + CCt - 1) / CCt;
    const int t = n / BNt, nn = n % BNt, ch = c / CCt, cc = c % CCt;
    const int slice = tap * (CCt / 16) + cc / 16, k = cc % 16;
    const long long off_in = (long long)slice * BNt * 32 +
                             (((k >> 3) * (BNt >> 3) + (nn >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2);
    return ((long long)t * nch + ch) * wtile_bytes_of<BNt, CCt>() + off_in;
}
__host__ __device__ inline long long row_wtile_index(int n, int tap, int c, int Cs) {
    return wtile_index<ROW_BN, ROW_CC>(n, tap, c, Cs);
}

// Most output rows one CTA can pack (the launcher's upper bound for rows).
__host__ __device__ inline int row_group(int W, int nacc, bool grad) {
    return grad || W > ROW_T ? 1 : (nacc * 128 - W) / (W + 2) + 1;
}

// BN x CC: output-tile width and source chunk of the weight layout
// (32 x 64, or 64 x 32 for forward layers with at least 64 outputs).
template <int BN, int CC, bool GRAD, int NACC = 1>
__global__ void __launch_bounds__(ROW_NT) k_conv_rows(const ConvRowArgs a) {
    static_assert((BN == 32 && CC == 64) || (BN == 64 && CC == 32 && !GRAD), "weight layouts");
    static_assert(NACC == 1 || (NACC == 2 && !GRAD), "two accumulators in the forward direction only");
    constexpr int TCOLS = NACC * BN;
    constexpr int WTILE = wtile_bytes_of<BN, CC>();
    constexpr int HR = row_halo_rows(ROW_T);          // staged rows per 8-channel block
    constexpr int A_BYTES = (CC / 8) * HR * 16;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar, wbar;
    __shared__ uint32_t tmem_base;
    unsigned char* As = tc_smem;
    unsigned char* Bs = tc_smem + A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int segs = (a.W + ROW_T - 1) / ROW_T;
    const int R = a.rows, groups = (a.H + R - 1) / R;
    const int seg = blockIdx.x % segs, y = ((blockIdx.x / segs) % groups) * R, b = blockIdx.x / (segs * groups);
    const int rows_here = min(R, a.H - y);
    const int x0 = seg * ROW_T, T = min(ROW_T, a.W - x0), Tp = T + 2;
    const int n0 = blockIdx.y * BN;
    const int sgn = GRAD ? -1 : 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    uint32_t phase = 0;
    bool ok = true;
    const int nchunks = (a.Cs + CC - 1) / CC;
    const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(a.w) +
                                (long long)blockIdx.y * nchunks * WTILE;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int c_base = ch * CC;
        const int csteps = min(CC, (a.Cs - c_base + 15) & ~15) / 16;       // K = 16 steps
        const int cgroups = 2 * csteps;                                    // 8-channel groups
        // the chunk's weights: one bulk copy of the pre-tiled block (lands while
        // the threads stage the source rows)
        if (tid == 0) {
            tfp::mbar_arrive_expect_tx(&wbar, (uint32_t)WTILE);
            tfp::bulk_g2s(Bs, wsrc + (long long)ch * WTILE, (uint32_t)WTILE, &wbar);
        }
        // stage the source rows: pixel q of row r (q = 0 .. Tp-1) at block g, row
        // r*Tp + q, by asynchronous 16-byte copies (zero-filled past Cs)
        const int na = (R + 2) * Tp * cgroups;
        for (int i = tid; i < na; i += ROW_NT) {
            const int g = i % cgroups, q = (i / cgroups) % Tp, r = i / (cgroups * Tp);
            const int c = c_base + 8 * g;
            int yy = y + sgn * (r - 1), xx = x0 - 1 + q;
            yy = yy < 0 ? yy + a.H : (yy >= a.H ? yy - a.H : yy);
            xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
            const bool in = c < a.Cs;
            const __nv_bfloat16* src =
                src_piece(a.src, a.src2, a.C1, a.H, a.W, a.Cs, b, yy, xx, in ? c : 0);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             smem_u32(As + (g * HR + r * Tp + q) * 16)),
                         "l"(src), "r"(in ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        ok = ok && tfp::wait_bounded(&wbar, phase & 1u, kPolls);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // Descriptors are linear in their address field (address >> 4, below
            // 2^14 here): offsets in 16-byte units are added to base descriptors.
            const uint64_t ad0 = smem_desc(smem_u32(As), HR * 16, 128);
            const uint64_t bd0 = smem_desc(smem_u32(Bs), BN * 16, 128);
            const uint32_t idesc = instr_desc(BM, BN);
            uint32_t acc = ch > 0 ? 1u : 0u;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                // source pixel of output pixel r for this tap: staged row (1 + dy), column r + 1 + dx
                // (the staging already applied the sign of the row offset)
                const int dx = sgn * (tap % 3 - 1);
                uint64_t ad = ad0 + (uint64_t)((tap / 3) * Tp + 1 + dx);
                uint64_t bd = bd0 + (uint64_t)((tap * (CC / 16) * BN * 32) >> 4);
                for (int s = 0; s < csteps; ++s) {
#pragma unroll
                    for (int q = 0; q < NACC; ++q)   // accumulator q: tile rows 128 q ..
                        mma_f16(tbase + (uint32_t)(q * BN), ad + (uint64_t)(q * 128), bd, idesc, acc);
                    acc = 1;
                    ad += 2 * HR;              // next 16-channel step: two group blocks
                    bd += (BN * 32) >> 4;      // next weight slice
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bar)));
        }
        ok = ok && mbar_wait(&bar, phase);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();   // the next chunk overwrites the staged tiles
    }
    ok = __syncthreads_and(ok) != 0;   // the loads below are warp-collective
    if (!ok && tid == 0) atomicExch(a.err, TF_ERR_TIMEOUT);
#pragma unroll 1
    for (int q = 0; q < NACC && ok; ++q) {
        // tensor-memory lane of accumulator q = tile row m = 128 q + lane_row:
        // output row m / Tp of the group, pixel m % Tp (valid below T)
        const int lane_row = (warp & 3) * 32 + (tid & 31);
        const int m = q * 128 + lane_row, rr = m / Tp, xq = m - rr * Tp;
        const bool valid = xq < T && rr < rows_here;
        const size_t p = (size_t)(b * a.H + y + rr) * a.W + x0 + xq;
        const int half = warp >> 2;                          // columns [half * BN/2, (half+1) * BN/2)
#pragma unroll 1
        for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2) && n0 + c0 < a.Nout; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(q * BN + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (!valid) continue;   // halo positions and rows past the group are discarded
            const int n = n0 + c0;
            if (GRAD) {
                float* d = a.dx + p * a.Nout + n;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n + j < a.Nout) d[j] += __uint_as_float(r[j]);
            } else {
                float z[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    z[j] = __uint_as_float(r[j]) + (n + j < a.Nout ? a.bias[n + j] : 0.f);
                    if (a.relu) z[j] = fmaxf(z[j], 0.f);
                }
                __nv_bfloat16* d = a.out + p * a.Nout + n;
                if (n + 16 <= a.Nout) {
                    reinterpret_cast<uint4*>(d)[0] = make_uint4(pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]),
                                                                pack_bf16(z[4], z[5]), pack_bf16(z[6], z[7]));
                    reinterpret_cast<uint4*>(d)[1] = make_uint4(pack_bf16(z[8], z[9]), pack_bf16(z[10], z[11]),
                                                                pack_bf16(z[12], z[13]), pack_bf16(z[14], z[15]));
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n + j < a.Nout) d[j] = __float2bfloat16_rn(z[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(TCOLS));
}

// ---------------------------------------------------------------------------
// Row-walking 3x3 convolution (forward) for rows of a multiple of 128 pixels.
//
// One CTA owns the 128-pixel segment x0 .. x0 + 127 of image b, output
// channels n0 .. n0 + BN - 1, and a run of consecutive output rows
// [ya, yb).  It loads the weights of all its source-channel chunks once (one
// bulk copy of the pre-tiled blocks) and keeps a ring of S (4 .. 8) source
// rows in shared memory, all source channels, in the staging layout of
// k_conv_rows (16-byte pixel rows, one 130-row block per 8-channel group).
// Output row i reads source rows i - 1, i, i + 1; at that point source rows
// up to i + S - 2 are already on their way (the copies run S - 3 rows ahead of
// their use), and the epilogue of row i - 1 drains the other of two
// tensor-memory accumulators while the MMAs of row i run.  Per output row the MMAs are issued in
// k_conv_rows' order (chunk, tap, 16-channel step), so both kernels
// accumulate the same products in the same sequence.
// ---------------------------------------------------------------------------
struct ConvWalkArgs {
    const __nv_bfloat16* src;   // NHWC, Cs channels
    const __nv_bfloat16* w;     // pre-tiled weights, see row_wtile_index
    const float* bias;
    __nv_bfloat16* out;         // NHWC BF16, Nout channels
    int B, H, W, Cs, Nout, relu;
    int rb;                     // row blocks per (image, segment, output tile)
    int slots;                  // ring depth S, 4 .. WALK_MAX_SLOTS
    int* err;
    const __nv_bfloat16* src2;  // concatenated source, as in ConvRowArgs (or null)
    int C1;
};

constexpr int WALK_MAX_SLOTS = 8;
constexpr int WALK_ROWS = ROW_T + 2;    // staged pixel rows per 8-channel group

// 8-channel groups staged per source row (source channels padded to K = 16 steps)
__host__ __device__ constexpr int walk_groups(int Cs) { return 2 * ((Cs + 15) / 16); }

template <int BN = ROW_BN, int CC = ROW_CC>
__host__ __device__ constexpr int walk_smem_bytes(int Cs, int slots) {
    return ((Cs + CC - 1) / CC) * wtile_bytes_of<BN, CC>() + slots * walk_groups(Cs) * WALK_ROWS * 16;
}

// cp.async.wait_group takes an immediate: wait until at most n (1 .. 5) of
// this thread's most recent copy groups are still pending.
__device__ __forceinline__ void cp_async_wait_upto(int n) {
    switch (n) {
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    }
}

// BN x CC: weight layout as in k_conv_rows (32 x 64, or 64 x 32).
template <int BN, int CC>
__global__ void __launch_bounds__(ROW_NT) k_conv_walk(const ConvWalkArgs a) {
    static_assert((BN == 32 && CC == 64) || (BN == 64 && CC == 32), "weight layouts");
    constexpr int WTILE = wtile_bytes_of<BN, CC>();
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t wbar, mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(16) float sbias[BN];   // this tile's bias (0 past Nout)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nch = (a.Cs + CC - 1) / CC, cg = walk_groups(a.Cs), csteps = cg / 2;
    const uint32_t slot_bytes = (uint32_t)cg * WALK_ROWS * 16;
    const int S = a.slots;
    const int g_first = tid % cg, q_first = tid / cg, g_step = ROW_NT % cg, q_step = ROW_NT / cg;
    unsigned char* Bs = tc_smem;
    unsigned char* Rs = tc_smem + nch * WTILE;
    const int segs = a.W / ROW_T;
    int u = blockIdx.x;
    const int blk = u % a.rb;
    u /= a.rb;
    const int seg = u % segs, b = u / segs;
    const int ya = (int)((long long)blk * a.H / a.rb), yb = (int)((long long)(blk + 1) * a.H / a.rb);
    const int rows = yb - ya, x0 = seg * ROW_T, n0 = blockIdx.y * BN;
    if (tid < BN) sbias[tid] = n0 + tid < a.Nout ? a.bias[n0 + tid] : 0.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const uint32_t wbytes = (uint32_t)nch * WTILE;
        tfp::mbar_arrive_expect_tx(&wbar, wbytes);
        tfp::bulk_g2s(Bs, reinterpret_cast<const unsigned char*>(a.w) + (long long)blockIdx.y * wbytes,
                      wbytes, &wbar);
    }
    // source row j (output-row coordinates: image row ya + j, periodic) into
    // ring slot (j + S) mod S, by 16-byte asynchronous copies (zero past Cs)
    auto stage = [&](int j) {
        int yy = ya + j;
        yy = yy < 0 ? yy + a.H : (yy >= a.H ? yy - a.H : yy);
        unsigned char* dst = Rs + (uint32_t)((j + S) % S) * slot_bytes;
        int g = g_first, q = q_first;       // element i = q * cg + g, stepping by ROW_NT
        for (int i = tid; i < WALK_ROWS * cg; i += ROW_NT) {
            const int c = 8 * g;
            int xx = x0 - 1 + q;
            xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
            const bool in = c < a.Cs;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             smem_u32(dst + (g * WALK_ROWS + q) * 16)),
                         "l"(src_piece(a.src, a.src2, a.C1, a.H, a.W, a.Cs, b, yy, xx, in ? c : 0)),
                         "r"(in ? 16 : 0)
                         : "memory");
            g += g_step;
            q += q_step;
            if (g >= cg) {
                g -= cg;
                ++q;
            }
        }
    };
    // warps w and w + 4 share tensor-memory lanes 32 (w % 4) ..; each takes half
    // of the BN output columns, in blocks of 16
    auto epilogue = [&](int i) {
        const int lane_row = (warp & 3) * 32 + (tid & 31);
        const size_t p = (size_t)(b * a.H + ya + i) * a.W + x0 + lane_row;
#pragma unroll
        for (int blk = 0; blk < BN / 32; ++blk) {
            const int c0 = (warp >> 2) * (BN / 2) + 16 * blk;
            if (n0 + c0 >= a.Nout) break;   // uniform per warp
            uint32_t r[16];
            const uint32_t taddr =
                tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((i & 1) * BN + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            const int n = n0 + c0;
            float z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                z[j] = __uint_as_float(r[j]) + sbias[c0 + j];
                if (a.relu) z[j] = fmaxf(z[j], 0.f);
            }
            __nv_bfloat16* d = a.out + p * a.Nout + n;
            if (n + 16 <= a.Nout) {
                reinterpret_cast<uint4*>(d)[0] = make_uint4(pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]),
                                                            pack_bf16(z[4], z[5]), pack_bf16(z[6], z[7]));
                reinterpret_cast<uint4*>(d)[1] = make_uint4(pack_bf16(z[8], z[9]), pack_bf16(z[10], z[11]),
                                                            pack_bf16(z[12], z[13]), pack_bf16(z[14], z[15]));
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n + j < a.Nout) d[j] = __float2bfloat16_rn(z[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    };
    // Copy groups: sources -1 .. 1, then one group per source 2 .. S - 3;
    // iteration i commits the group of source i + S - 2, so the group of
    // source i + 1 has S - 3 younger groups when row i needs it.
    const int D = S - 3;
    stage(-1);
    stage(0);
    stage(1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int j = 2; j <= S - 3; ++j) {
        if (j <= rows) stage(j);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    bool ok = tfp::wait_bounded(&wbar, 0, kPolls);
    int issued = 0, drained = 0;   // output rows whose MMAs were issued / seen complete
    for (int i = 0; i < rows; ++i) {
        if (i >= 1) {
            ok = ok && mbar_wait(&mbar[(i - 1) & 1], ((i - 1) >> 1) & 1);
            if (ok) drained = i;
        }
        // source i + S - 2 goes into the slot of source i - 2, read by row i - 1 only
        if (ok && i + S - 2 <= rows) stage(i + S - 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        cp_async_wait_upto(D);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // Descriptors are linear in their address field (address >> 4, far
            // below 2^14 here), so offsets are added to a base descriptor.
            const uint32_t acc_col = tbase + (uint32_t)((i & 1) * BN);
            const uint32_t idesc = instr_desc(BM, BN);
            const int sm1 = (i - 1 + S) % S, s0 = i % S, sp1 = (i + 1) % S;
            const uint64_t dsl[3] = {smem_desc(smem_u32(Rs) + (uint32_t)sm1 * slot_bytes, WALK_ROWS * 16, 128),
                                     smem_desc(smem_u32(Rs) + (uint32_t)s0 * slot_bytes, WALK_ROWS * 16, 128),
                                     smem_desc(smem_u32(Rs) + (uint32_t)sp1 * slot_bytes, WALK_ROWS * 16, 128)};
            const uint64_t bd0 = smem_desc(smem_u32(Bs), BN * 16, 128);
            uint32_t acc = 0;
            for (int ch = 0; ch < nch; ++ch) {
                const int nst = min(CC / 16, csteps - ch * (CC / 16));
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    // A: slot of source row i + dy, K-step gs = ch * 4 + s, pixel column 1 + dx
                    uint64_t ad = dsl[tap / 3] + (uint64_t)((2 * ch * (CC / 16) * WALK_ROWS + 1 + tap % 3 - 1));
                    uint64_t bd = bd0 + (uint64_t)((ch * WTILE + tap * (CC / 16) * BN * 32) >> 4);
                    for (int st = 0; st < nst; ++st) {
                        mma_f16(acc_col, ad, bd, idesc, acc);
                        acc = 1;
                        ad += 2 * WALK_ROWS;        // next 16-channel step: two group blocks
                        bd += (BN * 32) >> 4;       // next weight slice
                    }
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[i & 1])));
        }
        issued = i + 1;
        if (i >= 1) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            epilogue(i - 1);
        }
    }
    if (ok && rows > 0) {
        ok = mbar_wait(&mbar[(rows - 1) & 1], ((rows - 1) >> 1) & 1);
        ok = __syncthreads_and(ok) != 0;
        if (ok) {
            drained = rows;
            asm volatile("tcgen05.fence::after_thread_sync;");
            epilogue(rows - 1);
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(a.err, TF_ERR_TIMEOUT);
        // let issued MMAs finish (bounded) before their tensor memory is freed
        for (int i = drained; i < issued; ++i) mbar_wait(&mbar[i & 1], (i >> 1) & 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(2 * BN));
}

}  // namespace tcg
