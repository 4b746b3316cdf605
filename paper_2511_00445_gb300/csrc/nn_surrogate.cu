// Convolutional surrogate of the coupled step (declared in include/twofluid.h):
// U-Net forward / backward with tcgen05 GEMMs (nn_tc.cuh), Adam, training
// pairs captured from solver contexts, and prediction back into a context.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nn_tc.cuh"
#include "tf_internal.h"

namespace {

typedef __nv_bfloat16 bf16;
constexpr int EB = 256;             // threads of the element-wise kernels
constexpr int kHeadBlocks = 608;    // pixel ranges of the head's parameter gradient
constexpr int CIN = TF_SUR_IN, COUT = TF_SUR_OUT;

__device__ __forceinline__ int wrap_i(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ------------------------------------------------------------ GEMM operations
// Weight gradient: dW[o][tap][c] = sum_p dz[p][o] in[p + d(tap)][c], from
// channel-major copies dzT[o][p] and inT[c][p].  Split z of the pixels writes
// its partial sums to part[z][M][N]; k_sum_splits then adds the splits in
// order, so training is reproducible bit for bit (no floating-point atomics).
struct ConvBwdW {
    int M, N, K;         // M = cout, N = 9 cin, K = pixels
    int* err;
    const bf16* dzT;
    const bf16* inT;
    float* part;
    int H, W, cin;
    __device__ uint4 a_chunk(int m, int k8) const {
        const int k = k8 * 8;
        if (m >= M || k >= K) return make_uint4(0, 0, 0, 0);
        return *reinterpret_cast<const uint4*>(dzT + (size_t)m * K + k);
    }
    __device__ uint4 b_chunk(int n, int k8) const {
        const int k = k8 * 8;
        if (n >= N || k >= K) return make_uint4(0, 0, 0, 0);
        const int tap = n / cin, c = n - tap * cin;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const int x = k % W, t = k / W, y = t % H, b = t / H;    // 8 pixels of one row (W % 8 == 0)
        const bf16* row = inT + (size_t)c * K + (size_t)(b * H + wrap_i(y + dy, H)) * W;
        if (dx == 0) return *reinterpret_cast<const uint4*>(row + x);
        __align__(16) bf16 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = row[wrap_i(x + j + dx, W)];
        return *reinterpret_cast<const uint4*>(v);
    }
    __device__ void epilogue(int m, int n0, const float (&v)[16]) const {
        float* dst = part + ((size_t)blockIdx.z * M + m) * N + n0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (n0 + j < N) dst[j] = v[j];
    }
};

// Splits the pixel range of a weight-gradient GEMM is cut into: about two
// CTAs per SM of 152 over the output tiles (an upper bound; run_gemm may use
// fewer, never more).
inline int wgrad_splits(int M, int N) {
    const int tiles = ((M + 127) / 128) * ((N + 63) / 64);
    return (304 + tiles - 1) / tiles;
}

template <int BN, class Op>
cudaError_t run_gemm(const Op& op, int splits, cudaStream_t st, int* used_splits) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(tcg::k_gemm<BN, Op>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tcg::smem_bytes<BN>());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int chunks = (op.K + tcg::BK - 1) / tcg::BK;
    if (splits > chunks) splits = chunks;
    if (splits < 1) splits = 1;
    const int per = (chunks + splits - 1) / splits;
    splits = (chunks + per - 1) / per;
    const dim3 grid((op.M + tcg::BM - 1) / tcg::BM, (op.N + BN - 1) / BN, splits);
    tcg::k_gemm<BN, Op><<<grid, tcg::NTHREADS, tcg::smem_bytes<BN>(), st>>>(op, per);
    *used_splits = splits;
    return cudaGetLastError();
}

// Row-segment convolutions (forward and input gradient, tcg::k_conv_rows).
template <int BN, int CC, bool GRAD, int NACC>
cudaError_t run_rows(const tcg::ConvRowArgs& a, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(tcg::k_conv_rows<BN, CC, GRAD, NACC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tcg::row_smem_bytes<BN, CC>());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    // the most rows per CTA that still gives every SM a CTA (else one row):
    // packed rows make each MMA do more useful work, so they win as long as
    // the grid covers the SMs (measured on the 4 x 256^2 prediction)
    const int segs = (a.W + tcg::ROW_T - 1) / tcg::ROW_T, tiles = (a.Nout + BN - 1) / BN;
    const long long want = sms;
    int R = tcg::row_group(a.W, NACC, GRAD);
    while (R > 1 && (long long)segs * ((a.H + R - 1) / R) * a.B * tiles < want) --R;
    tcg::ConvRowArgs r = a;
    r.rows = R;
    const dim3 grid(segs * ((a.H + R - 1) / R) * a.B, tiles);
    tcg::k_conv_rows<BN, CC, GRAD, NACC><<<grid, tcg::ROW_NT, tcg::row_smem_bytes<BN, CC>(), st>>>(r);
    return cudaGetLastError();
}

// Row-walking forward convolution (tcg::k_conv_walk): for rows of a multiple
// of 128 pixels and up to 128 source channels, so that the weights and a
// ring of at least four source rows fit in shared memory.  The ring depth S
// and the CTAs per SM are chosen together to keep the most source rows in
// flight per SM (CTAs x (S - 3)); the rows of each (image, segment, output
// tile) are then cut into rb blocks so that the grid fills the resident CTA
// slots once.
constexpr int kWalkMaxCs = 128;

bool walks_forward(int W, int Cs) { return W % tcg::ROW_T == 0 && Cs <= kWalkMaxCs; }
constexpr int kWalkDynSmem = 227 * 1024 - 1024;   // per-CTA limit less the static part
constexpr int kSmemPerSM = 228 * 1024;

template <int BN, int CC>
cudaError_t run_walk(const tcg::ConvRowArgs& r, cudaStream_t st) {
    static bool configured = false;
    static int sms = 0, regs = 0, static_smem = 0;
    if (!configured) {
        int dev = 0;
        cudaFuncAttributes fa{};
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tcg::k_conv_walk<BN, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWalkDynSmem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tcg::k_conv_walk<BN, CC>);
        if (e != cudaSuccess) return e;
        regs = fa.numRegs > 0 ? fa.numRegs : 1;
        static_smem = (int)fa.sharedSizeBytes;
        configured = true;
    }
    int best_s = 0, best_cta = 0, best_score = -1;
    for (int S = 4; S <= tcg::WALK_MAX_SLOTS; ++S) {
        const int smem = tcg::walk_smem_bytes<BN, CC>(r.Cs, S);
        if (smem > kWalkDynSmem) break;
        int cta = kSmemPerSM / (smem + static_smem + 1024);          // 1 KB reserved per CTA
        cta = std::min(cta, 65536 / (tcg::ROW_NT * regs));
        cta = std::min(cta, 2048 / tcg::ROW_NT);
        cta = std::min(cta, 512 / (2 * BN));                         // tensor-memory columns
        const int score = cta * (S - 3);
        if (cta >= 1 && score >= best_score) {
            best_score = score;
            best_s = S;
            best_cta = cta;
        }
    }
    if (best_s == 0) return cudaErrorInvalidValue;
    const int segs = r.W / tcg::ROW_T, tiles = (r.Nout + BN - 1) / BN;
    const long long units = (long long)r.B * segs * tiles;
    long long rb = ((long long)sms * best_cta + units - 1) / units;
    if (rb < 1) rb = 1;
    if (rb > r.H) rb = r.H;
    const tcg::ConvWalkArgs a{r.src, r.w, r.bias, r.out, r.B, r.H, r.W, r.Cs, r.Nout, r.relu,
                              (int)rb, best_s, r.err, r.src2, r.C1};
    const dim3 grid((unsigned)(r.B * segs * rb), (unsigned)tiles);
    tcg::k_conv_walk<BN, CC><<<grid, tcg::ROW_NT, tcg::walk_smem_bytes<BN, CC>(r.Cs, best_s), st>>>(a);
    return cudaGetLastError();
}

// Forward: rows of a multiple of 128 pixels with few source channels walk
// (walks_forward); other layers run the row-segment kernel with the layer's
// weight layout (a.bn), rows of at most 64 pixels packing several output
// rows into two accumulators.
template <bool GRAD>
cudaError_t conv_rows(const tcg::ConvRowArgs& a, cudaStream_t st) {
    if (GRAD) return run_rows<tcg::ROW_BN, tcg::ROW_CC, true, 1>(a, st);
    if (walks_forward(a.W, a.Cs))
        return a.bn == 64 ? run_walk<64, 32>(a, st) : run_walk<tcg::ROW_BN, tcg::ROW_CC>(a, st);
    if (a.bn == 64)
        return a.W <= 64 ? run_rows<64, 32, false, 2>(a, st) : run_rows<64, 32, false, 1>(a, st);
    if (a.W <= 64) return run_rows<tcg::ROW_BN, tcg::ROW_CC, false, 2>(a, st);
    return run_rows<tcg::ROW_BN, tcg::ROW_CC, false, 1>(a, st);
}

// Bytes of one layer's pre-tiled weights: bn = 32 (tcg::row_wtile_index,
// 32 outputs x 64 source channels per block) or 64 (64 x 32).
size_t wtile_bytes(int nout, int cs, int bn = 32) {
    const int cc = bn == 64 ? 32 : tcg::ROW_CC;
    return (size_t)((nout + bn - 1) / bn) * ((cs + cc - 1) / cc) * tcg::ROW_WTILE;
}

template <class Op>
cudaError_t gemm(const Op& op, int splits, cudaStream_t st, int* used_splits) {
    if (op.N >= 128) return run_gemm<128>(op, splits, st, used_splits);
    if (op.N >= 64) return run_gemm<64>(op, splits, st, used_splits);
    if (op.N >= 32) return run_gemm<32>(op, splits, st, used_splits);
    return run_gemm<16>(op, splits, st, used_splits);
}

// ------------------------------------------------------ element-wise kernels
inline unsigned blocks(long long n) { return (unsigned)((n + EB - 1) / EB); }

// 2x2 average pool, 8 channels (16 bytes) per thread.
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int B, int H, int W,
                       int C) {   // in: H x W, out: H/2 x W/2
    const int G = C / 8;
    const long long n = (long long)B * (H / 2) * (W / 2) * G;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const int g = (int)(i % G);
    long long t = i / G;
    const int x = (int)(t % (W / 2));
    t /= (W / 2);
    const int y = (int)(t % (H / 2)), b = (int)(t / (H / 2));
    auto at = [&](int yy, int xx) {
        return *reinterpret_cast<const uint4*>(in + ((size_t)(b * H + yy) * W + xx) * C + 8 * g);
    };
    const uint4 q0 = at(2 * y, 2 * x), q1 = at(2 * y, 2 * x + 1), q2 = at(2 * y + 1, 2 * x),
                q3 = at(2 * y + 1, 2 * x + 1);
    const bf16* v0 = reinterpret_cast<const bf16*>(&q0);
    const bf16* v1 = reinterpret_cast<const bf16*>(&q1);
    const bf16* v2 = reinterpret_cast<const bf16*>(&q2);
    const bf16* v3 = reinterpret_cast<const bf16*>(&q3);
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float s4 = __bfloat162float(v0[k]) + __bfloat162float(v1[k]) + __bfloat162float(v2[k]) +
                         __bfloat162float(v3[k]);
        o[k] = __float2bfloat16_rn(0.25f * s4);
    }
    *reinterpret_cast<uint4*>(out + (size_t)(i / G) * C + 8 * g) = *reinterpret_cast<const uint4*>(o);
}

__global__ void k_pool_bwd(const float* __restrict__ d, float* __restrict__ dx, int B, int H,
                           int W, int C) {   // d: H/2 x W/2, dx: H x W (accumulate)
    const long long n = (long long)B * H * W * C;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long t = i / C;
    const int x = (int)(t % W);
    t /= W;
    const int y = (int)(t % H), b = (int)(t / H);
    dx[i] += 0.25f * d[((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
}

// Nearest upsampling of src (H/2 x W/2, Cs channels) into channels [0, Cs) of
// the concatenation dst (H x W, Cd channels); k_copy_ch puts the skip into
// channels [Cs, Cd).  8 channels (16 bytes) per thread.
__global__ void k_up_into(const bf16* __restrict__ src, bf16* __restrict__ dst, int B, int H,
                          int W, int Cs, int Cd) {
    const int G = Cs / 8;
    const long long n = (long long)B * H * W * G;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const int g = (int)(i % G);
    const long long p = i / G;
    const int x = (int)(p % W);
    const long long t = p / W;
    const int y = (int)(t % H), b = (int)(t / H);
    *reinterpret_cast<uint4*>(dst + p * Cd + 8 * g) = *reinterpret_cast<const uint4*>(
        src + ((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * Cs + 8 * g);
}

__global__ void k_copy_ch(const bf16* __restrict__ src, bf16* __restrict__ dst, long long P,
                          int Cs, int Cd, int off) {
    const int G = Cs / 8;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= P * G) return;
    const long long p = i / G;
    const int g = (int)(i % G);
    *reinterpret_cast<uint4*>(dst + p * Cd + off + 8 * g) =
        *reinterpret_cast<const uint4*>(src + p * Cs + 8 * g);
}

// Gradient of [upsampled, skip]: the skip part accumulates into dskip, the
// upsampled part sums over each 2x2 block into dsrc.
__global__ void k_cat_bwd_skip(const float* __restrict__ dcat, float* __restrict__ dskip,
                               long long P, int Cs, int Cd) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= P * (Cd - Cs)) return;
    const int Ck = Cd - Cs;
    const long long p = i / Ck;
    dskip[i] += dcat[p * Cd + Cs + (i % Ck)];
}

__global__ void k_cat_bwd_up(const float* __restrict__ dcat, float* __restrict__ dsrc, int B,
                             int H, int W, int Cs, int Cd) {   // dsrc: H/2 x W/2 x Cs
    const long long n = (long long)B * (H / 2) * (W / 2) * Cs;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % Cs);
    long long t = i / Cs;
    const int x = (int)(t % (W / 2));
    t /= (W / 2);
    const int y = (int)(t % (H / 2)), b = (int)(t / (H / 2));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            s += dcat[((size_t)(b * H + 2 * y + dy) * W + 2 * x + dx) * Cd + c];
    dsrc[i] += s;
}

// dz = bf16(dout * (out > 0)) and its channel-major copy dzT[c][p].
__global__ void k_relu_mask(const float* __restrict__ dout, const bf16* __restrict__ out,
                            bf16* __restrict__ dz, bf16* __restrict__ dzT, long long P, int C) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= P * C) return;
    const float g = __bfloat162float(out[i]) > 0.f ? dout[i] : 0.f;
    const bf16 v = __float2bfloat16_rn(g);
    dz[i] = v;
    dzT[(i % C) * P + i / C] = v;
}

__global__ void k_to_cm(const bf16* __restrict__ in, bf16* __restrict__ inT, long long P, int C) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= P * C) return;
    inT[(i % C) * P + i / C] = in[i];
}

// Bias gradient: db[o] += sum_p dzT[o][p] (one block per output channel).
__global__ void k_bias_grad(const bf16* __restrict__ dzT, long long P, float* __restrict__ db) {
    __shared__ float red[EB];
    float s = 0.f;
    for (long long p = threadIdx.x; p < P; p += EB) s += __bfloat162float(dzT[blockIdx.x * P + p]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = EB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(db + blockIdx.x, red[0]);
}

// Head: pred[p][o] = bh[o] + sum_c Wh[o][c] h[p][c] (FP32 weights, summed in
// channel order).  One thread per pixel reads its C channels as 16-byte
// pieces (C a multiple of 8); the weights sit in shared memory (dynamic,
// (COUT * C + COUT) floats).
__global__ void k_head(const bf16* __restrict__ h, const float* __restrict__ Wh,
                       const float* __restrict__ bh, float* __restrict__ pred, long long P, int C) {
    extern __shared__ float head_w[];
    for (int i = threadIdx.x; i < COUT * C + COUT; i += EB) head_w[i] = i < COUT * C ? Wh[i] : bh[i - COUT * C];
    __syncthreads();
    const long long p = (long long)blockIdx.x * EB + threadIdx.x;
    if (p >= P) return;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = head_w[COUT * C + o];
    const uint4* hp = reinterpret_cast<const uint4*>(h + p * C);
    for (int g = 0; g < C / 8; ++g) {
        const uint4 v = hp[g];
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float x = __uint_as_float(k & 1 ? w4[k >> 1] & 0xFFFF0000u : w4[k >> 1] << 16);
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] = fmaf(head_w[o * C + 8 * g + k], x, acc[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < COUT; ++o) pred[p * COUT + o] = acc[o];
}

// Loss terms and dpred = 2 (pred - target) / n; per-block partial loss sums.
__global__ void k_loss(const float* __restrict__ pred, const float* __restrict__ tgt,
                       float* __restrict__ dpred, long long n, double* __restrict__ part) {
    __shared__ double red[EB];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * EB + threadIdx.x; i < n; i += (long long)gridDim.x * EB) {
        const float d = pred[i] - tgt[i];
        dpred[i] = 2.f * d / (float)n;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = EB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Head backward, input part: dh[p][c] += sum_o Wh[o][c] dpred[p][o].
__global__ void k_head_bwd(const bf16* __restrict__ h, const float* __restrict__ dpred,
                           const float* __restrict__ Wh, float* __restrict__ dh, long long P, int C) {
    for (long long p = (long long)blockIdx.x * EB + threadIdx.x; p < P; p += (long long)gridDim.x * EB) {
        float g[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) g[o] = dpred[p * COUT + o];
        for (int c = 0; c < C; ++c) {
            float s = 0.f;
#pragma unroll
            for (int o = 0; o < COUT; ++o) s += Wh[o * C + c] * g[o];
            dh[p * C + c] += s;
        }
    }
}

// Head backward, parameter part: block b sums pixels [b P / nb, (b + 1) P / nb)
// in order; thread k owns entry k of [dWh (COUT x C) | dbh (COUT)]:
// dWh[o][c] = sum_p dpred[p][o] h[p][c], dbh[o] = sum_p dpred[p][o].  Each
// block writes its partial row part[b][.]; k_head_sum adds the rows in order.
__global__ void k_head_wgrad(const bf16* __restrict__ h, const float* __restrict__ dpred,
                             float* __restrict__ part, long long P, int C) {
    const int nk = COUT * C + COUT;
    const long long p0 = (long long)blockIdx.x * P / gridDim.x, p1 = (long long)(blockIdx.x + 1) * P / gridDim.x;
    for (int k = threadIdx.x; k < nk; k += EB) {
        const bool w = k < COUT * C;
        const int o = w ? k / C : k - COUT * C, c = w ? k - o * C : 0;
        float s = 0.f;
        for (long long p = p0; p < p1; ++p)
            s += dpred[p * COUT + o] * (w ? __bfloat162float(h[p * C + c]) : 1.f);
        part[(size_t)blockIdx.x * nk + k] = s;
    }
}

// dst[i] += sum_z part[z][i] for z = 0 .. nz - 1, in that order.
__global__ void k_sum_splits(const float* __restrict__ part, int nz, long long n, float* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[(size_t)z * n + i];
    dst[i] += s;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of one convolution's weights w[o][tap][c], pre-tiled for the
// forward pass (rows o, source channels c) and for the input gradient (rows
// c, source channels o).  Tile entries outside the layer stay zero.
__global__ void k_weights_bf16(const float* __restrict__ w, unsigned char* __restrict__ wf,
                               unsigned char* __restrict__ wg, int cout, int cin, int bn) {
    const long long n = (long long)cout * 9 * cin;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % cin);
    const int tap = (int)((i / cin) % 9), o = (int)(i / (9LL * cin));
    const bf16 v = __float2bfloat16_rn(w[i]);
    *reinterpret_cast<bf16*>(wf + (bn == 64 ? tcg::wtile_index<64, 32>(o, tap, c, cin)
                                             : tcg::row_wtile_index(o, tap, c, cin))) = v;
    *reinterpret_cast<bf16*>(wg + tcg::row_wtile_index(c, tap, o, cout)) = v;
}

// Raw fields of a solver instance: phi - phi_ref, Q_xx, Q_xy, u1x, u1y, u2x, u2y.
__global__ void k_capture(const float* __restrict__ phi, const float* __restrict__ Q,
                          const float* __restrict__ mac, long long N, int b, float* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= N) return;
    dst[i] = phi[b * N + i];
    dst[N + i] = Q[2 * b * N + i];
    dst[2 * N + i] = Q[(2 * b + 1) * N + i];
    for (int k = 0; k < 4; ++k) dst[(3 + k) * N + i] = mac[(8 * b + k) * N + i];
}

// Per-channel sums over the pairs: [0..6] input, [7..13] input^2,
// [14..20] increment, [21..27] increment^2 (partials per block).
__global__ void k_stats(const float* __restrict__ data, long long N, int n_pairs,
                        double* __restrict__ part) {
    __shared__ double red[28][32];
    double s[28];
    for (int k = 0; k < 28; ++k) s[k] = 0.0;
    const long long total = (long long)n_pairs * N;
    for (long long j = (long long)blockIdx.x * EB + threadIdx.x; j < total; j += (long long)gridDim.x * EB) {
        const long long pr = j / N, i = j % N;
        const float* in = data + pr * 14 * N;
        const float* tg = in + 7 * N;
        for (int c = 0; c < 7; ++c) {
            const double a = in[c * N + i], d = (double)tg[c * N + i] - a;
            s[c] += a;
            s[7 + c] += a * a;
            s[14 + c] += d;
            s[21 + c] += d * d;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 28; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        double v = 0.0;
        for (int w = 0; w < EB / 32; ++w) v += red[threadIdx.x][w];
        part[blockIdx.x * 28 + threadIdx.x] = v;
    }
}

// Normalisation constants: mean[7], inv_std[7], dmean[7], dstd[7].
struct Norm {
    float mean[7], inv_std[7], dmean[7], dstd[7];
};

// Minibatch from pairs idx[0..B): x (BF16, 8 channels) and target (FP32, 7).
__global__ void k_assemble(const float* __restrict__ data, const int* __restrict__ idx,
                           const float* __restrict__ zeta, Norm nm, float zscale, long long N,
                           int B, bf16* __restrict__ x, float* __restrict__ tgt) {
    const long long j = (long long)blockIdx.x * EB + threadIdx.x;
    if (j >= (long long)B * N) return;
    const int bi = (int)(j / N);
    const long long i = j % N;
    const float* in = data + (long long)idx[bi] * 14 * N;
    const float* tg = in + 7 * N;
    __align__(16) bf16 xv[8];
    for (int c = 0; c < 7; ++c) {
        const float a = in[c * N + i];
        xv[c] = __float2bfloat16_rn((a - nm.mean[c]) * nm.inv_std[c]);
        if (tgt) tgt[j * 7 + c] = (tg[c * N + i] - a - nm.dmean[c]) / nm.dstd[c];
    }
    xv[7] = __float2bfloat16_rn(zeta[idx[bi]] * zscale);
    *reinterpret_cast<uint4*>(x + j * 8) = *reinterpret_cast<const uint4*>(xv);
}

// Prediction written into instance b of a solver context: the stored phi
// deviation and Q planes, and the populations at the equilibrium of the rest
// densities and the predicted velocities (pull layout: f_i(x) is stored at
// x - c_i), in the context's storage mode.  FP32 arithmetic.
__global__ void k_writeback(const float* __restrict__ raw, const float* __restrict__ pred, Norm nm,
                            int nx, int ny, int b, float* __restrict__ phi, float* __restrict__ Q,
                            void* __restrict__ f, const DevParams* __restrict__ prm, int storage) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * EB + threadIdx.x;
    if (i >= N) return;
    float v[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) v[c] = raw[c * N + i] + nm.dmean[c] + nm.dstd[c] * pred[i * 7 + c];
    phi[b * N + i] = v[0];
    Q[2 * b * N + i] = v[1];
    Q[(2 * b + 1) * N + i] = v[2];
    const int x = (int)(i % nx), y = (int)(i / nx);
#pragma unroll
    for (int fl = 0; fl < 2; ++fl) {
        const float ux = v[3 + 2 * fl], uy = v[4 + 2 * fl];
        const float rho = fl ? prm[b].rho2 : prm[b].rho1;
        const float uu = ux * ux + uy * uy;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float cu = d2q9_cx(k) * ux + d2q9_cy(k) * uy;
            const float w = d2q9_w(k);
            const float dev = w * (rho - 1.f) + w * rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu);
            const int sx = wrap_i(x - d2q9_cx(k), nx), sy = wrap_i(y - d2q9_cy(k), ny);
            pop_store(f, pop_index(b, fl, k, (long long)sy * nx + sx, N), dev, storage);
        }
    }
}

// SplitMix64 (Steele, Lea & Flood 2014) for weight initialisation and
// minibatch draws.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform(uint64_t& s) { return (double)(splitmix(s) >> 11) * 0x1.0p-53; }

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Conv {
    int cin, cout, level;
    long long w_off, b_off;      // offsets into the flat FP32 parameter vector
    size_t wb, wt;               // byte offsets of the BF16 copies
    int in_t, out_t;             // activation tensors
    int bn = 32;                 // forward weight layout (see forward_bn)
};
struct Tensor {
    int C, level;
    size_t act, grad;            // byte offsets (BF16 activations, FP32 gradients)
};
enum OpKind { OP_CONV, OP_POOL, OP_CAT };
struct Op {
    int kind, a, b, c;           // conv: a = conv index; pool: a -> b; cat: up a, skip b -> c
};

}  // namespace

struct tf_surrogate {
    tf_sur_config cfg{};
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    std::vector<Conv> convs;
    std::vector<Tensor> tensors;
    std::vector<Op> ops;
    long long n_params = 0, head_w = 0, head_b = 0;
    int x_t = 0, dec0_t = 0;     // input and last decoder tensors
    // workspace regions (byte offsets)
    size_t p_off = 0, g_off = 0, m_off = 0, v_off = 0, wbf_off = 0, act_off = 0, grad_off = 0;
    size_t dz_off = 0, dzT_off = 0, inT_off = 0, pred_off = 0, tgt_off = 0, dpred_off = 0;
    size_t data_off = 0, zeta_off = 0, idx_off = 0, part_off = 0, err_off = 0;
    size_t raw_off = 0, wpart_off = 0, hpart_off = 0, total = 0;
    long long max_cp = 0;        // largest pixels x channels of any tensor at max_batch
    std::vector<float> zeta;     // per pair
    Norm norm{};
    float zscale = 1.f;
    bool norm_ready = false;
    int adam_t = 0;
    std::string last_error;
    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    long long pixels(int level, int B) const {
        return (long long)B * (cfg.ny >> level) * (cfg.nx >> level);
    }
};

namespace {

int sfail(tf_surrogate* s, int code, const std::string& msg) {
    if (s) s->last_error = msg;
    return code;
}
#define SCK(s, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return sfail(s, TF_ERR_CUDA, std::string(#call) + ": " +     \
                                                                cudaGetErrorString(e_));   \
    } while (0)

bool valid_cfg(const tf_sur_config& c) {
    if (c.levels < 1 || c.levels > 5) return false;
    if (c.base_channels != 16 && c.base_channels != 32 && c.base_channels != 64) return false;
    const int q = 8 << (c.levels - 1);
    if (c.nx < q || c.ny < q || c.nx % q || c.ny % q) return false;
    if (c.nx > 4096 || c.ny > 4096) return false;
    return c.max_batch >= 1 && c.max_pairs >= 1 && c.horizon >= 1;
}

// Builds the layer graph and the workspace layout; returns the byte total.
size_t plan(tf_surrogate* s) {
    const tf_sur_config& c = s->cfg;
    const int L = c.levels, B = c.max_batch;
    s->convs.clear();
    s->tensors.clear();
    s->ops.clear();
    auto tensor = [&](int C, int level) {
        s->tensors.push_back(Tensor{C, level, 0, 0});
        return (int)s->tensors.size() - 1;
    };
    long long np = 0;
    auto conv = [&](int in_t, int cout) {
        const Tensor t = s->tensors[in_t];
        Conv cv{t.C, cout, t.level, np, np + (long long)cout * 9 * t.C, 0, 0, in_t, 0};
        // forward layers with a multiple of 64 outputs take 64-wide output
        // tiles (half the MMAs of 32-wide ones): on the row-segment kernel for
        // rows of at least 64 pixels (narrower rows leave too small a grid:
        // measured slower on the 4 x 256^2 prediction), and on the walking
        // kernel up to 96 source channels (weights and a four-row ring must fit)
        const int W = c.nx >> t.level;
        const bool walk = walks_forward(W, t.C);
        cv.bn = cout % 64 == 0 && t.C % 32 == 0 && (walk ? t.C <= 96 : W >= 64) ? 64 : 32;
        np += (long long)cout * 9 * t.C + cout;
        cv.out_t = tensor(cout, t.level);
        s->convs.push_back(cv);
        s->ops.push_back(Op{OP_CONV, (int)s->convs.size() - 1, 0, 0});
        return cv.out_t;
    };
    s->x_t = tensor(CIN, 0);
    std::vector<int> skip(L);
    int h = s->x_t;
    for (int l = 0; l < L; ++l) {
        if (l > 0) {
            const int p = tensor(s->tensors[h].C, l);
            s->ops.push_back(Op{OP_POOL, h, p, 0});
            h = p;
        }
        h = conv(h, c.base_channels << l);
        h = conv(h, c.base_channels << l);
        skip[l] = h;
    }
    for (int l = L - 2; l >= 0; --l) {
        const int cat = tensor(s->tensors[h].C + s->tensors[skip[l]].C, l);
        s->ops.push_back(Op{OP_CAT, h, skip[l], cat});
        h = conv(cat, c.base_channels << l);
        h = conv(h, c.base_channels << l);
    }
    s->dec0_t = h;
    s->head_w = np;
    np += (long long)COUT * c.base_channels;
    s->head_b = np;
    np += COUT;
    s->n_params = np;

    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    s->p_off = take(np * 4);
    s->g_off = take(np * 4);
    s->m_off = take(np * 4);
    s->v_off = take(np * 4);
    for (Conv& cv : s->convs) {
        cv.wb = take(wtile_bytes(cv.cout, cv.cin, cv.bn));
        cv.wt = take(wtile_bytes(cv.cin, cv.cout));
    }
    long long max_cp = 0;
    for (Tensor& t : s->tensors) {
        const long long cp = s->pixels(t.level, B) * t.C;
        if (cp > max_cp) max_cp = cp;
        t.act = take((size_t)cp * 2);
        t.grad = take((size_t)cp * 4);
    }
    s->max_cp = max_cp;
    s->dz_off = take((size_t)max_cp * 2);
    s->dzT_off = take((size_t)max_cp * 2);
    s->inT_off = take((size_t)max_cp * 2);
    const long long P0 = s->pixels(0, B), N = (long long)c.nx * c.ny;
    s->pred_off = take((size_t)P0 * COUT * 4);
    s->tgt_off = take((size_t)P0 * COUT * 4);
    s->dpred_off = take((size_t)P0 * COUT * 4);
    s->data_off = take((size_t)c.max_pairs * 14 * N * 4);
    s->raw_off = take((size_t)B * 14 * N * 4);             // prediction inputs (one per instance)
    s->zeta_off = take((size_t)(c.max_pairs + B) * 4);
    s->idx_off = take((size_t)B * 4);
    s->part_off = take(1024 * 28 * 8);
    size_t wpart = 0;                                          // weight-gradient split partials
    for (const Conv& cv : s->convs) {
        const size_t mn = (size_t)cv.cout * 9 * cv.cin;
        wpart = std::max(wpart, (size_t)wgrad_splits(cv.cout, 9 * cv.cin) * mn);
    }
    s->wpart_off = take(wpart * 4);
    s->hpart_off = take((size_t)kHeadBlocks * (COUT * c.base_channels + COUT) * 4);
    s->err_off = take(64);
    s->total = off;
    return off;
}

// ---------------------------------------------------------------- passes
// keep_cat: write every concatenation [upsampled, skip] into its tensor (the
// backward pass reads it).  A forward-only pass leaves them virtual: the
// convolution that consumes one reads the two parts in place.
cudaError_t forward_pass(tf_surrogate* s, int B, bool keep_cat) {
    cudaStream_t st = s->stream;
    int* err = s->at<int>(s->err_off);
    const float* P = s->at<float>(s->p_off);
    int virt_cat = -1, virt_up = -1, virt_skip = -1;   // the pending virtual concatenation
    for (const Op& op : s->ops) {
        if (op.kind == OP_CONV) {
            const Conv& cv = s->convs[op.a];
            const Tensor& ti = s->tensors[cv.in_t];
            const int H = s->cfg.ny >> ti.level, W = s->cfg.nx >> ti.level;
            tcg::ConvRowArgs g{s->at<bf16>(ti.act), s->at<bf16>(cv.wb), P + cv.b_off,
                               s->at<bf16>(s->tensors[cv.out_t].act), nullptr,
                               B, H, W, cv.cin, cv.cout, 1, err};
            g.bn = cv.bn;
            if (cv.in_t == virt_cat) {
                g.src = s->at<bf16>(s->tensors[virt_up].act);
                g.src2 = s->at<bf16>(s->tensors[virt_skip].act);
                g.C1 = s->tensors[virt_up].C;
                virt_cat = -1;
            }
            cudaError_t e = conv_rows<false>(g, st);
            if (e != cudaSuccess) return e;
        } else if (op.kind == OP_POOL) {
            const Tensor& a = s->tensors[op.a];
            const int H = s->cfg.ny >> a.level, W = s->cfg.nx >> a.level;
            k_pool<<<blocks((long long)B * H * W * a.C / 32), EB, 0, st>>>(
                s->at<bf16>(a.act), s->at<bf16>(s->tensors[op.b].act), B, H, W, a.C);
        } else if (!keep_cat) {
            virt_cat = op.c;
            virt_up = op.a;
            virt_skip = op.b;
        } else {
            const Tensor& up = s->tensors[op.a];
            const Tensor& sk = s->tensors[op.b];
            const Tensor& cat = s->tensors[op.c];
            const int H = s->cfg.ny >> cat.level, W = s->cfg.nx >> cat.level;
            const long long Pp = (long long)B * H * W;
            k_up_into<<<blocks(Pp * up.C / 8), EB, 0, st>>>(s->at<bf16>(up.act), s->at<bf16>(cat.act),
                                                           B, H, W, up.C, cat.C);
            k_copy_ch<<<blocks(Pp * sk.C / 8), EB, 0, st>>>(s->at<bf16>(sk.act), s->at<bf16>(cat.act),
                                                           Pp, sk.C, cat.C, up.C);
        }
    }
    const Tensor& d0 = s->tensors[s->dec0_t];
    const long long P0 = s->pixels(0, B);
    k_head<<<blocks(P0), EB, (COUT * d0.C + COUT) * sizeof(float), st>>>(
        s->at<bf16>(d0.act), P + s->head_w, P + s->head_b, s->at<float>(s->pred_off), P0, d0.C);
    return cudaGetLastError();
}

// Loss of the current prediction against s->tgt and the gradients in s->g.
cudaError_t backward_pass(tf_surrogate* s, int B, double* loss) {
    cudaStream_t st = s->stream;
    int* err = s->at<int>(s->err_off);
    const float* P = s->at<float>(s->p_off);
    float* G = s->at<float>(s->g_off);
    cudaError_t e = cudaMemsetAsync(G, 0, s->n_params * 4, st);
    for (const Tensor& t : s->tensors)
        if (e == cudaSuccess) e = cudaMemsetAsync(s->ws + t.grad, 0, (size_t)s->pixels(t.level, B) * t.C * 4, st);
    if (e != cudaSuccess) return e;
    const long long P0 = s->pixels(0, B);
    const long long n = P0 * COUT;
    const int lb = 256;
    k_loss<<<lb, EB, 0, st>>>(s->at<float>(s->pred_off), s->at<float>(s->tgt_off),
                              s->at<float>(s->dpred_off), n, s->at<double>(s->part_off));
    const Tensor& d0 = s->tensors[s->dec0_t];
    k_head_bwd<<<152, EB, 0, st>>>(s->at<bf16>(d0.act), s->at<float>(s->dpred_off), P + s->head_w,
                                   s->at<float>(d0.grad), P0, d0.C);
    const long long nhead = (long long)COUT * d0.C + COUT;     // [dWh | dbh] at G + head_w
    k_head_wgrad<<<kHeadBlocks, EB, 0, st>>>(s->at<bf16>(d0.act), s->at<float>(s->dpred_off),
                                            s->at<float>(s->hpart_off), P0, d0.C);
    k_sum_splits<<<blocks(nhead), EB, 0, st>>>(s->at<float>(s->hpart_off), kHeadBlocks, nhead,
                                               G + s->head_w);
    for (int k = (int)s->ops.size() - 1; k >= 0; --k) {
        const Op& op = s->ops[k];
        if (op.kind == OP_CONV) {
            const Conv& cv = s->convs[op.a];
            const Tensor& ti = s->tensors[cv.in_t];
            const Tensor& to = s->tensors[cv.out_t];
            const int H = s->cfg.ny >> ti.level, W = s->cfg.nx >> ti.level;
            const long long Pp = (long long)B * H * W;
            bf16* dz = s->at<bf16>(s->dz_off);
            bf16* dzT = s->at<bf16>(s->dzT_off);
            bf16* inT = s->at<bf16>(s->inT_off);
            k_relu_mask<<<blocks(Pp * cv.cout), EB, 0, st>>>(s->at<float>(to.grad), s->at<bf16>(to.act),
                                                             dz, dzT, Pp, cv.cout);
            k_to_cm<<<blocks(Pp * cv.cin), EB, 0, st>>>(s->at<bf16>(ti.act), inT, Pp, cv.cin);
            ConvBwdW gw;
            gw.M = cv.cout;
            gw.N = 9 * cv.cin;
            gw.K = (int)Pp;
            gw.err = err;
            gw.dzT = dzT;
            gw.inT = inT;
            gw.part = s->at<float>(s->wpart_off);
            gw.H = H;
            gw.W = W;
            gw.cin = cv.cin;
            int used = 0;
            e = gemm(gw, wgrad_splits(gw.M, gw.N), st, &used);
            if (e != cudaSuccess) return e;
            const long long mn = (long long)gw.M * gw.N;
            k_sum_splits<<<blocks(mn), EB, 0, st>>>(gw.part, used, mn, G + cv.w_off);
            k_bias_grad<<<cv.cout, EB, 0, st>>>(dzT, Pp, G + cv.b_off);
            if (cv.in_t != s->x_t) {
                const tcg::ConvRowArgs gd{dz, s->at<bf16>(cv.wt), nullptr, nullptr,
                                          s->at<float>(ti.grad), B, H, W, cv.cout, cv.cin, 0, err};
                e = conv_rows<true>(gd, st);
                if (e != cudaSuccess) return e;
            }
        } else if (op.kind == OP_POOL) {
            const Tensor& a = s->tensors[op.a];
            const int H = s->cfg.ny >> a.level, W = s->cfg.nx >> a.level;
            k_pool_bwd<<<blocks((long long)B * H * W * a.C), EB, 0, st>>>(
                s->at<float>(s->tensors[op.b].grad), s->at<float>(a.grad), B, H, W, a.C);
        } else {
            const Tensor& up = s->tensors[op.a];
            const Tensor& sk = s->tensors[op.b];
            const Tensor& cat = s->tensors[op.c];
            const int H = s->cfg.ny >> cat.level, W = s->cfg.nx >> cat.level;
            const long long Pp = (long long)B * H * W;
            k_cat_bwd_skip<<<blocks(Pp * sk.C), EB, 0, st>>>(s->at<float>(cat.grad),
                                                             s->at<float>(sk.grad), Pp, up.C, cat.C);
            k_cat_bwd_up<<<blocks(Pp * up.C / 4), EB, 0, st>>>(s->at<float>(cat.grad),
                                                              s->at<float>(up.grad), B, H, W, up.C,
                                                              cat.C);
        }
    }
    if (loss) {
        std::vector<double> part(lb);
        e = cudaMemcpyAsync(part.data(), s->at<double>(s->part_off), lb * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        double t = 0.0;
        for (double v : part) t += v;
        *loss = t / (double)n;
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t refresh_bf16(tf_surrogate* s) {
    const float* P = s->at<float>(s->p_off);
    for (const Conv& cv : s->convs)
        k_weights_bf16<<<blocks((long long)cv.cout * 9 * cv.cin), EB, 0, s->stream>>>(
            P + cv.w_off, s->at<unsigned char>(cv.wb), s->at<unsigned char>(cv.wt), cv.cout, cv.cin, cv.bn);
    return cudaGetLastError();
}

int check_status(tf_surrogate* s) {
    int flag = 0;
    SCK(s, cudaMemcpyAsync(&flag, s->at<int>(s->err_off), sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    if (flag) {
        SCK(s, cudaMemsetAsync(s->at<int>(s->err_off), 0, sizeof(int), s->stream));
        return sfail(s, flag, "a tensor-core GEMM wait timed out");
    }
    return TF_OK;
}

int upload_x(tf_surrogate* s, const float* x, int batch) {
    const long long n = s->pixels(0, batch) * CIN;
    std::vector<uint16_t> h(n);
    for (long long i = 0; i < n; ++i) {
        const bf16 v = __float2bfloat16_rn(x[i]);
        std::memcpy(&h[i], &v, 2);
    }
    SCK(s, cudaMemcpyAsync(s->ws + s->tensors[s->x_t].act, h.data(), n * 2, cudaMemcpyHostToDevice,
                           s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    return TF_OK;
}

}  // namespace

extern "C" {

size_t tf_sur_workspace_bytes(const tf_sur_config* cfg) {
    if (!cfg || !valid_cfg(*cfg)) return 0;
    tf_surrogate tmp;
    tmp.cfg = *cfg;
    return plan(&tmp);
}

int tf_sur_create(const tf_sur_config* cfg, void* d_workspace, size_t workspace_bytes, void* stream,
                  tf_surrogate** out) {
    if (!out) return TF_ERR_ARG;
    *out = nullptr;
    if (!cfg || !valid_cfg(*cfg)) return TF_ERR_ARG;
    tf_surrogate* s = new (std::nothrow) tf_surrogate();
    if (!s) return TF_ERR_ARG;
    s->cfg = *cfg;
    const size_t need = plan(s);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255) || workspace_bytes < need) {
        delete s;
        return TF_ERR_WORKSPACE;
    }
    s->ws = static_cast<char*>(d_workspace);
    s->stream = static_cast<cudaStream_t>(stream);
    s->zeta.assign(cfg->max_pairs, 0.f);
    cudaError_t e = cudaMemsetAsync(s->ws, 0, s->total, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        delete s;
        return TF_ERR_CUDA;
    }
    *out = s;
    return TF_OK;
}

int tf_sur_destroy(tf_surrogate* s) {
    if (!s) return TF_ERR_ARG;
    cudaStreamSynchronize(s->stream);
    delete s;
    return TF_OK;
}

const char* tf_sur_last_error(const tf_surrogate* s) { return s ? s->last_error.c_str() : "null surrogate"; }

int64_t tf_sur_num_params(const tf_surrogate* s) { return s ? s->n_params : -1; }

int tf_sur_set_weights(tf_surrogate* s, const float* host, int64_t n) {
    if (!s) return TF_ERR_ARG;
    if (!host || n != s->n_params) return sfail(s, TF_ERR_ARG, "weight count mismatch");
    SCK(s, cudaMemcpyAsync(s->at<float>(s->p_off), host, n * 4, cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemsetAsync(s->at<float>(s->m_off), 0, n * 4, s->stream));
    SCK(s, cudaMemsetAsync(s->at<float>(s->v_off), 0, n * 4, s->stream));
    s->adam_t = 0;
    SCK(s, refresh_bf16(s));
    SCK(s, cudaStreamSynchronize(s->stream));
    return TF_OK;
}

int tf_sur_get_weights(tf_surrogate* s, float* host, int64_t n) {
    if (!s) return TF_ERR_ARG;
    if (!host || n != s->n_params) return sfail(s, TF_ERR_ARG, "weight count mismatch");
    SCK(s, cudaMemcpyAsync(host, s->at<float>(s->p_off), n * 4, cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    return TF_OK;
}

int tf_sur_init_weights(tf_surrogate* s, uint64_t seed) {
    if (!s) return TF_ERR_ARG;
    std::vector<float> w(s->n_params, 0.f);
    uint64_t st = seed;
    auto normal = [&]() {   // Box-Muller on two SplitMix64 uniforms
        const double u1 = 1.0 - uniform(st), u2 = uniform(st);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    };
    for (const Conv& cv : s->convs) {
        const double sd = std::sqrt(2.0 / (9.0 * cv.cin));
        for (long long i = 0; i < (long long)cv.cout * 9 * cv.cin; ++i) w[cv.w_off + i] = (float)(sd * normal());
    }
    const int C0 = s->cfg.base_channels;
    for (long long i = 0; i < (long long)COUT * C0; ++i) w[s->head_w + i] = (float)(normal() / std::sqrt((double)C0));
    return tf_sur_set_weights(s, w.data(), s->n_params);
}

int tf_sur_forward(tf_surrogate* s, const float* x, int batch, float* out) {
    const TfRange nvtx_range("tf_sur_forward");
    if (!s) return TF_ERR_ARG;
    if (!x || !out || batch < 1 || batch > s->cfg.max_batch) return sfail(s, TF_ERR_ARG, "bad batch or null array");
    int rc = upload_x(s, x, batch);
    if (rc != TF_OK) return rc;
    SCK(s, forward_pass(s, batch, false));
    if ((rc = check_status(s)) != TF_OK) return rc;
    SCK(s, cudaMemcpyAsync(out, s->at<float>(s->pred_off), s->pixels(0, batch) * COUT * 4,
                           cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    return TF_OK;
}

int tf_sur_gradients(tf_surrogate* s, const float* x, const float* target, int batch, double* loss,
                     float* grad, int64_t n) {
    if (!s) return TF_ERR_ARG;
    if (!x || !target || batch < 1 || batch > s->cfg.max_batch)
        return sfail(s, TF_ERR_ARG, "bad batch or null array");
    if (grad && n != s->n_params) return sfail(s, TF_ERR_ARG, "gradient count mismatch");
    int rc = upload_x(s, x, batch);
    if (rc != TF_OK) return rc;
    SCK(s, cudaMemcpyAsync(s->at<float>(s->tgt_off), target, s->pixels(0, batch) * COUT * 4,
                           cudaMemcpyHostToDevice, s->stream));
    SCK(s, forward_pass(s, batch, true));
    double l = 0.0;
    SCK(s, backward_pass(s, batch, &l));
    if ((rc = check_status(s)) != TF_OK) return rc;
    if (loss) *loss = l;
    if (grad) {
        SCK(s, cudaMemcpyAsync(grad, s->at<float>(s->g_off), n * 4, cudaMemcpyDeviceToHost, s->stream));
        SCK(s, cudaStreamSynchronize(s->stream));
    }
    return TF_OK;
}

int tf_sur_add_pair(tf_surrogate* s, int slot, tf_ctx* ctx, int inst, int which) {
    if (!s || !ctx) return TF_ERR_ARG;
    if (slot < 0 || slot >= s->cfg.max_pairs || (which != 0 && which != 1) || inst < 0 ||
        inst >= ctx->batch)
        return sfail(s, TF_ERR_ARG, "bad slot, instance or role");
    if (ctx->nx != s->cfg.nx || ctx->ny != s->cfg.ny || ctx->stream != s->stream)
        return sfail(s, TF_ERR_ARG, "solver grid or stream differs from the surrogate's");
    SCK(s, tf_launch_flush(ctx));
    SCK(s, tf_launch_macro(ctx, ctx->d.macro));
    const long long N = ctx->N;
    k_capture<<<blocks(N), EB, 0, s->stream>>>(ctx->d.phi[ctx->pcur], ctx->d.Q[ctx->pcur], ctx->d.macro,
                                               N, inst,
                                               s->at<float>(s->data_off) + ((long long)slot * 2 + which) * 7 * N);
    SCK(s, cudaGetLastError());
    s->zeta[slot] = (float)ctx->params[inst].zeta;
    return TF_OK;
}

int tf_sur_fit_normalisation(tf_surrogate* s, int n_pairs) {
    if (!s) return TF_ERR_ARG;
    if (n_pairs < 1 || n_pairs > s->cfg.max_pairs) return sfail(s, TF_ERR_ARG, "bad pair count");
    const long long N = (long long)s->cfg.nx * s->cfg.ny;
    const int nb = 512;
    k_stats<<<nb, EB, 0, s->stream>>>(s->at<float>(s->data_off), N, n_pairs, s->at<double>(s->part_off));
    SCK(s, cudaGetLastError());
    std::vector<double> part((size_t)nb * 28);
    SCK(s, cudaMemcpyAsync(part.data(), s->at<double>(s->part_off), part.size() * 8, cudaMemcpyDeviceToHost,
                           s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    double t[28] = {};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 28; ++k) t[k] += part[(size_t)b * 28 + k];
    const double cnt = (double)n_pairs * N;
    for (int c = 0; c < 7; ++c) {
        const double m = t[c] / cnt, var = t[7 + c] / cnt - m * m;
        const double dm = t[14 + c] / cnt, dvar = t[21 + c] / cnt - dm * dm;
        s->norm.mean[c] = (float)m;
        s->norm.inv_std[c] = (float)(1.0 / std::sqrt(var > 1e-30 ? var : 1e-30));
        s->norm.dmean[c] = (float)dm;
        s->norm.dstd[c] = (float)std::sqrt(dvar > 1e-30 ? dvar : 1e-30);
    }
    float zmax = 0.f;
    for (int p = 0; p < n_pairs; ++p) zmax = std::fmax(zmax, std::fabs(s->zeta[p]));
    s->zscale = zmax > 0.f ? 1.f / zmax : 1.f;
    SCK(s, cudaMemcpyAsync(s->at<float>(s->zeta_off), s->zeta.data(), n_pairs * 4, cudaMemcpyHostToDevice,
                           s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    s->norm_ready = true;
    return TF_OK;
}

int tf_sur_train(tf_surrogate* s, int n_pairs, int steps, int batch, double lr, uint64_t seed,
                 double* losses) {
    const TfRange nvtx_range("tf_sur_train");
    if (!s) return TF_ERR_ARG;
    if (!s->norm_ready) return sfail(s, TF_ERR_ARG, "call tf_sur_fit_normalisation first");
    if (n_pairs < 1 || n_pairs > s->cfg.max_pairs || steps < 0 || batch < 1 || batch > s->cfg.max_batch ||
        !(lr > 0))
        return sfail(s, TF_ERR_ARG, "bad training arguments");
    const long long N = (long long)s->cfg.nx * s->cfg.ny;
    uint64_t st = seed;
    std::vector<int> idx(batch);
    for (int it = 0; it < steps; ++it) {
        for (int b = 0; b < batch; ++b) idx[b] = (int)(splitmix(st) % (uint64_t)n_pairs);
        SCK(s, cudaMemcpyAsync(s->at<int>(s->idx_off), idx.data(), batch * 4, cudaMemcpyHostToDevice,
                               s->stream));
        k_assemble<<<blocks((long long)batch * N), EB, 0, s->stream>>>(
            s->at<float>(s->data_off), s->at<int>(s->idx_off), s->at<float>(s->zeta_off), s->norm,
            s->zscale, N, batch, s->at<bf16>(s->tensors[s->x_t].act), s->at<float>(s->tgt_off));
        SCK(s, forward_pass(s, batch, true));
        double l = 0.0;
        SCK(s, backward_pass(s, batch, losses ? &l : nullptr));
        if (losses) losses[it] = l;
        s->adam_t += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
        k_adam<<<blocks(s->n_params), EB, 0, s->stream>>>(s->at<float>(s->p_off), s->at<float>(s->g_off),
                                                         s->at<float>(s->m_off), s->at<float>(s->v_off),
                                                         s->n_params, (float)lr, b1, b2, c1, c2, 1e-8f);
        SCK(s, refresh_bf16(s));
    }
    return check_status(s);
}

int tf_sur_predict(tf_surrogate* s, tf_ctx* ctx, int inst) {
    const TfRange nvtx_range("tf_sur_predict");
    if (!s || !ctx) return TF_ERR_ARG;
    if (!s->norm_ready) return sfail(s, TF_ERR_ARG, "call tf_sur_fit_normalisation first");
    const int i0 = inst < 0 ? 0 : inst, nb = inst < 0 ? ctx->batch : 1;
    if (inst < -1 || inst >= ctx->batch) return sfail(s, TF_ERR_ARG, "bad instance");
    if (nb > s->cfg.max_batch) return sfail(s, TF_ERR_ARG, "more instances than max_batch");
    if (ctx->nx != s->cfg.nx || ctx->ny != s->cfg.ny || ctx->stream != s->stream)
        return sfail(s, TF_ERR_ARG, "solver grid or stream differs from the surrogate's");
    const long long N = ctx->N;
    SCK(s, tf_launch_flush(ctx));
    SCK(s, tf_launch_macro(ctx, ctx->d.macro));
    // Prediction inputs: slot k holds instance i0 + k; their zetas follow the dataset's.
    float* raw = s->at<float>(s->raw_off);
    std::vector<float> z(nb);
    std::vector<int> idx(nb);
    for (int k = 0; k < nb; ++k) {
        k_capture<<<blocks(N), EB, 0, s->stream>>>(ctx->d.phi[ctx->pcur], ctx->d.Q[ctx->pcur],
                                                   ctx->d.macro, N, i0 + k, raw + (long long)k * 14 * N);
        z[k] = (float)ctx->params[i0 + k].zeta;
        idx[k] = k;
    }
    float* zslot = s->at<float>(s->zeta_off) + s->cfg.max_pairs;
    SCK(s, cudaMemcpyAsync(zslot, z.data(), nb * 4, cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(s->at<int>(s->idx_off), idx.data(), nb * 4, cudaMemcpyHostToDevice, s->stream));
    k_assemble<<<blocks((long long)nb * N), EB, 0, s->stream>>>(
        raw, s->at<int>(s->idx_off), zslot, s->norm, s->zscale, N, nb,
        s->at<bf16>(s->tensors[s->x_t].act), nullptr);
    SCK(s, forward_pass(s, nb, false));
    for (int k = 0; k < nb; ++k)
        k_writeback<<<blocks(N), EB, 0, s->stream>>>(
            raw + (long long)k * 14 * N, s->at<float>(s->pred_off) + (long long)k * N * COUT, s->norm,
            ctx->nx, ctx->ny, i0 + k, ctx->d.phi[ctx->pcur], ctx->d.Q[ctx->pcur], ctx->d.f[ctx->fcur],
            ctx->d.prm, ctx->storage);
    SCK(s, cudaGetLastError());
    // (copies from pageable host memory return once the source is staged, so
    // the host vectors may go out of scope without a synchronisation)
    return TF_OK;
}

// Instance `inst` of the raw state (populations, phi, Q) from src to dst.
static int copy_instance(tf_surrogate* s, const tf_ctx* src, tf_ctx* dst, int inst) {
    const long long N = src->N;
    const size_t pb = tf_pop_bytes(src->storage);
    SCK(s, cudaMemcpyAsync(static_cast<char*>(dst->d.f[dst->fcur]) + 18 * inst * N * pb,
                           static_cast<const char*>(src->d.f[src->fcur]) + 18 * inst * N * pb,
                           18 * N * pb, cudaMemcpyDeviceToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(dst->d.phi[dst->pcur] + inst * N, src->d.phi[src->pcur] + inst * N,
                           N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(dst->d.Q[dst->pcur] + 2 * inst * N, src->d.Q[src->pcur] + 2 * inst * N,
                           2 * N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream));
    return TF_OK;
}

int tf_sur_judged_predict(tf_surrogate* s, tf_ctx* ctx, tf_ctx* shadow, int inst, double max_err_L,
                          double max_err_E, double out[4], int* fell_back) {
    if (!s || !ctx || !shadow) return TF_ERR_ARG;
    if (shadow == ctx || shadow->nx != ctx->nx || shadow->ny != ctx->ny || shadow->batch != ctx->batch ||
        shadow->storage != ctx->storage || shadow->stream != ctx->stream || inst < 0 || inst >= ctx->batch)
        return sfail(s, TF_ERR_ARG, "shadow must match the context's shape, storage and stream");
    SCK(s, tf_launch_flush(ctx));
    SCK(s, tf_launch_flush(shadow));
    int rc = copy_instance(s, ctx, shadow, inst);
    if (rc != TF_OK) return rc;
    if ((rc = tf_step(shadow, s->cfg.horizon)) != TF_OK) return sfail(s, rc, tf_last_error(shadow));
    if ((rc = tf_sur_predict(s, ctx, inst)) != TF_OK) return rc;
    const int ns = tf_n_shell(ctx);
    std::vector<double> Ep(ns), Es(ns);
    double Lp = 0.0, Ls = 0.0, tp = 0.0, ts = 0.0;
    if ((rc = tf_length_scale(ctx, inst, &Lp)) != TF_OK ||
        (rc = tf_energy_spectrum(ctx, inst, Ep.data(), ns, &tp)) != TF_OK)
        return sfail(s, rc, tf_last_error(ctx));
    if ((rc = tf_length_scale(shadow, inst, &Ls)) != TF_OK ||
        (rc = tf_energy_spectrum(shadow, inst, Es.data(), ns, &ts)) != TF_OK)
        return sfail(s, rc, tf_last_error(shadow));
    double num = 0.0, den = 0.0;
    for (int m = 0; m < ns; ++m) {
        num += std::fabs(Ep[m] - Es[m]);
        den += Es[m];
    }
    const double eL = Ls > 0.0 ? std::fabs(Lp - Ls) / Ls : 0.0;
    const double eE = den > 0.0 ? num / den : 0.0;
    const bool back = !(eL <= max_err_L && eE <= max_err_E);
    if (back) {
        SCK(s, tf_launch_flush(shadow));
        if ((rc = copy_instance(s, shadow, ctx, inst)) != TF_OK) return rc;
    }
    SCK(s, cudaStreamSynchronize(s->stream));
    if (out) {
        out[0] = eL;
        out[1] = eE;
        out[2] = Lp;
        out[3] = Ls;
    }
    if (fell_back) *fell_back = back ? 1 : 0;
    return TF_OK;
}

}  // extern "C"
