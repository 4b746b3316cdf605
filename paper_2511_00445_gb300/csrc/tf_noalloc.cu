// Fixed-footprint variant of the concentration statistics (tf_phi_stats) for
// callers that must not allocate device memory; declared in twofluid.h as
// tf_phi_stats_noalloc.
//
// Scratch: the per-block FP64 partials live in one file-scope device array of
// TF_NOALLOC_MAX_BLOCKS x 2 doubles (16 KiB).  Every GPU that loads the
// library holds this array until the process exits.  Host code cannot use the
// array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress on the current device (no allocation; a lookup per
// call stays valid if the application resets its device context, which can
// move the array).  Calls share the array: each call overwrites exactly the
// partials it later reads, and two calls whose kernels overlap on the GPU race.
//
// The variance is merged from per-block (mean, sum of squared deviations)
// pairs with the pairwise update of Chan, Golub and LeVeque ("Updating
// formulae and a pairwise algorithm for computing sample variances", 1979),
// so inputs whose mean is large against their spread keep their accuracy.
#include <cmath>

#include "twofluid.h"
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr long long kChunk = (long long)kThreads * kPerThread;   // elements per block
constexpr int kMaxBlocks = TF_NOALLOC_MAX_BLOCKS;

static __device__ __align__(256) double g_noalloc_partials[2 * kMaxBlocks];

__device__ __forceinline__ double block_sum(double a) {
    __shared__ double sa[kThreads / 32];
    __shared__ double total;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sa[wid] = a;
    __syncthreads();
    if (wid == 0) {
        a = lane < kThreads / 32 ? sa[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) total = a;
    }
    __syncthreads();
    const double t = total;
    __syncthreads();   // the next call may overwrite sa / total
    return t;
}

// Partial (count n, mean m, sum of squared deviations q) of a set of values.
struct Moments {
    double n, m, q;
};

// Pairwise update: the moments of the union of two disjoint sets.
__device__ __forceinline__ Moments merge(const Moments& a, const Moments& b) {
    const double n = a.n + b.n;
    if (n == 0.0) return a;
    const double d = b.m - a.m;
    return {n, a.m + d * (b.n / n), a.q + b.q + d * d * (a.n * b.n / n)};
}

__device__ __forceinline__ Moments shfl_down(const Moments& v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.n, o), __shfl_down_sync(0xffffffffu, v.m, o),
            __shfl_down_sync(0xffffffffu, v.q, o)};
}

// Block j: the mean and the sum of squared deviations of elements
// [j*kChunk, min(n, (j+1)*kChunk)), two passes over values held in registers.
__global__ void __launch_bounds__(kThreads)
k_noalloc_partial(const float* __restrict__ v, long long n, double* __restrict__ part) {
    const long long base = (long long)blockIdx.x * kChunk;
    const long long rem = n - base;
    const double cnt = (double)(rem < kChunk ? rem : kChunk);
    double x[kPerThread];
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        x[k] = i < n ? (double)v[i] : 0.0;
        s += x[k];
    }
    const double mean = block_sum(s) / cnt;
    double q = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        if (i < n) q += (x[k] - mean) * (x[k] - mean);
    }
    q = block_sum(q);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = mean;
        part[2 * blockIdx.x + 1] = q;
    }
}

// One block: merge the partials in a fixed order, then mean and deviation.
__global__ void __launch_bounds__(kThreads)
k_noalloc_finish(const double* __restrict__ part, int nblocks, long long n, double ref,
                 double* __restrict__ out) {
    __shared__ Moments sw[kThreads / 32];
    Moments acc{0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < nblocks; j += kThreads) {
        const long long rem = n - (long long)j * kChunk;
        acc = merge(acc, Moments{(double)(rem < kChunk ? rem : kChunk), part[2 * j], part[2 * j + 1]});
    }
    for (int o = 16; o > 0; o >>= 1) acc = merge(acc, shfl_down(acc, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sw[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < kThreads / 32 ? sw[lane] : Moments{0.0, 0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1) acc = merge(acc, shfl_down(acc, o));
        if (lane == 0) {
            out[0] = ref + acc.m;
            out[1] = sqrt(acc.q / acc.n);
        }
    }
}

}  // namespace

extern "C" int tf_phi_stats_noalloc(const float* d_values, long long n, double phi_ref,
                                    double* d_out, void* stream) {
    if (!d_values || !d_out || n <= 0 || !std::isfinite(phi_ref)) return TF_ERR_ARG;
    if (n > TF_NOALLOC_MAX_ELEMS) return TF_ERR_TOO_LARGE;
    void* part = nullptr;
    if (cudaGetSymbolAddress(&part, g_noalloc_partials) != cudaSuccess || !part) return TF_ERR_CUDA;
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_partial<<<nblocks, kThreads, 0, st>>>(d_values, n, static_cast<double*>(part));
    k_noalloc_finish<<<1, kThreads, 0, st>>>(static_cast<const double*>(part), nblocks, n, phi_ref,
                                             d_out);
    return cudaGetLastError() == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}
