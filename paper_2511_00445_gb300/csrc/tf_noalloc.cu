// Fixed-footprint variant of the concentration statistics (tf_phi_stats) for
// callers that must not allocate device memory; declared in twofluid.h as
// tf_phi_stats_noalloc.
//
// Scratch: the per-block FP64 partial sums live in one file-scope device
// array of TF_NOALLOC_MAX_BLOCKS x 2 doubles (16 KiB).  Every GPU that loads
// the library holds this array until the process exits.  Host code cannot use
// the array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress (with that device current) and
// caches it.  Calls share the array: each call overwrites exactly the partials
// it later reads, and two calls whose kernels overlap on the GPU race.
#include <cmath>

#include "twofluid.h"
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr long long kChunk = (long long)kThreads * kPerThread;   // elements per block
constexpr int kMaxBlocks = TF_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[2 * kMaxBlocks];

// Device address of g_noalloc_partials on each device, looked up on first use.
double* g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[kThreads / 32], sb[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        a = lane < kThreads / 32 ? sa[lane] : 0.0;
        b = lane < kThreads / 32 ? sb[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Block j sums elements [j*kChunk, min(n, (j+1)*kChunk)) and their squares.
__global__ void __launch_bounds__(kThreads)
k_noalloc_partial(const float* __restrict__ v, long long n, double* __restrict__ part) {
    const long long base = (long long)blockIdx.x * kChunk;
    double s = 0.0, s2 = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        if (i < n) {
            const double x = v[i];
            s += x;
            s2 += x * x;
        }
    }
    block_sum2(s, s2);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = s2;
    }
}

// One block: sum the partials in a fixed order, then mean and deviation.
__global__ void __launch_bounds__(kThreads)
k_noalloc_finish(const double* __restrict__ part, int nblocks, long long n, double ref,
                 double* __restrict__ out) {
    double s = 0.0, s2 = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += kThreads) {
        s += part[2 * j];
        s2 += part[2 * j + 1];
    }
    block_sum2(s, s2);
    if (threadIdx.x == 0) {
        const double m = s / (double)n;
        const double var = s2 / (double)n - m * m;
        out[0] = ref + m;
        out[1] = sqrt(var > 0.0 ? var : 0.0);
    }
}

int partials_on_current_device(double** addr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TF_ERR_ARG;
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return TF_ERR_CUDA;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *addr = g_partials_addr[dev];
    return TF_OK;
}

}  // namespace

extern "C" int tf_phi_stats_noalloc(const float* d_values, long long n, double phi_ref,
                                    double* d_out, void* stream) {
    if (!d_values || !d_out || n <= 0 || !std::isfinite(phi_ref)) return TF_ERR_ARG;
    if (n > TF_NOALLOC_MAX_ELEMS) return TF_ERR_TOO_LARGE;
    double* part = nullptr;
    const int rc = partials_on_current_device(&part);
    if (rc != TF_OK) return rc;
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_partial<<<nblocks, kThreads, 0, st>>>(d_values, n, part);
    k_noalloc_finish<<<1, kThreads, 0, st>>>(part, nblocks, n, phi_ref, d_out);
    return cudaGetLastError() == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}
