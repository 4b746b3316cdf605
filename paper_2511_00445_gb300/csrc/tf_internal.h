// Internal declarations shared by the CUDA translation units of libtwofluid.
// Not part of the public ABI (see include/twofluid.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "twofluid.h"

// NVTX range named after an entry point, open while the call runs on the
// host (it marks the call and the launches it enqueues in a profiler's
// timeline; without a tool attached to NVTX the calls do nothing).
struct TfRange {
    explicit TfRange(const char* name) { nvtxRangePushA(name); }
    ~TfRange() { nvtxRangePop(); }
    TfRange(const TfRange&) = delete;
    TfRange& operator=(const TfRange&) = delete;
};

// ---------------------------------------------------------------------------
// D2Q9 velocity set (Sec. III): rest, axes counter-clockwise from +x, then
// diagonals counter-clockwise from (+1, +1).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int d2q9_cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int d2q9_cy(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr float d2q9_w(int i) {
    return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// Exact weights in double: the stored FP32 deviations are f_i - w_i with these.
__host__ __device__ constexpr double d2q9_wd(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------
// Population storage (TF_STORE_*): the stored value is the deviation
// d_i = f_i - w_i, widened to FP32 on load and rounded to nearest on store.
// FP16 carries d_i * 2^12 (an exact scale both ways) so that deviations down
// to 1.5e-8 stay normal.  Zero bits are d_i = 0 in every mode.  load_cg reads
// through L2 only (ld.global.cg): for data other CTAs of the same launch wrote.
//
// Layout: the two fluids' deviations of one direction and site are adjacent,
// [B][9][N][2] (fluid fastest), so that a site's pull or store of direction i
// is one 8-byte (FP32) or 4-byte (16-bit) access holding the (fluid 1,
// fluid 2) pair the paired collision works on (2048^2 step against separate
// fluid planes [B][18][N]: strip kernel 292 -> 277 us, tile kernel 346 -> 315
// us).  load2 / store2 move such a
// pair (type T2) with the same per-element conversions as load / store.
// store2_stream is store2 with an evict-first (streaming) store, for a step
// whose state is larger than L2: the new populations are read only by the
// next step, so they need not displace the source rows prefetched into L2
// for this step's pulls (2048^2 strip kernel: 264.6 -> 262.9 us).
// ---------------------------------------------------------------------------
struct PopF32 {
    typedef float T;
    static constexpr int kMode = TF_STORE_F32;
    __device__ static float load(const T* p) { return *p; }
    __device__ static float load_cg(const T* p) { return __ldcg(p); }
    __device__ static void store(T* p, float d) { *p = d; }
    typedef float2 T2;   // (fluid 1, fluid 2)
    __device__ static float2 load2(const T2* p) { return *p; }
    __device__ static float2 load2_cg(const T2* p) { return __ldcg(p); }
    __device__ static void store2(T2* p, float2 d) { *p = d; }
    __device__ static void store2_stream(T2* p, float2 d) { __stcs(p, d); }
};
struct PopF16 {
    typedef __half T;
    static constexpr int kMode = TF_STORE_F16;
    __device__ static float load(const T* p) { return __fmul_rn(__half2float(*p), 0x1p-12f); }
    __device__ static float load_cg(const T* p) {
        const unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
        return __fmul_rn(__half2float(__ushort_as_half(v)), 0x1p-12f);
    }
    __device__ static void store(T* p, float d) { *p = __float2half_rn(__fmul_rn(d, 0x1p12f)); }
    __device__ static float2 widen(__half2 h) {
        return make_float2(__fmul_rn(__low2float(h), 0x1p-12f), __fmul_rn(__high2float(h), 0x1p-12f));
    }
    typedef __half2 T2;
    __device__ static float2 load2(const T2* p) { return widen(*p); }
    __device__ static float2 load2_cg(const T2* p) {
        const unsigned v = __ldcg(reinterpret_cast<const unsigned*>(p));
        return widen(*reinterpret_cast<const __half2*>(&v));
    }
    __device__ static void store2(T2* p, float2 d) {
        *p = __floats2half2_rn(__fmul_rn(d.x, 0x1p12f), __fmul_rn(d.y, 0x1p12f));
    }
    __device__ static void store2_stream(T2* p, float2 d) {
        const __half2 h = __floats2half2_rn(__fmul_rn(d.x, 0x1p12f), __fmul_rn(d.y, 0x1p12f));
        __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&h));
    }
};
struct PopBF16 {
    typedef __nv_bfloat16 T;
    static constexpr int kMode = TF_STORE_BF16;
    __device__ static float load(const T* p) { return __bfloat162float(*p); }
    __device__ static float load_cg(const T* p) {
        const unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
        return __bfloat162float(__ushort_as_bfloat16(v));
    }
    __device__ static void store(T* p, float d) { *p = __float2bfloat16_rn(d); }
    __device__ static float2 widen(__nv_bfloat162 h) { return make_float2(__low2float(h), __high2float(h)); }
    typedef __nv_bfloat162 T2;
    __device__ static float2 load2(const T2* p) { return widen(*p); }
    __device__ static float2 load2_cg(const T2* p) {
        const unsigned v = __ldcg(reinterpret_cast<const unsigned*>(p));
        return widen(*reinterpret_cast<const __nv_bfloat162*>(&v));
    }
    __device__ static void store2(T2* p, float2 d) { *p = __floats2bfloat162_rn(d.x, d.y); }
    __device__ static void store2_stream(T2* p, float2 d) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(d.x, d.y);
        __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&h));
    }
};

// Bytes per stored population element.
inline size_t tf_pop_bytes(int storage) { return storage == TF_STORE_F32 ? 4 : 2; }

// Element index of fluid fl's deviation of direction k at site `site` of
// instance b (layout [B][9][N][2]).
__host__ __device__ __forceinline__ long long pop_index(long long b, int fl, int k, long long site,
                                                        long long N) {
    return ((9 * b + k) * N + site) * 2 + fl;
}

// Run-time dispatch for kernels off the hot path (storage uniform per launch).
__device__ __forceinline__ float pop_load(const void* base, long long i, int storage) {
    if (storage == TF_STORE_F16) return PopF16::load(static_cast<const __half*>(base) + i);
    if (storage == TF_STORE_BF16) return PopBF16::load(static_cast<const __nv_bfloat16*>(base) + i);
    return PopF32::load(static_cast<const float*>(base) + i);
}
__device__ __forceinline__ void pop_store(void* base, long long i, float d, int storage) {
    if (storage == TF_STORE_F16)
        PopF16::store(static_cast<__half*>(base) + i, d);
    else if (storage == TF_STORE_BF16)
        PopBF16::store(static_cast<__nv_bfloat16*>(base) + i, d);
    else
        PopF32::store(static_cast<float*>(base) + i, d);
}

// Per-instance parameters in the form the kernels use (FP32, precomputed).
// mu(phi_ref + d) = A_ch f'(phi_ref + d) - kappa lap(d) with the cubic
// A_ch f'(c + d) = mu0 + mu1 d + mu2 d^2 + mu3 d^3 expanded about c.
struct DevParams {
    float omega1, omega2;   // 1 / tau_k
    float guo1, guo2;       // 1 - 1 / (2 tau_k)
    float gamma, zeta, lam, K;
    float GammaQ, A_Q, C_Q, M;
    float kappa, dt_fd, phi_ref, rho1;
    float mu0, mu1, mu2, mu3;
    float rho2, pad0, pad1, pad2;
};

// Device buffers carved out of the caller's workspace.
struct DevBuffers {
    void* f[2];        // populations [B][9][N][2 fluids] in the storage type (pull
                       // layout: post-collision deviations of the previous step)
    float* phi[2];     // phi - phi_ref  [B][N]
    float* Q[2];       // Q_xx, Q_xy     [B][2][N]
    float* u[2];       // u1x, u1y, u2x, u2y [B][4][N]
    float* mu;         // scratch: chemical potential [B][N]
    float* tau;        // scratch: fluid-1 stress (elastic + active) xx, xy, yx, yy [B][4][N]
    float* macro;      // scratch: u1x u1y u2x u2y rho1 rho2 (G1+G2)x (G1+G2)y [B][8][N]
    DevParams* prm;    // [B]
    double* red_part;  // reduction partials [B][red_blocks][8]
    double* red_out;   // reduction results [B][8]
    double2* cbuf[2];  // complex FFT buffers, N each
    double* shell_part;// shell histogram partials [shell_blocks][2 (n_shell + 1)]
    double* shell_out; // [n_shell]
    double* stage;     // FP64 staging plane [N] (and small results)
    float* snap;       // reference fields of the temporal correlations [B][5][N]
    int* flags;        // device status words
};

struct tf_ctx {
    int nx = 0, ny = 0, batch = 0, n_sub = 5, storage = TF_STORE_F32;
    long long N = 0;                 // nx * ny
    std::vector<tf_params> params;
    std::vector<DevParams> dparams;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    DevBuffers d{};
    int fcur = 0;                    // population buffer holding the current state
    int pcur = 0;                    // phi/Q buffer holding the current state
    int ucur = 0;                    // velocity buffer written by the last fused launch
    bool fd_pending = false;         // fused path: sub-steps of the last step not yet applied
    int tile_rows = 0;               // fused path: tile rows per instance (0: not planned yet)
    int tile_cols = 0;               // fused path: tile columns per instance
    bool wide_tiles = false;         // fused path: the wide tile geometry
    int step_kernel = TF_KERNEL_AUTO;// requested steady-state kernel (tf_set_step_kernel)
    bool use_strip = false;          // fused path: steady-state steps run the strip kernel
    int strip_cols = 0;              // strip kernel: strips per instance
    int strip_segs = 0;              // strip kernel: row segments per strip
    int64_t steps = 0;
    int64_t launches = 0;            // kernels launched by this context
    int n_shell = 0;
    std::vector<char> has_snap;      // per instance: tf_snapshot taken
    int red_blocks = 0;
    int shell_blocks = 0;
    std::string last_error;
    // Host-buffer pipeline of a batch (tf_advance_host), created on first use
    // and released by tf_destroy: one stream for uploads, one for downloads,
    // compute lanes, their events, and a private stream to capture on (the
    // context's stream may be the legacy default stream, which cannot be).
    cudaStream_t xfer_in = nullptr, xfer_out = nullptr, xfer_cap = nullptr;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> events;
    // Captured pipelines for pinned buffers, keyed by what they bake in.
    struct HostGraph {
        const void* in;
        void* out;
        int64_t n;
        int fcur, pcur, ucur;
        bool fd_pending;
        cudaGraphExec_t exec;
        int fcur_end, pcur_end, ucur_end;
        bool fd_pending_end;
        int64_t launches;
    };
    std::vector<HostGraph> host_graphs;
};

// Workspace carving (tf_api.cu).
size_t tf_layout(const tf_params& p0, int batch, DevBuffers* d, char* base);

// Precompute the kernel parameter block of one instance.
DevParams tf_make_devparams(const tf_params& p);

// ---- step kernels (tf_step.cu, tf_fused.cu) ---------------------------------
// Advance the whole batch by n steps on ctx->stream (fused path when
// available, else the per-stage kernels).
cudaError_t tf_launch_steps(tf_ctx* ctx, int64_t n);
// Apply pending sub-steps so that the buffers hold the plain state.
cudaError_t tf_launch_flush(tf_ctx* ctx);
// Per-stage kernels: forces, LBM, then n_sub separate sub-step launches.
cudaError_t tf_unfused_steps(tf_ctx* ctx, int64_t n);
// Fused kernels (tf_fused.cu): one launch per step for n_sub == 5.
bool tf_fused_supported(const tf_ctx* ctx);
cudaError_t tf_fused_steps(tf_ctx* ctx, int64_t n);
cudaError_t tf_fused_flush(tf_ctx* ctx);
cudaError_t tf_configure_fused_kernels();
// Plan (once per context, again after tf_set_step_kernel) the tile rows and
// columns of the tile kernel and the strips and segments of the strip kernel.
cudaError_t tf_plan_fused(tf_ctx* ctx);
// Whether the strip kernel can step this context (nx a multiple of 4, n_sub = 5).
bool tf_strip_supported(const tf_ctx* ctx);
// Buffer cursors of the fused path (the fields of tf_ctx of the same names).
struct FusedCursor {
    int fcur, pcur, ucur;
    bool fd_pending;
};
// Fused launches of instances [inst0, inst0 + count) only, on `stream`: n
// steps, then the pending sub-steps when `flush`.  The launches start from the
// cursors in *cur and advance them; the context's own cursors and step count
// are left alone (every instance of a context moves through the same buffers).
cudaError_t tf_fused_span(tf_ctx* ctx, int inst0, int count, int64_t n, bool flush,
                          cudaStream_t stream, FusedCursor* cur);
// One tile launch over rows [y_lo, y_hi) of instance inst only, on `stream`:
// the LBM-only pass (lbm, from a plain state) or the FD-only pass of the
// pending sub-steps (!lbm), reading and writing the buffers `cur` names.  The
// LBM-only pass loads phi, Q within 4 rows of the band (it uses 2) and pulls
// populations within 1 row; the FD-only pass loads phi, Q and u within 12.
cudaError_t tf_fused_band(tf_ctx* ctx, int inst, int y_lo, int y_hi, bool lbm, cudaStream_t stream,
                          FusedCursor cur);
// Evaluate mu, the fluid-1 stress, the Guo velocities, densities and the
// non-drag force sum of the current state into d.mu, d.tau and macro_out
// ([B][8][N]: u1x u1y u2x u2y rho1 rho2 (G1+G2)x (G1+G2)y).
cudaError_t tf_launch_macro(tf_ctx* ctx, float* macro_out);

// ---- field / observable kernels (tf_observe.cu) ---------------------------
cudaError_t tf_launch_init(tf_ctx* ctx, int inst, uint64_t seed, double phi0,
                           double dphi, double S0);
cudaError_t tf_launch_zero_state(tf_ctx* ctx);
cudaError_t tf_launch_write_field(tf_ctx* ctx, int inst, int field, const double* dsrc);
cudaError_t tf_launch_set_equilibrium(tf_ctx* ctx, int inst, const double* du1,
                                      const double* du2);
cudaError_t tf_launch_read_field(tf_ctx* ctx, int inst, int field, double* ddst);
cudaError_t tf_launch_conserved(tf_ctx* ctx, int inst, double* dout8);
cudaError_t tf_launch_phase_difference(tf_ctx* ctx, int inst, double* dout6);
cudaError_t tf_launch_phi_stats(tf_ctx* ctx, int inst, double* dout2);
// Scan the latest phi, Q and velocity planes of every instance for NaN / Inf;
// a hit records TF_ERR_NONFINITE in d.flags[0] (kept until tf_sync reads it).
cudaError_t tf_launch_nonfinite_scan(tf_ctx* ctx);
// which: 0 = structure factor of phi - <phi>, 1 = kinetic-energy spectrum of u_c.
// Writes n_shell shell sums to d.shell_out[0..n_shell-1] and the all-mode
// total to d.shell_out[n_shell].
cudaError_t tf_launch_spectrum(tf_ctx* ctx, int inst, int which);
cudaError_t tf_launch_shell_counts(tf_ctx* ctx);
// Shell-averaged spatial correlation (which = TF_CORR_*) into dout[n_shell].
cudaError_t tf_launch_correlation(tf_ctx* ctx, int inst, int which, double* dout);
// Reference fields for the temporal correlations; then the six sums
// (uu', uu, ww', ww, QQ', QQ) against the current state.
cudaError_t tf_launch_snapshot(tf_ctx* ctx, int inst);
cudaError_t tf_launch_time_correlation(tf_ctx* ctx, int inst, double* dout6);
// Plaquette charge counts (+1/2, -1/2, other) as doubles.
cudaError_t tf_launch_defects(tf_ctx* ctx, int inst, double* dout3);
// One-time kernel attributes (large dynamic shared memory).
cudaError_t tf_configure_observe_kernels();
