// C ABI of libtwofluid (declared in include/twofluid.h): argument checks,
// workspace carving, host <-> device staging and checkpoint I/O.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tf_internal.h"
#include "tf_fused.cuh"   // tile geometry constants and tile_col of the fused kernel

// Tile planning of the fused per-context kernel (defined in tf_fused.cu).
bool wide_for(int nx, int ny, int batch, long long slots);
int tile_rows_for(int ntx, int ny, int tym, int batch, long long slots);

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxDim = 32768;
constexpr int kMaxFFT = 8192;
constexpr uint64_t kMagic = 0x31444C4655464F57ull;  // checkpoint tag
constexpr int kVersion = 2;   // 2: tf_params gained dt and check_every

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

int fail(tf_ctx* ctx, int code, const char* msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

int fail_cuda(tf_ctx* ctx, const char* where, cudaError_t e) {
    if (ctx) {
        ctx->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return TF_ERR_CUDA;
}

#define TF_CK(ctx, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fail_cuda(ctx, #call, e_); \
    } while (0)

const char* check_params(const tf_params& p) {
    if (p.nx < 1 || p.ny < 1 || p.nx > kMaxDim || p.ny > kMaxDim) return "nx, ny must be in [1, 32768]";
    if (p.n_sub < 1 || p.n_sub > 64) return "n_sub must be in [1, 64]";
    if (p.storage != TF_STORE_F32 && p.storage != TF_STORE_F16 && p.storage != TF_STORE_BF16)
        return "storage must be TF_STORE_F32, TF_STORE_F16 or TF_STORE_BF16";
    if (!(p.tau1 > 0.5) || !(p.tau2 > 0.5)) return "tau1, tau2 must exceed 1/2";
    if (!(p.rho1 > 0) || !(p.rho2 > 0)) return "rho1, rho2 must be positive";
    const double v[] = {p.gamma, p.zeta, p.lambda, p.K, p.Gamma_Q, p.A_Q,
                        p.C_Q,   p.M,    p.A_ch,   p.kappa, p.phi_ref};
    for (double x : v)
        if (!std::isfinite(x)) return "parameters must be finite";
    if (!(p.dt > 0) || !std::isfinite(p.dt)) return "dt must be positive and finite (1 for lattice units)";
    if (p.check_every < 0) return "check_every must be >= 0";
    return nullptr;
}

bool valid_inst(const tf_ctx* ctx, int inst) { return inst >= 0 && inst < ctx->batch; }

bool is_pop_field(int field) {
    return (field >= TF_FIELD_F1 && field < TF_FIELD_F1 + 9) ||
           (field >= TF_FIELD_F2 && field < TF_FIELD_F2 + 9);
}

int red_blocks_for(long long N) {
    long long b = (N + 2047) / 2048;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

int shell_blocks_for(long long N) {
    long long b = (N + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 296) b = 296;
    return (int)b;
}

}  // namespace

DevParams tf_make_devparams(const tf_params& p) {
    DevParams d{};
    d.omega1 = (float)(1.0 / p.tau1);
    d.omega2 = (float)(1.0 / p.tau2);
    d.guo1 = (float)(1.0 - 0.5 / p.tau1);
    d.guo2 = (float)(1.0 - 0.5 / p.tau2);
    d.gamma = (float)p.gamma;
    d.zeta = (float)p.zeta;
    d.lam = (float)p.lambda;
    d.K = (float)p.K;
    d.GammaQ = (float)p.Gamma_Q;
    d.A_Q = (float)p.A_Q;
    d.C_Q = (float)p.C_Q;
    d.M = (float)p.M;
    d.kappa = (float)p.kappa;
    d.dt_fd = (float)(p.dt / p.n_sub);
    d.phi_ref = (float)p.phi_ref;
    d.rho1 = (float)p.rho1;
    d.rho2 = (float)p.rho2;
    // A_ch f'(c + d) with f'(x) = 2x - 6x^2 + 4x^3, Taylor-expanded about c
    // (exact: f' is a cubic).
    const double c = (double)d.phi_ref;
    d.mu0 = (float)(p.A_ch * (2 * c - 6 * c * c + 4 * c * c * c));
    d.mu1 = (float)(p.A_ch * (2 - 12 * c + 12 * c * c));
    d.mu2 = (float)(p.A_ch * (-6 + 12 * c));
    d.mu3 = (float)(p.A_ch * 4);
    return d;
}

size_t tf_layout(const tf_params& p0, int batch, DevBuffers* d, char* base) {
    const size_t N = (size_t)p0.nx * (size_t)p0.ny, B = (size_t)batch;
    const int n_shell = (p0.nx < p0.ny ? p0.nx : p0.ny) / 2 + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off = align_up(off + bytes);
        return p;
    };
    DevBuffers t{};
    for (int k = 0; k < 2; ++k) t.f[k] = take(18 * B * N * tf_pop_bytes(p0.storage));
    for (int k = 0; k < 2; ++k) t.phi[k] = (float*)take(B * N * sizeof(float));
    for (int k = 0; k < 2; ++k) t.Q[k] = (float*)take(2 * B * N * sizeof(float));
    for (int k = 0; k < 2; ++k) t.u[k] = (float*)take(4 * B * N * sizeof(float));
    t.mu = (float*)take(B * N * sizeof(float));
    t.tau = (float*)take(4 * B * N * sizeof(float));
    t.macro = (float*)take(8 * B * N * sizeof(float));
    t.prm = (DevParams*)take(B * sizeof(DevParams));
    t.red_part = (double*)take((size_t)red_blocks_for((long long)N) * 8 * sizeof(double));
    t.red_out = (double*)take(16 * sizeof(double));
    for (int k = 0; k < 2; ++k) t.cbuf[k] = (double2*)take(N * sizeof(double2));
    t.shell_part =
        (double*)take((size_t)shell_blocks_for((long long)N) * 2 * (n_shell + 1) * sizeof(double));
    t.shell_out = (double*)take((size_t)(n_shell + 1) * sizeof(double));
    t.stage = (double*)take(N * sizeof(double));
    t.snap = (float*)take(5 * B * N * sizeof(float));
    t.flags = (int*)take(64 * sizeof(int));
    if (d) *d = t;
    return off;
}

extern "C" {

size_t tf_workspace_bytes(const tf_params* params, int batch) {
    if (!params || batch < 1) return 0;
    for (int b = 0; b < batch; ++b) {
        if (check_params(params[b])) return 0;
        if (params[b].nx != params[0].nx || params[b].ny != params[0].ny ||
            params[b].n_sub != params[0].n_sub || params[b].storage != params[0].storage)
            return 0;
    }
    return tf_layout(params[0], batch, nullptr, nullptr);
}

int tf_create(const tf_params* params, int batch, void* d_workspace, size_t workspace_bytes,
              void* stream, tf_ctx** out) {
    if (!out) return TF_ERR_ARG;
    *out = nullptr;
    if (!params || batch < 1) return TF_ERR_ARG;
    for (int b = 0; b < batch; ++b)
        if (check_params(params[b])) return TF_ERR_ARG;
    const size_t need = tf_workspace_bytes(params, batch);
    if (need == 0) return TF_ERR_ARG;
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0 || workspace_bytes < need)
        return TF_ERR_WORKSPACE;
    tf_ctx* ctx = new (std::nothrow) tf_ctx();
    if (!ctx) return TF_ERR_ARG;
    ctx->nx = params[0].nx;
    ctx->ny = params[0].ny;
    ctx->batch = batch;
    ctx->n_sub = params[0].n_sub;
    ctx->storage = params[0].storage;
    ctx->N = (long long)ctx->nx * ctx->ny;
    ctx->params.assign(params, params + batch);
    ctx->has_snap.assign(batch, 0);
    for (int b = 0; b < batch; ++b) ctx->dparams.push_back(tf_make_devparams(params[b]));
    ctx->stream = (cudaStream_t)stream;
    ctx->ws = (char*)d_workspace;
    ctx->ws_bytes = workspace_bytes;
    tf_layout(params[0], batch, &ctx->d, ctx->ws);
    ctx->n_shell = (ctx->nx < ctx->ny ? ctx->nx : ctx->ny) / 2 + 1;
    ctx->red_blocks = red_blocks_for(ctx->N);
    ctx->shell_blocks = shell_blocks_for(ctx->N);
    cudaError_t e = tf_configure_observe_kernels();
    if (e == cudaSuccess) e = tf_configure_fused_kernels();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d.prm, ctx->dparams.data(), batch * sizeof(DevParams),
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = tf_launch_zero_state(ctx);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d.flags, 0, 64 * sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        delete ctx;
        return TF_ERR_CUDA;
    }
    *out = ctx;
    return TF_OK;
}

// Streams and events of the host-buffer pipeline (see advance_pipelined).
static void release_pipeline(tf_ctx* ctx) {
    for (auto& g : ctx->host_graphs) cudaGraphExecDestroy(g.exec);
    ctx->host_graphs.clear();
    for (cudaStream_t s : ctx->lanes) cudaStreamSynchronize(s);
    if (ctx->xfer_in) cudaStreamSynchronize(ctx->xfer_in);
    if (ctx->xfer_out) cudaStreamSynchronize(ctx->xfer_out);
    for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
    for (cudaStream_t s : ctx->lanes) cudaStreamDestroy(s);
    if (ctx->xfer_in) cudaStreamDestroy(ctx->xfer_in);
    if (ctx->xfer_out) cudaStreamDestroy(ctx->xfer_out);
    if (ctx->xfer_cap) cudaStreamDestroy(ctx->xfer_cap);
    ctx->events.clear();
    ctx->lanes.clear();
    ctx->xfer_in = ctx->xfer_out = ctx->xfer_cap = nullptr;
}

int tf_destroy(tf_ctx* ctx) {
    if (!ctx) return TF_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    release_pipeline(ctx);
    delete ctx;
    return e == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

const char* tf_last_error(const tf_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

int tf_init_fields(tf_ctx* ctx, int inst, uint64_t seed, double phi0, double dphi, double S0) {
    if (!ctx) return TF_ERR_ARG;
    if (inst != -1 && !valid_inst(ctx, inst)) return fail(ctx, TF_ERR_ARG, "bad instance index");
    if (!std::isfinite(phi0) || !std::isfinite(dphi) || !std::isfinite(S0))
        return fail(ctx, TF_ERR_ARG, "non-finite initial-condition parameter");
    if (inst != -1) TF_CK(ctx, tf_launch_flush(ctx));  // other instances keep their state
    ctx->fd_pending = false;
    TF_CK(ctx, tf_launch_init(ctx, inst, seed, phi0, dphi, S0));
    ctx->steps = 0;
    return TF_OK;
}

int tf_write_field(tf_ctx* ctx, int inst, int field, const double* host) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !host) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    if (!(field == TF_FIELD_PHI || field == TF_FIELD_QXX || field == TF_FIELD_QXY ||
          is_pop_field(field)))
        return fail(ctx, TF_ERR_ARG, "field is not writable");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, cudaMemcpyAsync(ctx->d.stage, host, ctx->N * sizeof(double),
                               cudaMemcpyHostToDevice, ctx->stream));
    TF_CK(ctx, tf_launch_write_field(ctx, inst, field, ctx->d.stage));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_set_equilibrium(tf_ctx* ctx, int inst, const double* u1, const double* u2) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst)) return fail(ctx, TF_ERR_ARG, "bad instance index");
    TF_CK(ctx, tf_launch_flush(ctx));
    double* d1 = nullptr;
    double* d2 = nullptr;
    if (u1) {
        d1 = (double*)ctx->d.cbuf[0];
        TF_CK(ctx, cudaMemcpyAsync(d1, u1, 2 * ctx->N * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
    }
    if (u2) {
        d2 = (double*)ctx->d.cbuf[1];
        TF_CK(ctx, cudaMemcpyAsync(d2, u2, 2 * ctx->N * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
    }
    TF_CK(ctx, tf_launch_set_equilibrium(ctx, inst, d1, d2));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_read_field(tf_ctx* ctx, int inst, int field, double* host) {
    const TfRange nvtx_range("tf_read_field");
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !host) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    if (!((field >= TF_FIELD_PHI && field <= TF_FIELD_OMEGA_C) || is_pop_field(field)))
        return fail(ctx, TF_ERR_ARG, "unknown field id");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_read_field(ctx, inst, field, ctx->d.stage));
    TF_CK(ctx, cudaMemcpyAsync(host, ctx->d.stage, ctx->N * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_step(tf_ctx* ctx, int64_t n) {
    const TfRange nvtx_range("tf_step");
    if (!ctx) return TF_ERR_ARG;
    if (n < 0) return fail(ctx, TF_ERR_ARG, "negative step count");
    if (n == 0) return TF_OK;
    const int64_t k = ctx->params[0].check_every;
    if (k <= 0) {
        TF_CK(ctx, tf_launch_steps(ctx, n));
        return TF_OK;
    }
    // Steps in chunks that end on multiples of k (of the step count), each
    // followed by the non-finite scan.
    while (n > 0) {
        const int64_t to_next = k - ctx->steps % k;
        const int64_t m = n < to_next ? n : to_next;
        TF_CK(ctx, tf_launch_steps(ctx, m));
        n -= m;
        if (ctx->steps % k == 0) TF_CK(ctx, tf_launch_nonfinite_scan(ctx));
    }
    return TF_OK;
}

int tf_set_step_kernel(tf_ctx* ctx, int kind) {
    if (!ctx) return TF_ERR_ARG;
    if (kind != TF_KERNEL_AUTO && kind != TF_KERNEL_TILE && kind != TF_KERNEL_STRIP)
        return fail(ctx, TF_ERR_ARG, "unknown step kernel");
    if (kind == TF_KERNEL_STRIP && !tf_strip_supported(ctx))
        return fail(ctx, TF_ERR_ARG, "the strip kernel needs n_sub = 5 and nx a multiple of 4");
    ctx->step_kernel = kind;
    // captured host-buffer pipelines bake in the kernel: drop them
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& g : ctx->host_graphs) cudaGraphExecDestroy(g.exec);
    ctx->host_graphs.clear();
    TF_CK(ctx, tf_plan_fused(ctx));
    return TF_OK;
}

int tf_step_kernel(tf_ctx* ctx) {
    if (!ctx) return TF_ERR_ARG;
    if (!tf_fused_supported(ctx)) return TF_KERNEL_TILE;
    if (ctx->tile_rows <= 0) TF_CK(ctx, tf_plan_fused(ctx));
    return ctx->use_strip ? TF_KERNEL_STRIP : TF_KERNEL_TILE;
}

int tf_sync(tf_ctx* ctx) {
    if (!ctx) return TF_ERR_ARG;
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    TF_CK(ctx, cudaGetLastError());
    // Device status word: a kernel that gave up a bounded wait wrote a code.
    int flag = 0;
    TF_CK(ctx, cudaMemcpyAsync(&flag, ctx->d.flags, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag != 0) {
        TF_CK(ctx, cudaMemsetAsync(ctx->d.flags, 0, sizeof(int), ctx->stream));
        TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
        return fail(ctx, flag, flag == TF_ERR_NONFINITE
                                   ? "the check_every scan found NaN or Inf in the state"
                                   : flag == TF_ERR_BOUNDS
                                         ? "an index check of the bounds-check build failed"
                                         : "a device-side bounded wait timed out");
    }
    return TF_OK;
}

int64_t tf_step_count(const tf_ctx* ctx) { return ctx ? ctx->steps : -1; }

int64_t tf_kernel_launches(const tf_ctx* ctx) { return ctx ? ctx->launches : -1; }

int tf_conserved(tf_ctx* ctx, int inst, double out[TF_NCONS]) {
    const TfRange nvtx_range("tf_conserved");
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !out) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_conserved(ctx, inst, ctx->d.red_out));
    TF_CK(ctx, cudaMemcpyAsync(out, ctx->d.red_out, TF_NCONS * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const tf_params& p = ctx->params[inst];
    out[0] += (double)(float)p.phi_ref * (double)ctx->N;   // stored deviations -> phi
    out[1] += (double)ctx->N;                                // deviations -> rho
    out[2] += (double)ctx->N;
    if (out[7] > 0) return fail(ctx, TF_ERR_NONFINITE, "non-finite values in the state");
    return TF_OK;
}

int tf_n_shell(const tf_ctx* ctx) { return ctx ? ctx->n_shell : 0; }

static int spectrum_common(tf_ctx* ctx, int inst, int which, double* out, int n_shell,
                           double* total) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst)) return fail(ctx, TF_ERR_ARG, "bad instance index");
    if (out && n_shell != ctx->n_shell) return fail(ctx, TF_ERR_ARG, "n_shell mismatch");
    if (ctx->nx > kMaxFFT || ctx->ny > kMaxFFT)
        return fail(ctx, TF_ERR_ARG, "spectra support nx, ny <= 8192");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_spectrum(ctx, inst, which));
    std::vector<double> buf(ctx->n_shell + 1);
    TF_CK(ctx, cudaMemcpyAsync(buf.data(), ctx->d.shell_out, buf.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (out) std::memcpy(out, buf.data(), ctx->n_shell * sizeof(double));
    if (total) *total = buf[ctx->n_shell];
    return TF_OK;
}

int tf_shell_counts(tf_ctx* ctx, double* out, int n_shell) {
    if (!ctx) return TF_ERR_ARG;
    if (!out || n_shell != ctx->n_shell) return fail(ctx, TF_ERR_ARG, "n_shell mismatch");
    TF_CK(ctx, tf_launch_shell_counts(ctx));
    TF_CK(ctx, cudaMemcpyAsync(out, ctx->d.shell_out, n_shell * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_structure_factor(tf_ctx* ctx, int inst, double* S, int n_shell) {
    const TfRange nvtx_range("tf_structure_factor");
    if (!S) return ctx ? fail(ctx, TF_ERR_ARG, "null array") : TF_ERR_ARG;
    return spectrum_common(ctx, inst, 0, S, n_shell, nullptr);
}

int tf_length_scale(tf_ctx* ctx, int inst, double* L) {
    const TfRange nvtx_range("tf_length_scale");
    if (!ctx) return TF_ERR_ARG;
    if (!L) return fail(ctx, TF_ERR_ARG, "null pointer");
    std::vector<double> S(ctx->n_shell);
    int rc = spectrum_common(ctx, inst, 0, S.data(), ctx->n_shell, nullptr);
    if (rc != TF_OK) return rc;
    const double k0 = 2.0 * M_PI / (double)(ctx->nx < ctx->ny ? ctx->nx : ctx->ny);
    double num = 0.0, den = 0.0;
    for (int m = 1; m < ctx->n_shell; ++m) {
        num += 0.5 * S[m];
        den += (double)m * k0 * 0.5 * S[m];
    }
    *L = den > 0.0 ? num / den : 0.0;
    return TF_OK;
}

int tf_energy_spectrum(tf_ctx* ctx, int inst, double* E, int n_shell, double* E_total) {
    const TfRange nvtx_range("tf_energy_spectrum");
    if (!E && !E_total) return ctx ? fail(ctx, TF_ERR_ARG, "null arrays") : TF_ERR_ARG;
    return spectrum_common(ctx, inst, 1, E, n_shell, E_total);
}

int tf_phase_difference(tf_ctx* ctx, int inst, double out[6]) {
    const TfRange nvtx_range("tf_phase_difference");
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !out) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_phase_difference(ctx, inst, ctx->d.red_out));
    double s[6];
    TF_CK(ctx, cudaMemcpyAsync(s, ctx->d.red_out, 6 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 6; ++k) out[k] = std::sqrt(s[k] / (double)ctx->N);
    return TF_OK;
}

int tf_phi_stats(tf_ctx* ctx, int inst, double* mean, double* stddev) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst)) return fail(ctx, TF_ERR_ARG, "bad instance index");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_phi_stats(ctx, inst, ctx->d.red_out));
    double s[2];
    TF_CK(ctx, cudaMemcpyAsync(s, ctx->d.red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const double md = s[0] / (double)ctx->N;   // mean of the stored deviation
    const double var = s[1] / (double)ctx->N - md * md;
    if (mean) *mean = (double)(float)ctx->params[inst].phi_ref + md;
    if (stddev) *stddev = std::sqrt(var > 0 ? var : 0.0);
    return TF_OK;
}

int tf_correlation(tf_ctx* ctx, int inst, int which, double* C, int n_shell) {
    const TfRange nvtx_range("tf_correlation");
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !C) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    if (which < TF_CORR_U || which > TF_CORR_Q) return fail(ctx, TF_ERR_ARG, "unknown correlation");
    if (n_shell != ctx->n_shell) return fail(ctx, TF_ERR_ARG, "n_shell must equal tf_n_shell()");
    if (ctx->nx > kMaxFFT || ctx->ny > kMaxFFT)
        return fail(ctx, TF_ERR_ARG, "correlations need nx, ny <= 8192");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_correlation(ctx, inst, which, ctx->d.shell_out));
    TF_CK(ctx, cudaMemcpyAsync(C, ctx->d.shell_out, n_shell * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_snapshot(tf_ctx* ctx, int inst) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst)) return fail(ctx, TF_ERR_ARG, "bad instance index");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_snapshot(ctx, inst));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->has_snap[inst] = 1;
    return TF_OK;
}

int tf_time_correlation(tf_ctx* ctx, int inst, double out[3]) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !out) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    if (!ctx->has_snap[inst]) return fail(ctx, TF_ERR_ARG, "no snapshot for this instance");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_time_correlation(ctx, inst, ctx->d.red_out));
    double s[6];
    TF_CK(ctx, cudaMemcpyAsync(s, ctx->d.red_out, 6 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 3; ++k) out[k] = s[2 * k + 1] != 0.0 ? s[2 * k] / s[2 * k + 1] : 0.0;
    return TF_OK;
}

int tf_defects(tf_ctx* ctx, int inst, int64_t out[3]) {
    const TfRange nvtx_range("tf_defects");
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || !out) return fail(ctx, TF_ERR_ARG, "bad instance or null array");
    TF_CK(ctx, tf_launch_flush(ctx));
    TF_CK(ctx, tf_launch_defects(ctx, inst, ctx->d.red_out));
    double s[3];
    TF_CK(ctx, cudaMemcpyAsync(s, ctx->d.red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 3; ++k) out[k] = (int64_t)s[k];   // exact: counts far below 2^53
    return TF_OK;
}

int tf_reynolds(tf_ctx* ctx, int inst, double* Re, double* L_a) {
    if (!ctx) return TF_ERR_ARG;
    if (!valid_inst(ctx, inst) || (!Re && !L_a)) return fail(ctx, TF_ERR_ARG, "bad instance or null pointers");
    double ph[6];
    const int rc = tf_phase_difference(ctx, inst, ph);
    if (rc != TF_OK) return rc;
    const tf_params& p = ctx->params[inst];
    const double La = p.zeta != 0.0 ? std::sqrt(p.K / std::fabs(p.zeta)) : HUGE_VAL;
    const double eta = p.rho1 * (p.tau1 - 0.5) / 3.0 + p.rho2 * (p.tau2 - 0.5) / 3.0;
    if (L_a) *L_a = La;
    if (Re) *Re = p.zeta != 0.0 ? (p.rho1 + p.rho2) * ph[3] * La / eta : HUGE_VAL;
    return TF_OK;
}

size_t tf_state_bytes(const tf_ctx* ctx) {
    if (!ctx) return 0;
    const size_t N = (size_t)ctx->N, B = (size_t)ctx->batch;
    return 18 * B * N * tf_pop_bytes(ctx->storage) + (1 + 2) * B * N * sizeof(float);
}

// Raw state blob: populations [B][9][N][2] (storage type), phi [B][N], Q [B][2][N] (FP32).
static int copy_state(tf_ctx* ctx, void* host, bool to_host) {
    const size_t N = (size_t)ctx->N, B = (size_t)ctx->batch;
    char* h = (char*)host;
    const size_t sf = 18 * B * N * tf_pop_bytes(ctx->storage), sp = B * N * sizeof(float),
                 sq = 2 * B * N * sizeof(float);
    void* dev[3] = {ctx->d.f[ctx->fcur], ctx->d.phi[ctx->pcur], ctx->d.Q[ctx->pcur]};
    const size_t sz[3] = {sf, sp, sq};
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
        if (to_host) {
            TF_CK(ctx, cudaMemcpyAsync(h + off, dev[k], sz[k], cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            TF_CK(ctx, cudaMemcpyAsync(dev[k], h + off, sz[k], cudaMemcpyHostToDevice, ctx->stream));
        }
        off += sz[k];
    }
    return TF_OK;
}

// Compute lanes of the pipeline: instances are dealt to them in turn, so that
// the steps of several instances can run at once when they outlast the copies.
constexpr int kLanes = 4;
// Row bands of a single instance's host-buffer advance (enqueue_banded):
// bands of about kBandRows rows, at most kMaxBands, at least 3 (and so at
// least kBandRows >= 12 rows, the reach of the FD-only pass).  More bands
// shorten the pipeline's head and tail (2048^2, one step: 981 MLUPS without
// bands, 1443 with 16 bands of 128 rows).
constexpr int kBandRows = 64;
constexpr int kMaxBands = 32;

static int bands_for(const tf_ctx* ctx) {
    const int k = ctx->ny / kBandRows;
    return k < 3 ? 0 : (k > kMaxBands ? kMaxBands : k);
}

static cudaError_t make_pipeline(tf_ctx* ctx) {
    if (ctx->xfer_in) return cudaSuccess;
    const int lanes = ctx->batch < kLanes ? ctx->batch : kLanes;
    const int per_instance = 2 * ctx->batch + lanes + 3, banded = 3 * kMaxBands + 4;
    const int events = per_instance > banded ? per_instance : banded;
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->xfer_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->xfer_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->xfer_cap, cudaStreamNonBlocking);
    for (int k = 0; k < lanes && e == cudaSuccess; ++k) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) ctx->lanes.push_back(s);
    }
    for (int k = 0; k < events && e == cudaSuccess; ++k) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->events.push_back(ev);
    }
    if (e != cudaSuccess) release_pipeline(ctx);
    return e;
}

#define PCK(x)                                  \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

// Host-buffer advance of a batch on the fused path, pipelined per instance.
// Instance b's upload, steps and download are queued on their own, so the
// upload of instance b + 1 and the download of instance b - 1 overlap the
// steps of instance b.  Uploads queue on one stream and downloads on another,
// both in instance order, so each instance's copies get the whole bandwidth of
// their direction; the steps of instance b run on lane b mod kLanes once its
// upload is done.  All side streams fork from and join back to `origin`.
// Every instance moves through the same buffer cursors, so the cursors
// afterwards (*end) are those of any one instance.  The raw state is
// [f: B x 9 x N x 2][phi: B x N][Q: B x 2 x N] on both sides, so an instance is
// three contiguous pieces.
static cudaError_t enqueue_pipeline(tf_ctx* ctx, cudaStream_t origin, const void* h_in, int64_t n,
                                    void* h_out, FusedCursor* end) {
    const size_t N = (size_t)ctx->N, B = (size_t)ctx->batch;
    const size_t pf = 18 * N * tf_pop_bytes(ctx->storage), pp = N * sizeof(float), pq = 2 * pp;
    const size_t off[3] = {0, B * pf, B * pf + B * pp}, len[3] = {pf, pp, pq};
    const int L = (int)ctx->lanes.size();
    cudaEvent_t* ev_in = ctx->events.data();               // [B]
    cudaEvent_t* ev_done = ev_in + B;                     // [B]
    cudaEvent_t* ev_join = ev_done + B;                   // [L + 2]
    cudaEvent_t ev_fork = ev_join[L + 2];
    PCK(cudaEventRecord(ev_fork, origin));
    PCK(cudaStreamWaitEvent(ctx->xfer_in, ev_fork, 0));
    PCK(cudaStreamWaitEvent(ctx->xfer_out, ev_fork, 0));
    for (int k = 0; k < L; ++k) PCK(cudaStreamWaitEvent(ctx->lanes[k], ev_fork, 0));
    const FusedCursor start{ctx->fcur, ctx->pcur, ctx->ucur, h_in ? false : ctx->fd_pending};
    *end = start;
    for (size_t b = 0; b < B; ++b) {
        cudaStream_t lane = ctx->lanes[b % L];
        if (h_in) {
            char* dev[3] = {(char*)ctx->d.f[start.fcur], (char*)ctx->d.phi[start.pcur],
                            (char*)ctx->d.Q[start.pcur]};
            for (int k = 0; k < 3; ++k)
                PCK(cudaMemcpyAsync(dev[k] + b * len[k], (const char*)h_in + off[k] + b * len[k], len[k],
                                    cudaMemcpyHostToDevice, ctx->xfer_in));
            PCK(cudaEventRecord(ev_in[b], ctx->xfer_in));
            PCK(cudaStreamWaitEvent(lane, ev_in[b], 0));
        }
        FusedCursor cur = start;
        PCK(tf_fused_span(ctx, (int)b, 1, n, h_out != nullptr, lane, &cur));
        *end = cur;
        if (h_out) {
            PCK(cudaEventRecord(ev_done[b], lane));
            PCK(cudaStreamWaitEvent(ctx->xfer_out, ev_done[b], 0));
            const char* dev[3] = {(const char*)ctx->d.f[cur.fcur], (const char*)ctx->d.phi[cur.pcur],
                                  (const char*)ctx->d.Q[cur.pcur]};
            for (int k = 0; k < 3; ++k)
                PCK(cudaMemcpyAsync((char*)h_out + off[k] + b * len[k], dev[k] + b * len[k], len[k],
                                    cudaMemcpyDeviceToHost, ctx->xfer_out));
        }
    }
    for (int k = 0; k < L; ++k) {
        PCK(cudaEventRecord(ev_join[k], ctx->lanes[k]));
        PCK(cudaStreamWaitEvent(origin, ev_join[k], 0));
    }
    PCK(cudaEventRecord(ev_join[L], ctx->xfer_out));
    PCK(cudaStreamWaitEvent(origin, ev_join[L], 0));
    PCK(cudaEventRecord(ev_join[L + 1], ctx->xfer_in));
    PCK(cudaStreamWaitEvent(origin, ev_join[L + 1], 0));
    return cudaSuccess;
}

// Host-buffer advance of a single instance in row bands, so that its upload,
// steps and download overlap.  From the uploaded plain state, band k's
// LBM-only pass needs the uploads of bands k - 1 .. k + 1 (it reads within
// 4 rows), its FD-only pass the LBM-only passes of bands k - 1 .. k + 1 (it
// reads within 12), and its download its FD-only pass.  Uploads go in the
// order K - 1, 0, 1, .., K - 2 on one stream, downloads on another, and the
// passes in order on one compute lane; with one step, the FD-only pass of
// band k - 1 follows the LBM-only pass of band k, and those of bands K - 1
// and 0 (which need the last LBM-only pass) come last.  With more steps the
// middle ones are whole-grid launches between the two banded passes.  Each
// band of the raw state is three strided pieces (9 population planes of fluid
// pairs, phi, 2 Q planes), one 2D copy each.
static cudaError_t enqueue_banded(tf_ctx* ctx, cudaStream_t origin, const void* h_in, int64_t n,
                                  void* h_out, FusedCursor* end) {
    const int K = bands_for(ctx);
    const size_t N = (size_t)ctx->N, nx = (size_t)ctx->nx, es = tf_pop_bytes(ctx->storage);
    cudaEvent_t* ev_in = ctx->events.data();   // [K]
    cudaEvent_t* ev_fd = ev_in + K;            // [K]: FD-only pass of band k done
    cudaEvent_t ev_fork = ev_in[2 * K];
    cudaEvent_t* ev_join = ev_in + 2 * K + 1;  // [3]
    cudaStream_t lane = ctx->lanes[0];
    PCK(cudaEventRecord(ev_fork, origin));
    PCK(cudaStreamWaitEvent(ctx->xfer_in, ev_fork, 0));
    PCK(cudaStreamWaitEvent(ctx->xfer_out, ev_fork, 0));
    PCK(cudaStreamWaitEvent(lane, ev_fork, 0));
    auto y_of = [&](int k) { return (int)((long long)k * ctx->ny / K); };
    auto copy_band = [&](int k, bool down, const FusedCursor& c) -> cudaError_t {
        const size_t r0 = (size_t)y_of(k), rows = (size_t)y_of(k + 1) - r0;
        char* host = down ? static_cast<char*>(h_out) : static_cast<char*>(const_cast<void*>(h_in));
        char* dev[3] = {(char*)ctx->d.f[c.fcur], (char*)ctx->d.phi[c.pcur], (char*)ctx->d.Q[c.pcur]};
        // populations: 9 direction planes of N fluid pairs
        const size_t elem[3] = {2 * es, sizeof(float), sizeof(float)}, planes[3] = {9, 1, 2};
        const size_t hoff[3] = {0, 18 * N * es, 18 * N * es + N * sizeof(float)};
        for (int q = 0; q < 3; ++q) {
            const size_t pitch = N * elem[q], off = r0 * nx * elem[q], w = rows * nx * elem[q];
            const cudaError_t e =
                down ? cudaMemcpy2DAsync(host + hoff[q] + off, pitch, dev[q] + off, pitch, w, planes[q],
                                         cudaMemcpyDeviceToHost, ctx->xfer_out)
                     : cudaMemcpy2DAsync(dev[q] + off, pitch, host + hoff[q] + off, pitch, w, planes[q],
                                         cudaMemcpyHostToDevice, ctx->xfer_in);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const FusedCursor start{ctx->fcur, ctx->pcur, ctx->ucur, false};
    for (int j = 0; j < K; ++j) {                 // uploads: K - 1, 0, 1, .., K - 2
        const int k = (j + K - 1) % K;
        PCK(copy_band(k, false, start));
        PCK(cudaEventRecord(ev_in[k], ctx->xfer_in));
    }
    // cursors after the LBM-only pass, after the n - 1 whole-grid steps, and at the end
    const FusedCursor lbm{start.fcur ^ 1, start.pcur, start.ucur ^ 1, true};
    FusedCursor mid = lbm;
    auto fd_band = [&](int k) -> cudaError_t {
        PCK(tf_fused_band(ctx, 0, y_of(k), y_of(k + 1), false, lane, mid));
        PCK(cudaEventRecord(ev_fd[k], lane));
        PCK(cudaStreamWaitEvent(ctx->xfer_out, ev_fd[k], 0));
        const FusedCursor fin{mid.fcur, mid.pcur ^ 1, mid.ucur, false};
        return copy_band(k, true, fin);
    };
    for (int k = 0; k < K; ++k) {
        for (int d = -1; d <= 1; ++d) PCK(cudaStreamWaitEvent(lane, ev_in[(k + d + K) % K], 0));
        PCK(tf_fused_band(ctx, 0, y_of(k), y_of(k + 1), true, lane, start));
        if (n == 1 && k >= 2) PCK(fd_band(k - 1));
    }
    if (n > 1) {
        PCK(tf_fused_span(ctx, 0, 1, n - 1, false, lane, &mid));
        for (int k = 0; k < K; ++k) PCK(fd_band(k));
    } else {
        PCK(fd_band(K - 1));
        PCK(fd_band(0));
    }
    *end = {mid.fcur, mid.pcur ^ 1, mid.ucur, false};
    PCK(cudaEventRecord(ev_join[0], lane));
    PCK(cudaStreamWaitEvent(origin, ev_join[0], 0));
    PCK(cudaEventRecord(ev_join[1], ctx->xfer_out));
    PCK(cudaStreamWaitEvent(origin, ev_join[1], 0));
    PCK(cudaEventRecord(ev_join[2], ctx->xfer_in));
    PCK(cudaStreamWaitEvent(origin, ev_join[2], 0));
    return cudaSuccess;
}

static bool pinned_or_null(const void* p) {
    if (!p) return true;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// The pipeline is some fifty stream operations, whose enqueueing would set the
// pace of a one-step call.  For pinned buffers it is captured once (on the
// private capture stream) into a CUDA graph per (buffers, n, cursors) and
// replayed on the context's stream; other host memory is enqueued directly.
constexpr size_t kHostGraphs = 4;

static int advance_pipelined(tf_ctx* ctx, const void* h_in, int64_t n, void* h_out, bool banded) {
    TF_CK(ctx, make_pipeline(ctx));
    auto enqueue = [&](cudaStream_t origin, FusedCursor* end) {
        return banded ? enqueue_banded(ctx, origin, h_in, n, h_out, end)
                      : enqueue_pipeline(ctx, origin, h_in, n, h_out, end);
    };
    FusedCursor probe{ctx->fcur, ctx->pcur, ctx->ucur, ctx->fd_pending};
    TF_CK(ctx, tf_fused_span(ctx, 0, 1, 0, false, ctx->stream, &probe));   // plans the tiles only
    FusedCursor end{};
    const bool pending = h_in ? false : ctx->fd_pending;
    if (pinned_or_null(h_in) && pinned_or_null(h_out)) {
        tf_ctx::HostGraph* g = nullptr;
        for (auto& c : ctx->host_graphs)
            if (c.in == h_in && c.out == h_out && c.n == n && c.fcur == ctx->fcur && c.pcur == ctx->pcur &&
                c.ucur == ctx->ucur && c.fd_pending == pending)
                g = &c;
        if (!g) {
            const int64_t launches0 = ctx->launches;
            TF_CK(ctx, cudaStreamBeginCapture(ctx->xfer_cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue(ctx->xfer_cap, &end);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(ctx->xfer_cap, &graph);
            if (e == cudaSuccess) e = e2;
            cudaGraphExec_t exec = nullptr;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            TF_CK(ctx, e);
            if (ctx->host_graphs.size() == kHostGraphs) {
                cudaGraphExecDestroy(ctx->host_graphs.front().exec);
                ctx->host_graphs.erase(ctx->host_graphs.begin());
            }
            ctx->host_graphs.push_back({h_in, h_out, n, ctx->fcur, ctx->pcur, ctx->ucur, pending, exec,
                                        end.fcur, end.pcur, end.ucur, end.fd_pending,
                                        ctx->launches - launches0});
            g = &ctx->host_graphs.back();
            ctx->launches = launches0;
        }
        TF_CK(ctx, cudaGraphLaunch(g->exec, ctx->stream));
        end = {g->fcur_end, g->pcur_end, g->ucur_end, g->fd_pending_end};
        ctx->launches += g->launches;
    } else {
        TF_CK(ctx, enqueue(ctx->stream, &end));
    }
    ctx->fcur = end.fcur;
    ctx->pcur = end.pcur;
    ctx->ucur = end.ucur;
    ctx->fd_pending = end.fd_pending;
    ctx->steps += n;
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_advance_host(tf_ctx* ctx, const void* h_in, int64_t n, void* h_out) {
    const TfRange nvtx_range("tf_advance_host");
    if (!ctx) return TF_ERR_ARG;
    if (n < 0) return fail(ctx, TF_ERR_ARG, "negative step count");
    if (ctx->batch > 1 && (h_in || h_out) && tf_fused_supported(ctx))
        return advance_pipelined(ctx, h_in, n, h_out, false);
    if (ctx->batch == 1 && h_in && h_out && n >= 1 && tf_fused_supported(ctx) && bands_for(ctx) >= 3)
        return advance_pipelined(ctx, h_in, n, h_out, true);
    int rc;
    if (h_in) {
        ctx->fd_pending = false;  // the uploaded raw state is a plain state
        if ((rc = copy_state(ctx, const_cast<void*>(h_in), false)) != TF_OK) return rc;
    }
    if (n > 0) TF_CK(ctx, tf_launch_steps(ctx, n));
    if (h_out) {
        TF_CK(ctx, tf_launch_flush(ctx));
        if ((rc = copy_state(ctx, h_out, true)) != TF_OK) return rc;
    }
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TF_OK;
}

int tf_plan_tiles(int nx, int ny, int batch, long long slots, int out[3], int* col_start, int cap) {
    if (nx < 1 || ny < 1 || nx > kMaxDim || ny > kMaxDim || batch < 1 || slots < 1 || !out)
        return TF_ERR_ARG;
    const bool wide = wide_for(nx, ny, batch, slots);
    const int txm = wide ? TX_WIDE : TX, tym = wide ? TY_WIDE : TY_DEFAULT;
    const int cols = (nx + txm - 1) / txm;
    out[0] = wide ? 1 : 0;
    out[1] = cols;
    out[2] = tile_rows_for(cols, ny, tym, batch, slots);
    if (col_start) {
        if (cap < cols + 1) return TF_ERR_ARG;
        for (int k = 0; k <= cols; ++k) col_start[k] = tile_col(k, cols, nx);
    }
    return TF_OK;
}

struct CkptHeader {
    uint64_t magic;
    int32_t version, nx, ny, batch, n_sub, storage;
    int64_t steps;
    uint64_t state_bytes;
};

int tf_save(tf_ctx* ctx, const char* path) {
    if (!ctx) return TF_ERR_ARG;
    if (!path) return fail(ctx, TF_ERR_ARG, "null path");
    std::vector<char> buf(tf_state_bytes(ctx));
    TF_CK(ctx, tf_launch_flush(ctx));
    int rc = copy_state(ctx, buf.data(), true);
    if (rc != TF_OK) return rc;
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    CkptHeader h{kMagic, kVersion, ctx->nx, ctx->ny, ctx->batch, ctx->n_sub, ctx->storage,
                 ctx->steps, (uint64_t)buf.size()};
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(ctx, TF_ERR_IO, "cannot open checkpoint for writing");
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 &&
              std::fwrite(ctx->params.data(), sizeof(tf_params), ctx->batch, fp) ==
                  (size_t)ctx->batch &&
              std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? TF_OK : fail(ctx, TF_ERR_IO, "short write to checkpoint");
}

int tf_load(tf_ctx* ctx, const char* path) {
    if (!ctx) return TF_ERR_ARG;
    if (!path) return fail(ctx, TF_ERR_ARG, "null path");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(ctx, TF_ERR_IO, "cannot open checkpoint for reading");
    CkptHeader h{};
    std::vector<tf_params> prm(ctx->batch);
    std::vector<char> buf(tf_state_bytes(ctx));
    bool ok = std::fread(&h, sizeof h, 1, fp) == 1;
    ok = ok && h.magic == kMagic && h.version == kVersion && h.nx == ctx->nx && h.ny == ctx->ny &&
         h.batch == ctx->batch && h.n_sub == ctx->n_sub && h.storage == ctx->storage &&
         h.state_bytes == buf.size();
    ok = ok && std::fread(prm.data(), sizeof(tf_params), ctx->batch, fp) == (size_t)ctx->batch;
    ok = ok && std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) return fail(ctx, TF_ERR_IO, "checkpoint header or size does not match this context");
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->fd_pending = false;
    int rc = copy_state(ctx, buf.data(), false);
    if (rc != TF_OK) return rc;
    TF_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->steps = h.steps;
    return TF_OK;
}

}  // extern "C"
