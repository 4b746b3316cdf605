// Fused coupled step of one context: one kernel launch per lattice step in
// steady state (the step regrouping, tile stages and shared-memory layout are
// described in tf_fused.cuh).  Launch sequence per run: LBM-only prologue,
// steady-state launches, FD-only epilogue before any read.
#include "tf_fused.cuh"
#include "tf_strip.cuh"

namespace {

// Two tile geometries: narrow (TX x TY_DEFAULT, the 100 KB layout) for grids
// whose tiles fit in one wave of resident CTAs, wide (TX_WIDE x TY_WIDE) for
// larger grids.  The wide layout's extra shared memory leaves less of the
// unified L1 for the population pulls, which cost the one-wave 4 x 256^2
// sweep 1-3%, while its wider rows cut the sub-step work per site on large
// grids (+5-6% at 1024^2 and 2048^2, measured).
template <bool WIDE>
struct CtxGeo {
    static constexpr int TXM = WIDE ? TX_WIDE : TX;
    static constexpr int TYM = WIDE ? TY_WIDE : TY_DEFAULT;
};

// One tile per CTA: tile (blockIdx.x, blockIdx.y) of instance blockIdx.z.
// The rows [y_lo, y_hi) (all ny rows, or a band of them) are cut into
// gridDim.y tile rows of floor or ceil((y_hi - y_lo) / gridDim.y) rows each
// (at most TYM; the host picks gridDim.y), the nx columns into gridDim.x tile
// columns of at most TXM columns (tile_col; the host picks gridDim.x).
template <bool DO_FD, bool DO_LBM, class S, bool WIDE>
__global__ void __launch_bounds__(NT, 2) k_fused(const TileArgs<S> a, int y_lo, int y_hi) {
    using C = CtxGeo<WIDE>;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tfp::mbar_init(&bar, 1);
        tfp::fence_mbar_init();
    }
    __syncthreads();
    const int y0 = y_lo + (int)((long long)blockIdx.y * (y_hi - y_lo) / gridDim.y);
    const int y1 = y_lo + (int)((long long)(blockIdx.y + 1) * (y_hi - y_lo) / gridDim.y);
    const int x0 = tile_col(blockIdx.x, gridDim.x, a.nx), x1 = tile_col(blockIdx.x + 1, gridDim.x, a.nx);
    TF_BC_BEGIN();
    fused_tile<DO_FD, DO_LBM, S, C::TYM, false, C::TXM>(a, blockIdx.z, x0, y0, x1 - x0, y1 - y0, &bar, 0);
    TF_BC_END(a.err);
}

template <bool DO_FD, bool DO_LBM, class S>
cudaError_t configure_one() {
    cudaError_t e = cudaFuncSetAttribute(k_fused<DO_FD, DO_LBM, S, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<DO_FD, DO_LBM, TY_DEFAULT, TX>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fused<DO_FD, DO_LBM, S, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<DO_FD, DO_LBM, TY_WIDE, TX_WIDE>::SMEM);
}

template <class S>
cudaError_t configure() {
    cudaError_t e = configure_one<true, true, S>();
    if (e == cudaSuccess) e = configure_one<false, true, S>();
    if (e == cudaSuccess) e = configure_one<true, false, S>();
    if (e == cudaSuccess) e = configure_strip<S>();
    return e;
}

// Launch target: instances [inst0, inst0 + count) on `stream`, reading and
// writing the buffers the cursors in `cur` name.  The kernels address
// instance blockIdx.z from their base pointers, so a span is the same kernel
// on bases offset by inst0.
struct Span {
    int inst0, count, tile_rows;
    cudaStream_t stream;
    FusedCursor* cur;
    int y_lo = 0, y_hi = 0;   // rows of a band launch (y_hi = 0: all rows, tile_rows tile rows)
};

template <class S>
TileArgs<S> span_args(tf_ctx* ctx, const Span& sp) {
    using T = typename S::T;
    DevBuffers& d = ctx->d;
    const int fc = sp.cur->fcur, pc = sp.cur->pcur, uc = sp.cur->ucur;
    const long long N = ctx->N, b0 = sp.inst0;
    return TileArgs<S>{static_cast<const T*>(d.f[fc]) + pop_index(b0, 0, 0, 0, N),
                       static_cast<T*>(d.f[fc ^ 1]) + pop_index(b0, 0, 0, 0, N),
                       d.phi[pc] + b0 * N, d.phi[pc ^ 1] + b0 * N, d.Q[pc] + b0 * 2 * N,
                       d.Q[pc ^ 1] + b0 * 2 * N, d.u[uc] + b0 * 4 * N, d.u[uc ^ 1] + b0 * 4 * N,
                       d.prm + b0, ctx->nx, ctx->ny, d.flags};
}

template <bool DO_FD, bool DO_LBM, class S, bool WIDE>
void launch_as(tf_ctx* ctx, const Span& sp) {
    using G = Geo<DO_FD, DO_LBM, CtxGeo<WIDE>::TYM, CtxGeo<WIDE>::TXM>;
    const TileArgs<S> a = span_args<S>(ctx, sp);
    if (DO_FD && DO_LBM && ctx->use_strip) {
        launch_strip<S>(a, dim3(ctx->strip_cols, ctx->strip_segs, sp.count), sp.stream);
        return;
    }
    const bool band = sp.y_hi > 0;
    const int y_lo = band ? sp.y_lo : 0, y_hi = band ? sp.y_hi : ctx->ny;
    const int rows = band ? (y_hi - y_lo + CtxGeo<WIDE>::TYM - 1) / CtxGeo<WIDE>::TYM : sp.tile_rows;
    const dim3 grid(ctx->tile_cols, rows, sp.count);
    k_fused<DO_FD, DO_LBM, S, WIDE><<<grid, NT, G::SMEM, sp.stream>>>(a, y_lo, y_hi);
}

template <bool DO_FD, bool DO_LBM>
cudaError_t launch(tf_ctx* ctx, const Span& sp) {
    const bool w = ctx->wide_tiles;
    if (ctx->storage == TF_STORE_F16)
        w ? launch_as<DO_FD, DO_LBM, PopF16, true>(ctx, sp) : launch_as<DO_FD, DO_LBM, PopF16, false>(ctx, sp);
    else if (ctx->storage == TF_STORE_BF16)
        w ? launch_as<DO_FD, DO_LBM, PopBF16, true>(ctx, sp) : launch_as<DO_FD, DO_LBM, PopBF16, false>(ctx, sp);
    else
        w ? launch_as<DO_FD, DO_LBM, PopF32, true>(ctx, sp) : launch_as<DO_FD, DO_LBM, PopF32, false>(ctx, sp);
    if (DO_LBM) {
        sp.cur->fcur ^= 1;
        sp.cur->ucur ^= 1;
    }
    if (DO_FD) sp.cur->pcur ^= 1;
    ctx->launches += 1;
    return cudaGetLastError();
}

// n steps (LBM-only first when nothing is pending), then the pending
// sub-steps when `flush`.
cudaError_t run(tf_ctx* ctx, const Span& sp, int64_t n, bool flush) {
    for (int64_t it = 0; it < n; ++it) {
        cudaError_t e = sp.cur->fd_pending ? launch<true, true>(ctx, sp) : launch<false, true>(ctx, sp);
        if (e != cudaSuccess) return e;
        sp.cur->fd_pending = true;
    }
    if (flush && sp.cur->fd_pending) {
        cudaError_t e = launch<true, false>(ctx, sp);
        sp.cur->fd_pending = false;
        return e;
    }
    return cudaSuccess;
}

FusedCursor cursor_of(const tf_ctx* ctx) { return {ctx->fcur, ctx->pcur, ctx->ucur, ctx->fd_pending}; }

void set_cursor(tf_ctx* ctx, const FusedCursor& c) {
    ctx->fcur = c.fcur;
    ctx->pcur = c.pcur;
    ctx->ucur = c.ucur;
    ctx->fd_pending = c.fd_pending;
}

}  // namespace

bool tf_fused_supported(const tf_ctx* ctx) { return ctx->n_sub == NS_FUSED; }

// The strip kernel indexes one fluid's nine population planes with 32-bit
// element offsets: 9 nx ny must stay below 2^31.
bool tf_strip_supported(const tf_ctx* ctx) {
    return ctx->n_sub == NS_FUSED && ctx->nx % 4 == 0 && 9LL * ctx->N < (1LL << 31);
}

cudaError_t tf_configure_fused_kernels() {
    cudaError_t e = configure<PopF32>();
    if (e == cudaSuccess) e = configure<PopF16>();
    if (e == cudaSuccess) e = configure<PopBF16>();
    return e;
}

// Tile rows of the per-context launches.  When the tiles of TY_DEFAULT rows
// fit in one wave of resident CTAs, the rows are cut finer (down to tiles of
// kMinTileRows rows) so that the wave is as full as possible: at one wave the
// step takes as long as one SM's tiles, and shorter tiles shorten that.
// Otherwise the fewest tile rows of at most TY_DEFAULT rows are used.
constexpr int kMinTileRows = 8;

// Narrow tiles while a step fits in one wave of resident CTAs (there the step
// lasts one SM's pair of tiles, so shorter tile rows matter more than wider
// tiles); wide tiles beyond.
bool wide_for(int nx, int ny, int batch, long long slots) {
    return (long long)((nx + TX - 1) / TX) * ((ny + TY_DEFAULT - 1) / TY_DEFAULT) * batch > slots;
}

int tile_rows_for(int ntx, int ny, int tym, int batch, long long slots) {
    const long long per_row = (long long)ntx * batch;   // tiles per tile row
    const int need = (ny + tym - 1) / tym;
    const long long fit = slots / per_row;          // tile rows that one wave holds
    if (fit <= need) return need;
    const int most = ny / kMinTileRows > need ? ny / kMinTileRows : need;
    return (int)(fit < most ? fit : most);
}

// Strip kernel plan: strips of at most ts::TWMAX columns (cut at multiples
// of 4 by tile_col), and as many row segments as fill one wave of resident
// CTAs, with segments of at least kMinSegRows rows (each segment recomputes
// up to 12 rows of sub-step halo above and below it).
constexpr int kMinSegRows = 32;
// TF_KERNEL_AUTO picks the strip kernel on grids of several waves of tiles
// when the strip plan keeps at least 90% of one wave of resident CTAs busy.
// Each strip segment (at least kMinSegRows rows) pays up to 12 rows of
// sub-step halo above and below it and a pipeline fill of about seven 8-row
// blocks, so a strip plan that leaves SMs idle loses to the tiles.  Measured
// (us per step, strip / tile): 2048^2 301 / 348, 1536^2 170 / 210, 1024^2
// (297 CTAs, 38-row segments) 90 / 98, 2 x 1024^2 161 / 181, 4 x 512^2 97 /
// 106; 768^2 (192 CTAs) 78 / 69, 640^2 (140 CTAs) 49 / 49, 512^2 (96 CTAs)
// 49 / 31.
constexpr int kAutoStripFillPct = 90;

int strip_segs_for(int ncols, int ny, int batch, long long slots) {
    const long long per = (long long)ncols * batch;
    long long segs = slots / per;
    const long long most = ny / kMinSegRows;
    if (segs > most) segs = most;
    return segs < 1 ? 1 : (int)segs;
}

cudaError_t plan_tile_rows(tf_ctx* ctx) {
    if (ctx->tile_rows > 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0, per_sm_strip = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_fused<true, true, PopF32, false>, NT, Geo<true, true, TY_DEFAULT, TX>::SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_strip, k_strip<PopF32>, NT,
                                                          ts::SMEM);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)sms * per_sm;
    ctx->wide_tiles = wide_for(ctx->nx, ctx->ny, ctx->batch, slots);
    const int txm = ctx->wide_tiles ? TX_WIDE : TX, tym = ctx->wide_tiles ? TY_WIDE : TY_DEFAULT;
    ctx->tile_cols = (ctx->nx + txm - 1) / txm;
    ctx->tile_rows = tile_rows_for(ctx->tile_cols, ctx->ny, tym, ctx->batch, slots);
    ctx->strip_cols = (ctx->nx + ts::TWMAX - 1) / ts::TWMAX;
    ctx->strip_segs = strip_segs_for(ctx->strip_cols, ctx->ny, ctx->batch,
                                     (long long)sms * (per_sm_strip > 0 ? per_sm_strip : 1));
    // Steady-state kernel (tf_set_step_kernel; AUTO: see kAutoStripFillPct).
    const bool can = tf_strip_supported(ctx) && per_sm_strip > 0;
    const long long strip_ctas = (long long)ctx->strip_cols * ctx->batch * ctx->strip_segs;
    const bool fills = strip_ctas * 100 >= (long long)sms * per_sm_strip * kAutoStripFillPct;
    ctx->use_strip = can && (ctx->step_kernel == TF_KERNEL_STRIP ||
                             (ctx->step_kernel == TF_KERNEL_AUTO && ctx->wide_tiles && fills));
    return cudaSuccess;
}

cudaError_t tf_fused_steps(tf_ctx* ctx, int64_t n) {
    cudaError_t e = plan_tile_rows(ctx);
    if (e != cudaSuccess) return e;
    FusedCursor c = cursor_of(ctx);
    e = run(ctx, Span{0, ctx->batch, ctx->tile_rows, ctx->stream, &c}, n, false);
    set_cursor(ctx, c);
    if (e == cudaSuccess) ctx->steps += n;
    return e;
}

cudaError_t tf_fused_flush(tf_ctx* ctx) {
    if (!ctx->fd_pending) return cudaSuccess;
    cudaError_t e = plan_tile_rows(ctx);
    if (e != cudaSuccess) return e;
    FusedCursor c = cursor_of(ctx);
    e = run(ctx, Span{0, ctx->batch, ctx->tile_rows, ctx->stream, &c}, 0, true);
    set_cursor(ctx, c);
    return e;
}

cudaError_t tf_fused_span(tf_ctx* ctx, int inst0, int count, int64_t n, bool flush,
                          cudaStream_t stream, FusedCursor* cur) {
    cudaError_t e = plan_tile_rows(ctx);
    if (e != cudaSuccess) return e;
    // The batch's tile plan: spans of different instances, launched on
    // different streams, then share the resident CTA slots as one batched
    // launch would.
    return run(ctx, Span{inst0, count, ctx->tile_rows, stream, cur}, n, flush);
}

cudaError_t tf_fused_band(tf_ctx* ctx, int inst, int y_lo, int y_hi, bool lbm, cudaStream_t stream,
                          FusedCursor cur) {
    cudaError_t e = plan_tile_rows(ctx);
    if (e != cudaSuccess) return e;
    const Span sp{inst, 1, ctx->tile_rows, stream, &cur, y_lo, y_hi};
    return lbm ? launch<false, true>(ctx, sp) : launch<true, false>(ctx, sp);
}

cudaError_t tf_plan_fused(tf_ctx* ctx) {
    ctx->tile_rows = 0;
    return plan_tile_rows(ctx);
}
