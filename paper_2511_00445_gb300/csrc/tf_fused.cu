// Fused coupled step of one context: one kernel launch per lattice step in
// steady state (the step regrouping, tile stages and shared-memory layout are
// described in tf_fused.cuh).  Launch sequence per run: LBM-only prologue,
// steady-state launches, FD-only epilogue before any read.
#include "tf_fused.cuh"

namespace {

// One tile per CTA: tile (blockIdx.x, blockIdx.y) of instance blockIdx.z.
template <bool DO_FD, bool DO_LBM, class S>
__global__ void __launch_bounds__(NT, 2) k_fused(const TileArgs<S> a) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tfp::mbar_init(&bar, 1);
        tfp::fence_mbar_init();
    }
    __syncthreads();
    fused_tile<DO_FD, DO_LBM, S, TY_DEFAULT>(a, blockIdx.z, blockIdx.x * TX,
                                             blockIdx.y * TY_DEFAULT, &bar, 0);
}

template <bool DO_FD, bool DO_LBM, class S>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(k_fused<DO_FD, DO_LBM, S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<DO_FD, DO_LBM, TY_DEFAULT>::SMEM);
}

template <class S>
cudaError_t configure() {
    cudaError_t e = configure_one<true, true, S>();
    if (e == cudaSuccess) e = configure_one<false, true, S>();
    if (e == cudaSuccess) e = configure_one<true, false, S>();
    return e;
}

template <bool DO_FD, bool DO_LBM, class S>
void launch_as(tf_ctx* ctx) {
    using G = Geo<DO_FD, DO_LBM, TY_DEFAULT>;
    using T = typename S::T;
    DevBuffers& d = ctx->d;
    const dim3 grid((ctx->nx + TX - 1) / TX, (ctx->ny + TY_DEFAULT - 1) / TY_DEFAULT, ctx->batch);
    const int fc = ctx->fcur, pc = ctx->pcur, uc = ctx->ucur;
    const TileArgs<S> a{static_cast<const T*>(d.f[fc]), static_cast<T*>(d.f[fc ^ 1]),
                        d.phi[pc], d.phi[pc ^ 1], d.Q[pc], d.Q[pc ^ 1], d.u[uc], d.u[uc ^ 1],
                        d.prm, ctx->nx, ctx->ny, d.flags};
    k_fused<DO_FD, DO_LBM, S><<<grid, NT, G::SMEM, ctx->stream>>>(a);
}

template <bool DO_FD, bool DO_LBM>
cudaError_t launch(tf_ctx* ctx) {
    if (ctx->storage == TF_STORE_F16)
        launch_as<DO_FD, DO_LBM, PopF16>(ctx);
    else if (ctx->storage == TF_STORE_BF16)
        launch_as<DO_FD, DO_LBM, PopBF16>(ctx);
    else
        launch_as<DO_FD, DO_LBM, PopF32>(ctx);
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
    cudaError_t e = configure<PopF32>();
    if (e == cudaSuccess) e = configure<PopF16>();
    if (e == cudaSuccess) e = configure<PopBF16>();
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
