// Ensembles (declared in include/twofluid.h): several contexts of possibly
// different grid sizes stepped together by one persistent cooperative kernel.
//
// Work-list: tile t of a step is found by scanning the groups' first-tile
// offsets (per tile shape); within a group the tiles are numbered instance
// by instance, row-major.  CTAs take tiles from a per-step atomic ticket
// counter (dynamic balance across uneven instance sizes), run the same
// per-tile code as the per-context kernel (tf_fused.cuh), and meet at a grid
// barrier between steps.  Every spin is bounded; a CTA that gives up raises
// the abort word so that the others leave too, and the code lands in the
// members' device status words.
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "tf_fused.cuh"

namespace {

// Candidate tile shapes (columns x rows, the largest tile of each; ens_tile
// balances the tiles of a group like the per-context tiles).
constexpr int kTileX[3] = {TX, TX, TX_WIDE};
constexpr int kTileY[3] = {32, 24, TY_WIDE};
// Candidates 0..5: persistent launches, tile shape c / 2 with 2 - c % 2 CTAs
// per SM; 6, 7: one launch per step over every tile of every group (k_ens_step)
// with the 32 x 32 and the 40 x 30 shape; 8: every group's own planned
// per-context launch (strip or tile kernel) per step.
constexpr int kCandidates = TF_ENS_CANDIDATES;
constexpr int kPersistentCandidates = 6;
constexpr int kGroupPlans = 8;
constexpr bool persistent_cfg(int c) { return c < kPersistentCandidates; }
constexpr int shape_of(int c) { return c < kPersistentCandidates ? c / 2 : (c == 6 ? 0 : 2); }
constexpr int ctas_of(int c) { return c < kPersistentCandidates ? 2 - c % 2 : 2; }
constexpr uint32_t kBarrierPolls = 1u << 23;   // x ~128 ns sleeps: about one second
constexpr int64_t kMaxStepsPerLaunch = 1024;

struct EnsGroup {
    void* f[2];              // population buffers: [0] = the group's current one at ensemble parity 0
    float* phi[2];
    float* Q[2];
    float* u[2];
    const DevParams* prm;
    int* err;                // the group's device status word
    int nx, ny, batch;
    int tiles_x[3];          // tile columns per tile shape
    long long begin[3];      // first tile of the group per tile shape
};

struct EnsCtl {
    unsigned int ticket[2];  // per-step tile counters (steps alternate)
    unsigned int arrive;     // grid-barrier arrivals
    unsigned int gen;        // grid-barrier generation
    int abort;               // set by a CTA that gave up a wait
    int pad[3];
};

template <int TY, int TXW>
constexpr int shape_index() {
    return TXW == TX_WIDE ? 2 : (TY == 32 ? 0 : 1);
}

// All CTAs of the launch meet here.  Thread 0 of each CTA arrives on a
// global counter; the last arrival resets the counter and the finished
// step's ticket slot, then bumps the generation the others spin on.
__device__ __forceinline__ bool grid_barrier(EnsCtl* ctl, int k, int* err, uint32_t polls) {
    __shared__ int s_ok;
    // Next step reads this step's stores through bulk copies (async proxy).
    tfp::fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int gen = *reinterpret_cast<volatile unsigned int*>(&ctl->gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&ctl->arrive, 1u);
        if (arrived == gridDim.x - 1) {
            ctl->arrive = 0;
            ctl->ticket[k & 1] = 0;
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            uint32_t it = 0;
            while (*reinterpret_cast<volatile unsigned int*>(&ctl->gen) == gen) {
                if (*reinterpret_cast<volatile int*>(&ctl->abort)) {
                    ok = 0;
                    break;
                }
                if (++it > polls) {
                    atomicExch(err, TF_ERR_TIMEOUT);
                    atomicExch(&ctl->abort, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    tfp::fence_proxy_async_global();
    return s_ok != 0;
}

// Tile t of a step: group g, instance b and rectangle.  Per group and shape
// the tiles are numbered instance by instance, row-major; the ny rows are cut
// into ceil(ny / TY) tile rows of floor or ceil(ny / that) rows, the nx columns
// into ceil(nx / TXW) columns by tile_col, so no tile is a thin remainder.
struct EnsTile {
    int g, b, x0, y0, tw, th;
};

template <int TY, int TXW>
__device__ __forceinline__ EnsTile ens_tile(const EnsGroup* __restrict__ groups, int n_groups,
                                            long long t) {
    constexpr int TI = shape_index<TY, TXW>();
    int g = 0;
    while (g + 1 < n_groups && groups[g + 1].begin[TI] <= t) ++g;
    const EnsGroup& G = groups[g];
    const long long local = t - G.begin[TI];
    const int ntx = G.tiles_x[TI], nty = (G.ny + TY - 1) / TY;
    const long long per = (long long)ntx * nty;
    const int b = (int)(local / per);
    const long long r = local - (long long)b * per;
    const int tyi = (int)(r / ntx), txi = (int)(r - (long long)tyi * ntx);
    const int y0 = (int)((long long)tyi * G.ny / nty);
    const int y1 = (int)((long long)(tyi + 1) * G.ny / nty);
    const int x0 = tile_col(txi, ntx, G.nx);
    return {g, b, x0, y0, tile_col(txi + 1, ntx, G.nx) - x0, y1 - y0};
}

// `steps` lattice steps of every tile of every group.  Parities fpar, ppar,
// upar select the current population, phi/Q and velocity buffers at step 0;
// each step flips the ones it writes.
template <bool DO_FD, bool DO_LBM, class S, int TY, int TXW>
__global__ void __launch_bounds__(NT, 2)
k_ens(const EnsGroup* __restrict__ groups, int n_groups, long long total, int steps, int fpar,
      int ppar, int upar, EnsCtl* ctl, uint32_t polls, int held) {
    using T = typename S::T;
    __shared__ __align__(8) uint64_t bar;
    __shared__ long long s_ticket;
    if (threadIdx.x == 0) {
        tfp::mbar_init(&bar, 1);
        tfp::fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    TF_BC_BEGIN();
    for (int k = 0; k < steps; ++k) {
        const int fp = fpar ^ (DO_LBM ? (k & 1) : 0);
        const int pp = ppar ^ (DO_FD ? (k & 1) : 0);
        const int up = upar ^ (DO_LBM ? (k & 1) : 0);
        for (;;) {
            if (threadIdx.x == 0)
                s_ticket = *reinterpret_cast<volatile int*>(&ctl->abort)
                               ? total
                               : (long long)atomicAdd(&ctl->ticket[k & 1], 1u);
            __syncthreads();
            const long long t = s_ticket;
            __syncthreads();
            if (t >= total) break;
            const EnsTile r = ens_tile<TY, TXW>(groups, n_groups, t);
            const EnsGroup& G = groups[r.g];
            const TileArgs<S> a{static_cast<const T*>(G.f[fp]), static_cast<T*>(G.f[fp ^ 1]),
                                G.phi[pp], G.phi[pp ^ 1], G.Q[pp], G.Q[pp ^ 1], G.u[up],
                                G.u[up ^ 1], G.prm, G.nx, G.ny, G.err};
            if (!fused_tile<DO_FD, DO_LBM, S, TY, true, TXW>(a, r.b, r.x0, r.y0, r.tw, r.th, &bar,
                                                           phase)) {
                if (threadIdx.x == 0) atomicExch(&ctl->abort, 1);
                return;
            }
            if ((G.nx & 3) == 0) ++phase;   // the tile went through the mbarrier
            __syncthreads();
        }
        // Failure drill (tf_ensemble_fault_drill): CTA `held` leaves at the
        // first barrier without arriving; it has no bulk copy in flight here.
        if (k == 0 && (int)blockIdx.x == held && k + 1 < steps) return;
        if (k + 1 < steps && !grid_barrier(ctl, k, groups[0].err, polls)) return;
    }
    TF_BC_END(groups[0].err);
}

// One step of every tile of every group, one tile per CTA (candidates 6, 7).
// Nothing in the launch reads what it writes, so the populations are read
// through L1 like in the per-context kernel, and no grid barrier is needed.
// The per-step parities are the launch's.
template <class S, int TY, int TXW>
__global__ void __launch_bounds__(NT, 2)
k_ens_step(const EnsGroup* __restrict__ groups, int n_groups, int fp, int pp, int up) {
    using T = typename S::T;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tfp::mbar_init(&bar, 1);
        tfp::fence_mbar_init();
    }
    __syncthreads();
    TF_BC_BEGIN();
    const EnsTile r = ens_tile<TY, TXW>(groups, n_groups, blockIdx.x);
    const EnsGroup& G = groups[r.g];
    const TileArgs<S> a{static_cast<const T*>(G.f[fp]), static_cast<T*>(G.f[fp ^ 1]),
                        G.phi[pp], G.phi[pp ^ 1], G.Q[pp], G.Q[pp ^ 1], G.u[up],
                        G.u[up ^ 1], G.prm, G.nx, G.ny, G.err};
    // a bulk copy that did not complete is reported in the group's status word
    fused_tile<true, true, S, TY, false, TXW>(a, r.b, r.x0, r.y0, r.tw, r.th, &bar, 0u);
    TF_BC_END(G.err);
}

enum Mode { kPrologue = 0, kSteady = 1 };

typedef void (*EnsKernel)(const EnsGroup*, int, long long, int, int, int, int, EnsCtl*, uint32_t,
                          int);

template <class S>
EnsKernel pick(int mode, int ti) {
    if (mode == kPrologue) return k_ens<false, true, S, 32, TX>;
    if (ti == 0) return k_ens<true, true, S, 32, TX>;
    if (ti == 1) return k_ens<true, true, S, 24, TX>;
    return k_ens<true, true, S, TY_WIDE, TX_WIDE>;
}

typedef void (*StepKernel)(const EnsGroup*, int, int, int, int);

template <class S>
StepKernel pick_step(int ti) {
    if (ti == 0) return k_ens_step<S, 32, TX>;
    return k_ens_step<S, TY_WIDE, TX_WIDE>;
}

StepKernel step_kernel_for(int storage, int ti) {
    if (storage == TF_STORE_F16) return pick_step<PopF16>(ti);
    if (storage == TF_STORE_BF16) return pick_step<PopBF16>(ti);
    return pick_step<PopF32>(ti);
}

EnsKernel kernel_for(int storage, int mode, int ti) {
    if (storage == TF_STORE_F16) return pick<PopF16>(mode, ti);
    if (storage == TF_STORE_BF16) return pick<PopBF16>(mode, ti);
    return pick<PopF32>(mode, ti);
}

size_t smem_for(int mode, int ti) {
    if (mode == kPrologue) return Geo<false, true, 32>::SMEM;
    if (ti == 0) return Geo<true, true, 32>::SMEM;
    if (ti == 1) return Geo<true, true, 24>::SMEM;
    return Geo<true, true, TY_WIDE, TX_WIDE>::SMEM;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct tf_ensemble {
    std::vector<tf_ctx*> groups;
    std::vector<int> base_f, base_p, base_u;   // member buffer index at ensemble parity 0
    std::vector<EnsGroup> host_groups;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;         // private stream used only to record graphs
    // Group-plan steps: groups 1 .. n-1 run on their own streams, forked from
    // and joined back to the launching one (in a captured graph: parallel
    // branches), so that one group's CTAs fill the last wave of another's.
    std::vector<cudaStream_t> branch;          // [n_groups - 1], empty: one stream
    std::vector<cudaEvent_t> branch_ev;        // [n_groups]: the fork, then one join per branch
    int storage = TF_STORE_F32;
    EnsGroup* d_groups = nullptr;
    EnsCtl* d_ctl = nullptr;
    long long tiles[3] = {0, 0, 0};
    int cfg = 0;                               // autotuner candidate in use
    int fpar = 0, ppar = 0, upar = 0;
    bool pending = false;                      // sub-steps of the last step not yet applied
    int sm_count = 0;
    double us[kCandidates] = {};
    bool graphs = true;
    uint32_t drill_polls = 0;                  // tf_ensemble_fault_drill: barrier poll limit (0: default)
    int drill_held = -1;                       // ... and the CTA that does not arrive (-1: none)
    std::map<std::tuple<int, int64_t, int, int, int, int, uint32_t, int>, cudaGraphExec_t> cache;
    int64_t launches = 0;
    std::string last_error;
};

namespace {

void release_branches(tf_ensemble* e) {
    for (cudaStream_t b : e->branch) cudaStreamDestroy(b);
    for (cudaEvent_t ev : e->branch_ev) cudaEventDestroy(ev);
    e->branch.clear();
    e->branch_ev.clear();
}

int efail(tf_ensemble* e, int code, const std::string& msg) {
    if (e) e->last_error = msg;
    return code;
}

int efail_cuda(tf_ensemble* e, const char* where, cudaError_t err) {
    return efail(e, TF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(err));
}

#define TF_ECK(e, call)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return efail_cuda(e, #call, e_);  \
    } while (0)

// CTAs of one step of group member c under its own per-context plan.
long long planned_ctas(tf_ctx* c) {
    if (c->tile_rows <= 0 && tf_plan_fused(c) != cudaSuccess) return 0;
    return c->use_strip ? (long long)c->strip_cols * c->strip_segs * c->batch
                        : (long long)c->tile_cols * c->tile_rows * c->batch;
}

int grid_for(tf_ensemble* e, int mode, int cfg) {
    if (mode == kSteady && cfg == kGroupPlans) {   // CTAs of all groups' launches of one step
        long long n = 0;
        for (tf_ctx* c : e->groups) n += planned_ctas(c);
        return (int)n;
    }
    const int ti = mode == kPrologue ? 0 : shape_of(cfg);
    if (mode == kSteady && !persistent_cfg(cfg)) return (int)e->tiles[ti];   // one CTA per tile
    const int want = mode == kPrologue ? 2 : ctas_of(cfg);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(e->storage, mode, ti), NT,
                                                      smem_for(mode, ti)) != cudaSuccess ||
        per_sm < 1)
        return 0;
    long long g = (long long)(want < per_sm ? want : per_sm) * e->sm_count;
    const long long tiles = e->tiles[ti];
    return (int)(g < tiles ? g : tiles);
}

// Persistent candidates: zero the control block, then one cooperative launch
// of `steps` steps on `grid` CTAs (grid_for; computed outside any stream
// capture) into `st`.  Per-step candidates: `steps` launches of k_ens_step.
cudaError_t enqueue(tf_ensemble* e, int mode, int steps, int cfg, int grid, cudaStream_t st) {
    const int ti = mode == kPrologue ? 0 : shape_of(cfg);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (mode == kSteady && cfg == kGroupPlans) {
        // each group's own launches, from the ensemble's buffer parities; the
        // groups are independent, so all but the first go on branch streams
        const size_t ng = e->groups.size();
        const bool fork = ng > 1 && e->branch.size() == ng - 1;
        cudaError_t err = cudaSuccess;
        if (fork) {
            err = cudaEventRecord(e->branch_ev[0], st);
            for (size_t g = 1; g < ng && err == cudaSuccess; ++g)
                err = cudaStreamWaitEvent(e->branch[g - 1], e->branch_ev[0], 0);
            if (err != cudaSuccess) return err;
        }
        for (size_t g = 0; g < ng; ++g) {
            tf_ctx* c = e->groups[g];
            FusedCursor cur{e->base_f[g] ^ e->fpar, e->base_p[g] ^ e->ppar,
                            e->base_u[g] ^ e->upar, true};
            err = tf_fused_span(c, 0, c->batch, steps, false, fork && g > 0 ? e->branch[g - 1] : st, &cur);
            if (err != cudaSuccess) return err;
        }
        if (fork) {
            for (size_t g = 1; g < ng && err == cudaSuccess; ++g) {
                err = cudaEventRecord(e->branch_ev[g], e->branch[g - 1]);
                if (err == cudaSuccess) err = cudaStreamWaitEvent(st, e->branch_ev[g], 0);
            }
        }
        return err;
    }
    if (mode == kSteady && !persistent_cfg(cfg)) {
        const StepKernel k = step_kernel_for(e->storage, ti);
        const size_t smem = smem_for(kSteady, ti);
        const int ng = (int)e->groups.size();
        for (int s = 0; s < steps; ++s) {
            const int f = s & 1;
            k<<<grid, NT, smem, st>>>(e->d_groups, ng, e->fpar ^ f, e->ppar ^ f, e->upar ^ f);
            const cudaError_t err = cudaGetLastError();
            if (err != cudaSuccess) return err;
        }
        return cudaSuccess;
    }
    cudaError_t err = cudaMemsetAsync(e->d_ctl, 0, sizeof(EnsCtl), st);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = smem_for(mode, ti);
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const EnsGroup* g = e->d_groups;
    const int ng = (int)e->groups.size();
    const long long total = e->tiles[ti];
    const uint32_t polls = e->drill_polls ? e->drill_polls : kBarrierPolls;
    return cudaLaunchKernelEx(&lc, kernel_for(e->storage, mode, ti), g, ng, total, steps, e->fpar,
                              e->ppar, e->upar, e->d_ctl, polls, e->drill_held);
}

// Issue one launch, from the graph cache when this shape was captured before.
// Graphs are recorded on the ensemble's private capture stream (the caller's
// stream may be the legacy default stream, which cannot be captured) and
// launched into the caller's stream.
int issue(tf_ensemble* e, int mode, int steps) {
    const auto key = std::make_tuple(mode, (int64_t)steps, e->fpar, e->ppar, e->upar,
                                     mode == kPrologue ? 0 : e->cfg, e->drill_polls, e->drill_held);
    const int grid = grid_for(e, mode, e->cfg);
    auto it = e->cache.find(key);
    if (it != e->cache.end()) {
        TF_ECK(e, cudaGraphLaunch(it->second, e->stream));
    } else {
        bool done = false;
        if (e->graphs) {
            cudaGraph_t graph = nullptr;
            cudaError_t e0 = e->cap_stream ? cudaStreamBeginCapture(e->cap_stream,
                                                                    cudaStreamCaptureModeThreadLocal)
                                           : cudaErrorNotSupported;
            cudaError_t e1 = cudaErrorUnknown, e2 = cudaErrorUnknown, e3 = cudaErrorUnknown;
            if (e0 == cudaSuccess) {
                e1 = enqueue(e, mode, steps, e->cfg, grid, e->cap_stream);
                e2 = cudaStreamEndCapture(e->cap_stream, &graph);
                cudaGraphExec_t exec = nullptr;
                if (e1 == cudaSuccess && e2 == cudaSuccess && graph) {
                    e3 = cudaGraphInstantiate(&exec, graph, 0);
                    if (e3 == cudaSuccess) {
                        e->cache[key] = exec;
                        TF_ECK(e, cudaGraphLaunch(exec, e->stream));
                        done = true;
                    }
                }
                if (graph) cudaGraphDestroy(graph);
            }
            if (!done) {
                // Launch directly from now on; keep the reason for tf_ensemble_last_error.
                const cudaError_t why = e0 != cudaSuccess ? e0 : (e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3));
                e->last_error = std::string("graph capture unavailable (") +
                                (e0 != cudaSuccess ? "begin" : e1 != cudaSuccess ? "launch" : e2 != cudaSuccess ? "end" : "instantiate") +
                                "): " + cudaGetErrorString(why);
                cudaGetLastError();
                e->graphs = false;
            }
        }
        if (!done) TF_ECK(e, enqueue(e, mode, steps, e->cfg, grid, e->stream));
    }
    e->launches += mode == kSteady && e->cfg == kGroupPlans
                       ? (int64_t)steps * (int64_t)e->groups.size()
                       : (mode == kSteady && !persistent_cfg(e->cfg) ? steps : 1);
    if (mode == kPrologue) {
        e->fpar ^= 1;
        e->upar ^= 1;
        e->pending = true;
    } else {
        e->fpar ^= steps & 1;
        e->ppar ^= steps & 1;
        e->upar ^= steps & 1;
    }
    return TF_OK;
}

// Members' host-side state mirrors the ensemble's after every call.
void publish(tf_ensemble* e, int64_t steps) {
    for (size_t g = 0; g < e->groups.size(); ++g) {
        tf_ctx* c = e->groups[g];
        c->fcur = e->base_f[g] ^ e->fpar;
        c->pcur = e->base_p[g] ^ e->ppar;
        c->ucur = e->base_u[g] ^ e->upar;
        c->fd_pending = e->pending;
        c->steps += steps;
    }
}

// (Re)build the descriptors from the members' current buffers, completing
// every member's pending sub-steps first, and upload them.
int normalise(tf_ensemble* e) {
    for (tf_ctx* c : e->groups) TF_ECK(e, tf_launch_flush(c));
    long long begin[3] = {0, 0, 0};
    for (size_t g = 0; g < e->groups.size(); ++g) {
        tf_ctx* c = e->groups[g];
        DevBuffers& d = c->d;
        EnsGroup& G = e->host_groups[g];
        e->base_f[g] = c->fcur;
        e->base_p[g] = c->pcur;
        e->base_u[g] = c->ucur;
        for (int k = 0; k < 2; ++k) {
            G.f[k] = d.f[c->fcur ^ k];
            G.phi[k] = d.phi[c->pcur ^ k];
            G.Q[k] = d.Q[c->pcur ^ k];
            G.u[k] = d.u[c->ucur ^ k];
        }
        G.prm = d.prm;
        G.err = d.flags;
        G.nx = c->nx;
        G.ny = c->ny;
        G.batch = c->batch;
        for (int ti = 0; ti < 3; ++ti) {
            G.tiles_x[ti] = (c->nx + kTileX[ti] - 1) / kTileX[ti];
            G.begin[ti] = begin[ti];
            begin[ti] += (long long)c->batch * G.tiles_x[ti] * ((c->ny + kTileY[ti] - 1) / kTileY[ti]);
        }
    }
    for (int ti = 0; ti < 3; ++ti) e->tiles[ti] = begin[ti];
    TF_ECK(e, cudaMemcpyAsync(e->d_groups, e->host_groups.data(),
                              e->host_groups.size() * sizeof(EnsGroup), cudaMemcpyHostToDevice,
                              e->stream));
    TF_ECK(e, cudaStreamSynchronize(e->stream));   // host_groups may change on the next call
    e->fpar = e->ppar = e->upar = 0;
    e->pending = false;
    return TF_OK;
}

// A member read between ensemble calls completes its own pending sub-steps;
// then the members no longer agree with the ensemble's parities.
bool members_in_step(const tf_ensemble* e) {
    for (size_t g = 0; g < e->groups.size(); ++g) {
        const tf_ctx* c = e->groups[g];
        if (c->fd_pending != e->pending || c->fcur != (e->base_f[g] ^ e->fpar) ||
            c->pcur != (e->base_p[g] ^ e->ppar) || c->ucur != (e->base_u[g] ^ e->upar))
            return false;
    }
    return true;
}

template <bool DO_FD, bool DO_LBM, class S, int TY, int TXW>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_ens<DO_FD, DO_LBM, S, TY, TXW>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<DO_FD, DO_LBM, TY, TXW>::SMEM);
}

template <class S, int TY, int TXW>
cudaError_t set_step_smem() {
    return cudaFuncSetAttribute(k_ens_step<S, TY, TXW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<true, true, TY, TXW>::SMEM);
}

template <class S>
cudaError_t configure_storage() {
    cudaError_t e = set_smem<false, true, S, 32, TX>();
    if (e == cudaSuccess) e = set_step_smem<S, 32, TX>();
    if (e == cudaSuccess) e = set_step_smem<S, TY_WIDE, TX_WIDE>();
    if (e == cudaSuccess) e = set_smem<true, true, S, 32, TX>();
    if (e == cudaSuccess) e = set_smem<true, true, S, 24, TX>();
    if (e == cudaSuccess) e = set_smem<true, true, S, TY_WIDE, TX_WIDE>();
    return e;
}

}  // namespace

extern "C" {

size_t tf_ensemble_workspace_bytes(int n_groups) {
    if (n_groups < 1 || n_groups > TF_ENS_MAX_GROUPS) return 0;
    return align256((size_t)n_groups * sizeof(EnsGroup)) + align256(sizeof(EnsCtl));
}

int tf_ensemble_create(tf_ctx* const* groups, int n_groups, void* d_workspace,
                       size_t workspace_bytes, void* stream, tf_ensemble** out) {
    if (!out) return TF_ERR_ARG;
    *out = nullptr;
    if (!groups || n_groups < 1 || n_groups > TF_ENS_MAX_GROUPS) return TF_ERR_ARG;
    const size_t need = tf_ensemble_workspace_bytes(n_groups);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255) || workspace_bytes < need)
        return TF_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int g = 0; g < n_groups; ++g) {
        const tf_ctx* c = groups[g];
        if (!c || c->n_sub != NS_FUSED || c->stream != st || c->storage != groups[0]->storage)
            return TF_ERR_ARG;
        for (int h = 0; h < g; ++h)
            if (groups[h] == c) return TF_ERR_ARG;
    }
    tf_ensemble* e = new (std::nothrow) tf_ensemble();
    if (!e) return TF_ERR_ARG;
    e->groups.assign(groups, groups + n_groups);
    e->base_f.assign(n_groups, 0);
    e->base_p.assign(n_groups, 0);
    e->base_u.assign(n_groups, 0);
    e->host_groups.assign(n_groups, EnsGroup{});
    e->stream = st;
    e->storage = groups[0]->storage;
    char* ws = static_cast<char*>(d_workspace);
    e->d_groups = reinterpret_cast<EnsGroup*>(ws);
    e->d_ctl = reinterpret_cast<EnsCtl*>(ws + align256((size_t)n_groups * sizeof(EnsGroup)));
    int dev = 0, coop = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (err == cudaSuccess) err = configure_storage<PopF32>();
    if (err == cudaSuccess) err = configure_storage<PopF16>();
    if (err == cudaSuccess) err = configure_storage<PopBF16>();
    if (err == cudaSuccess && cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        e->cap_stream = nullptr;   // graphs unavailable; launches go directly into the stream
        cudaGetLastError();
    }
    if (err == cudaSuccess && n_groups > 1) {
        // branch streams and events for the group-plan steps; without them
        // the groups' launches stay on one stream
        bool ok = true;
        for (int g = 1; g < n_groups && ok; ++g) {
            cudaStream_t b = nullptr;
            ok = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) e->branch.push_back(b);
        }
        for (int g = 0; g < n_groups && ok; ++g) {
            cudaEvent_t ev = nullptr;
            ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
            if (ok) e->branch_ev.push_back(ev);
        }
        if (!ok) {
            release_branches(e);
            cudaGetLastError();
        }
    }
    if (err != cudaSuccess || !coop) {
        release_branches(e);
        if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
        delete e;
        return TF_ERR_CUDA;
    }
    const int rc = normalise(e);
    if (rc != TF_OK) {
        release_branches(e);
        if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
        delete e;
        return rc;
    }
    *out = e;
    return TF_OK;
}

int tf_ensemble_destroy(tf_ensemble* e) {
    if (!e) return TF_ERR_ARG;
    cudaStreamSynchronize(e->stream);
    for (auto& kv : e->cache) cudaGraphExecDestroy(kv.second);
    release_branches(e);
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    delete e;
    return TF_OK;
}

const char* tf_ensemble_last_error(const tf_ensemble* e) {
    return e ? e->last_error.c_str() : "null ensemble";
}

int tf_ensemble_step(tf_ensemble* e, int64_t n) {
    const TfRange nvtx_range("tf_ensemble_step");
    if (!e) return TF_ERR_ARG;
    if (n < 0) return efail(e, TF_ERR_ARG, "negative step count");
    if (n == 0) return TF_OK;
    if (!members_in_step(e)) {
        const int rc = normalise(e);
        if (rc != TF_OK) return rc;
    }
    int64_t left = n;
    int rc = TF_OK;
    if (!e->pending) {
        rc = issue(e, kPrologue, 1);
        left -= 1;
    }
    while (rc == TF_OK && left > 0) {
        const int64_t k = left < kMaxStepsPerLaunch ? left : kMaxStepsPerLaunch;
        rc = issue(e, kSteady, (int)k);
        left -= k;
    }
    publish(e, n - left);
    return rc;
}

int tf_ensemble_sync(tf_ensemble* e) {
    if (!e) return TF_ERR_ARG;
    TF_ECK(e, cudaStreamSynchronize(e->stream));
    for (tf_ctx* c : e->groups) {
        const int rc = tf_sync(c);
        if (rc != TF_OK) return efail(e, rc, std::string("member: ") + tf_last_error(c));
    }
    return TF_OK;
}

int tf_ensemble_autotune(tf_ensemble* e, int steps_per_candidate) {
    const TfRange nvtx_range("tf_ensemble_autotune");
    if (!e) return TF_ERR_ARG;
    if (steps_per_candidate < 1 || steps_per_candidate > kMaxStepsPerLaunch)
        return efail(e, TF_ERR_ARG, "steps_per_candidate must be in [1, 1024]");
    int rc = TF_OK;
    if (!members_in_step(e) && (rc = normalise(e)) != TF_OK) return rc;
    int64_t done = 0;
    if (!e->pending) {
        if ((rc = issue(e, kPrologue, 1)) != TF_OK) return rc;
        done += 1;
    }
    cudaEvent_t t0, t1;
    TF_ECK(e, cudaEventCreate(&t0));
    TF_ECK(e, cudaEventCreate(&t1));
    int best = e->cfg;
    for (int c = 0; c < kCandidates && rc == TF_OK; ++c) {
        e->cfg = c;
        cudaEventRecord(t0, e->stream);
        rc = issue(e, kSteady, steps_per_candidate);
        cudaEventRecord(t1, e->stream);
        done += steps_per_candidate;
        float ms = 0.f;
        if (rc == TF_OK && cudaEventSynchronize(t1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess)
            e->us[c] = 1e3 * ms / steps_per_candidate;
        if (e->us[c] > 0 && (e->us[best] <= 0 || e->us[c] < e->us[best])) best = c;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    e->cfg = best;
    publish(e, done);
    if (rc != TF_OK) return rc;
    return tf_ensemble_sync(e);
}

int tf_ensemble_config(const tf_ensemble* e, int* tile_y, int* ctas_per_sm, int* grid,
                       int64_t* tiles_per_step, double* us_per_step, int* graphs) {
    if (!e) return TF_ERR_ARG;
    const int ti = shape_of(e->cfg);
    const bool plans = e->cfg == kGroupPlans;
    const int g = grid_for(const_cast<tf_ensemble*>(e), kSteady, e->cfg);
    if (tile_y) *tile_y = plans ? 0 : kTileY[ti];
    if (ctas_per_sm) *ctas_per_sm = ctas_of(e->cfg);
    if (grid) *grid = g;
    if (tiles_per_step) *tiles_per_step = plans ? g : e->tiles[ti];
    if (us_per_step)
        for (int c = 0; c < kCandidates; ++c) us_per_step[c] = e->us[c];
    if (graphs) *graphs = e->graphs ? 1 : 0;
    return TF_OK;
}

int64_t tf_ensemble_launches(const tf_ensemble* e) { return e ? e->launches : -1; }

int tf_ensemble_candidate(const tf_ensemble* e) { return e ? e->cfg : TF_ERR_ARG; }

int tf_ensemble_select(tf_ensemble* e, int candidate) {
    if (!e) return TF_ERR_ARG;
    if (candidate < 0 || candidate >= kCandidates)
        return efail(e, TF_ERR_ARG, "candidate out of range");
    e->cfg = candidate;
    return TF_OK;
}

int tf_ensemble_fault_drill(tf_ensemble* e, uint32_t barrier_polls, int held_cta) {
    if (!e) return TF_ERR_ARG;
    if (held_cta < -1) return efail(e, TF_ERR_ARG, "held_cta must be -1 or a CTA index");
    e->drill_polls = barrier_polls;
    e->drill_held = held_cta;
    return TF_OK;
}

}  // extern "C"
