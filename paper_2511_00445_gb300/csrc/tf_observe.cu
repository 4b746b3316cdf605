// Initial conditions, field conversion, FP64 reductions and spectral
// observables (Sec. III initial condition; Sec. IV observables).
#include <cmath>

#include "tf_device.cuh"
#include "tf_internal.h"

namespace {

constexpr int RB = 256;  // threads per reduction / conversion block

// SplitMix64 (S. Vigna): golden-ratio increment followed by the published
// 64-bit finaliser.  Used as a counter-based generator keyed by
// (seed, field, site index).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, int field, long long idx) {
    const uint64_t key = seed ^ ((uint64_t)field << 40) ^ (uint64_t)idx;
    return (double)(splitmix64(key) >> 11) * 0x1.0p-53;
}

// Sum NV doubles over the block; thread 0 of the block gets the result in v.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sm[RB / 32][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = lane < RB / 32 ? sm[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

// Deterministic second pass: out[k] = sum_j part[j*NV + k], fixed order.
template <int NV>
__global__ void __launch_bounds__(RB) k_finish(const double* __restrict__ part, int nparts,
                                               double* __restrict__ out) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int j = threadIdx.x; j < nparts; j += RB)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += part[(long long)j * NV + k];
    block_sum<NV>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = v[k];
}

// Non-finite scan of three FP32 arrays: any NaN or Inf sets *flag to
// TF_ERR_NONFINITE unless another code is already recorded there.
__global__ void __launch_bounds__(RB)
k_scan_nonfinite(const float* __restrict__ a, long long na, const float* __restrict__ b,
                 long long nb, const float* __restrict__ c, long long nc, int* __restrict__ flag) {
    const long long total = na + nb + nc;
    const long long stride = (long long)gridDim.x * RB;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < total; i += stride) {
        const float v = i < na ? a[i] : (i < na + nb ? b[i - na] : c[i - na - nb]);
        bad |= !isfinite(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(flag, 0, TF_ERR_NONFINITE);
}

// ---------------------------------------------------------------- init
__global__ void __launch_bounds__(RB)
k_init(void* __restrict__ f, float* __restrict__ phi, float* __restrict__ Q, long long N, int b0,
       int b1, uint64_t seed, double phi0, double dphi, double S0,
       const DevParams* __restrict__ prm, int storage) {
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const double up = uniform01(seed, 0, i);
    const double ut = uniform01(seed, 1, i);
    for (int b = b0; b < b1; ++b) {
        const DevParams& P = prm[b];
        phi[b * N + i] = (float)((phi0 + dphi * (2.0 * up - 1.0)) - (double)P.phi_ref);
        double sn, cs;
        sincospi(2.0 * ut, &sn, &cs);  // 2 theta = 2 pi U
        Q[2 * b * N + i] = (float)(S0 * cs);
        Q[(2 * b + 1) * N + i] = (float)(S0 * sn);
        for (int k = 0; k < 9; ++k) {
            pop_store(f, pop_index(b, 0, k, i, N), (float)(d2q9_wd(k) * ((double)P.rho1 - 1.0)), storage);
            pop_store(f, pop_index(b, 1, k, i, N), (float)(d2q9_wd(k) * ((double)P.rho2 - 1.0)),
                      storage);
        }
    }
}

// --------------------------------------------------------- field writes
// field: 0 phi, 1 Qxx, 2 Qxy, 16+i / 32+i populations (given pre-collision
// f_i(x); stored at x - c_i in the pull layout).
__global__ void __launch_bounds__(RB)
k_write(void* __restrict__ f, float* __restrict__ phi, float* __restrict__ Q,
        const double* __restrict__ src, int nx, int ny, int b, int field,
        const DevParams* __restrict__ prm, int storage) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const double v = src[i];
    if (field == TF_FIELD_PHI) {
        phi[b * N + i] = (float)(v - (double)prm[b].phi_ref);
    } else if (field == TF_FIELD_QXX || field == TF_FIELD_QXY) {
        Q[(2 * b + (field - TF_FIELD_QXX)) * N + i] = (float)v;
    } else {
        const int fl = field >= TF_FIELD_F2 ? 1 : 0;
        const int k = field - (fl ? TF_FIELD_F2 : TF_FIELD_F1);
        const int x = (int)(i % nx), y = (int)(i / nx);
        const int sx = tfd::wrap(x - d2q9_cx(k), nx), sy = tfd::wrap(y - d2q9_cy(k), ny);
        pop_store(f, pop_index(b, fl, k, (long long)sy * nx + sx, N), (float)(v - d2q9_wd(k)), storage);
    }
}

__global__ void __launch_bounds__(RB)
k_set_eq(void* __restrict__ f, const double* __restrict__ u1, const double* __restrict__ u2,
         int nx, int ny, int b, const DevParams* __restrict__ prm, int storage) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const int x = (int)(i % nx), y = (int)(i / nx);
    for (int fl = 0; fl < 2; ++fl) {
        const double* u = fl ? u2 : u1;
        const double ux = u ? u[i] : 0.0, uy = u ? u[N + i] : 0.0;
        const double rho = fl ? (double)prm[b].rho2 : (double)prm[b].rho1;
        const double uu = ux * ux + uy * uy;
        for (int k = 0; k < 9; ++k) {
            const double cu = d2q9_cx(k) * ux + d2q9_cy(k) * uy;
            const double w = d2q9_wd(k);
            const double dev = w * (rho - 1.0) + w * rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            const int sx = tfd::wrap(x - d2q9_cx(k), nx), sy = tfd::wrap(y - d2q9_cy(k), ny);
            pop_store(f, pop_index(b, fl, k, (long long)sy * nx + sx, N), (float)dev, storage);
        }
    }
}

// ------------------------------------------------- derived flow quantities
// u_c = phi u1 + (1 - phi) u2 (component comp) at site p of instance b, FP64.
__device__ __forceinline__ double mixture_u(const float* __restrict__ phi,
                                            const float* __restrict__ mac, long long N, int b,
                                            double c, int comp, long long p) {
    const float* m = mac + 8 * b * N;
    const double pv = c + (double)phi[b * N + p];
    return pv * (double)m[comp * N + p] + (1.0 - pv) * (double)m[(comp + 2) * N + p];
}

// Periodic neighbours of site i: east, west, north, south.
struct Nbrs {
    long long e, w, n, s;
};
__device__ __forceinline__ Nbrs nbrs_of(long long i, int nx, int ny) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    Nbrs r;
    r.e = (long long)y * nx + (x + 1 < nx ? x + 1 : 0);
    r.w = (long long)y * nx + (x > 0 ? x - 1 : nx - 1);
    r.n = (long long)(y + 1 < ny ? y + 1 : 0) * nx + x;
    r.s = (long long)(y > 0 ? y - 1 : ny - 1) * nx + x;
    return r;
}

// omega_c = d_x u_c,y - d_y u_c,x, central differences.
__device__ __forceinline__ double mixture_vorticity(const float* __restrict__ phi,
                                                    const float* __restrict__ mac, int nx,
                                                    int ny, int b, double c, long long i) {
    const long long N = (long long)nx * ny;
    const Nbrs g = nbrs_of(i, nx, ny);
    return 0.5 * (mixture_u(phi, mac, N, b, c, 1, g.e) - mixture_u(phi, mac, N, b, c, 1, g.w)) -
           0.5 * (mixture_u(phi, mac, N, b, c, 0, g.n) - mixture_u(phi, mac, N, b, c, 0, g.s));
}

// Energy and flow maps of Sec. IV (Fig. 6) at site i.
__device__ double energy_map(const float* __restrict__ phi, const float* __restrict__ Q,
                             const float* __restrict__ mac, int nx, int ny, int b, long long i,
                             int field, const DevParams* __restrict__ prm) {
    const long long N = (long long)nx * ny;
    const double c = prm[b].phi_ref;
    if (field == TF_FIELD_E_ELASTIC) {
        // K/2 sum_{k,i,j} (d_k Q_ij)^2 = K sum_k [(d_k Q_xx)^2 + (d_k Q_xy)^2]
        const float* qa = Q + 2 * b * N;
        const float* qb = qa + N;
        const Nbrs g = nbrs_of(i, nx, ny);
        const double ax = 0.5 * ((double)qa[g.e] - (double)qa[g.w]);
        const double ay = 0.5 * ((double)qa[g.n] - (double)qa[g.s]);
        const double bx = 0.5 * ((double)qb[g.e] - (double)qb[g.w]);
        const double by = 0.5 * ((double)qb[g.n] - (double)qb[g.s]);
        return (double)prm[b].K * (ax * ax + ay * ay + bx * bx + by * by);
    }
    if (field == TF_FIELD_OMEGA_C) return mixture_vorticity(phi, mac, nx, ny, b, c, i);
    const double ux = mixture_u(phi, mac, N, b, c, 0, i), uy = mixture_u(phi, mac, N, b, c, 1, i);
    const double uu = ux * ux + uy * uy;
    if (field == TF_FIELD_UC_MAG) return sqrt(uu);
    const float* m = mac + 8 * b * N;
    return 0.5 * ((double)m[4 * N + i] + (double)m[5 * N + i]) * uu;   // E_kin
}

// ---------------------------------------------------------- field reads
__global__ void __launch_bounds__(RB)
k_read(const void* __restrict__ f, const float* __restrict__ phi, const float* __restrict__ Q,
       const float* __restrict__ mac, const float* __restrict__ mu, double* __restrict__ dst,
       int nx, int ny, int b, int field, const DevParams* __restrict__ prm, int storage) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    double v;
    if (field == TF_FIELD_PHI) {
        v = (double)prm[b].phi_ref + (double)phi[b * N + i];
    } else if (field == TF_FIELD_QXX || field == TF_FIELD_QXY) {
        v = (double)Q[(2 * b + (field - TF_FIELD_QXX)) * N + i];
    } else if (field >= TF_FIELD_U1X && field <= TF_FIELD_RHO2) {
        v = (double)mac[(8 * b + (field - TF_FIELD_U1X)) * N + i];
    } else if (field == TF_FIELD_MU) {
        v = (double)mu[b * N + i];
    } else if (field >= TF_FIELD_E_ELASTIC && field <= TF_FIELD_OMEGA_C) {
        v = energy_map(phi, Q, mac, nx, ny, b, i, field, prm);
    } else {
        const int fl = field >= TF_FIELD_F2 ? 1 : 0;
        const int k = field - (fl ? TF_FIELD_F2 : TF_FIELD_F1);
        const int x = (int)(i % nx), y = (int)(i / nx);
        const int sx = tfd::wrap(x - d2q9_cx(k), nx), sy = tfd::wrap(y - d2q9_cy(k), ny);
        v = d2q9_wd(k) +
            (double)pop_load(f, pop_index(b, fl, k, (long long)sy * nx + sx, N), storage);
    }
    dst[i] = v;
}

// ------------------------------------------------------ conserved sums
// Sums of the stored state of instance b: phi deviations, population
// deviations (density), momenta, non-drag forces (from the macro planes),
// non-finite count.  The sum over sites of pulled values equals the sum of
// stored values, so densities and momenta need no streaming here.
__global__ void __launch_bounds__(RB)
k_conserved(const void* __restrict__ f, const float* __restrict__ phi,
            const float* __restrict__ Q, const float* __restrict__ mac, long long N, int b,
            double* __restrict__ part, int storage) {
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        float d1[9], d2[9];
        int bad = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            d1[k] = pop_load(f, pop_index(b, 0, k, i, N), storage);
            d2[k] = pop_load(f, pop_index(b, 1, k, i, N), storage);
            bad += !isfinite(d1[k]) + !isfinite(d2[k]);
        }
        const float p = phi[b * N + i], qa = Q[2 * b * N + i], qb = Q[(2 * b + 1) * N + i];
        bad += !isfinite(p) + !isfinite(qa) + !isfinite(qb);
        double r1 = 0, r2 = 0, mx = 0, my = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            r1 += d1[k];
            r2 += d2[k];
            mx += d2q9_cx(k) * ((double)d1[k] + (double)d2[k]);
            my += d2q9_cy(k) * ((double)d1[k] + (double)d2[k]);
        }
        v[0] += p;
        v[1] += r1;
        v[2] += r2;
        v[3] += mx;
        v[4] += my;
        v[5] += mac[(8 * b + 6) * N + i];
        v[6] += mac[(8 * b + 7) * N + i];
        v[7] += bad;
    }
    block_sum<8>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) part[blockIdx.x * 8 + k] = v[k];
}

// ---------------------------------------------------- phase differences
__global__ void __launch_bounds__(RB)
k_phase(const float* __restrict__ phi, const float* __restrict__ mac, int nx, int ny, int b,
        const DevParams* __restrict__ prm, double* __restrict__ part) {
    const long long N = (long long)nx * ny;
    const float* ph = phi + b * N;
    const float* m = mac + 8 * b * N;
    const double c = prm[b].phi_ref;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const long long e = (long long)y * nx + (x + 1 < nx ? x + 1 : 0);
        const long long w = (long long)y * nx + (x > 0 ? x - 1 : nx - 1);
        const long long n = (long long)(y + 1 < ny ? y + 1 : 0) * nx + x;
        const long long s = (long long)(y > 0 ? y - 1 : ny - 1) * nx + x;
        auto U = [&](int comp, long long p) { return (double)m[comp * N + p]; };
        auto UC = [&](int comp, long long p) {
            const double pv = c + (double)ph[p];
            return pv * U(comp, p) + (1.0 - pv) * U(comp + 2, p);
        };
        const double dux = U(0, i) - U(2, i), duy = U(1, i) - U(3, i);
        const double w1 = 0.5 * (U(1, e) - U(1, w)) - 0.5 * (U(0, n) - U(0, s));
        const double w2 = 0.5 * (U(3, e) - U(3, w)) - 0.5 * (U(2, n) - U(2, s));
        const double wc = 0.5 * (UC(1, e) - UC(1, w)) - 0.5 * (UC(0, n) - UC(0, s));
        const double ucx = UC(0, i), ucy = UC(1, i);
        v[0] += dux * dux + duy * duy;
        v[1] += (w1 - w2) * (w1 - w2);
        v[2] += U(0, i) * U(0, i) + U(1, i) * U(1, i);
        v[3] += ucx * ucx + ucy * ucy;
        v[4] += w1 * w1;
        v[5] += wc * wc;
    }
    block_sum<6>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = v[k];
}

__global__ void __launch_bounds__(RB)
k_phi_moments(const float* __restrict__ phi, long long N, int b, double* __restrict__ part) {
    double v[2] = {0, 0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const double p = phi[b * N + i];
        v[0] += p;
        v[1] += p * p;
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 2] = v[0];
        part[blockIdx.x * 2 + 1] = v[1];
    }
}

// ------------------------------------------------------------------ FFT
// Load the spectral input of instance b as complex doubles (ny rows of nx):
// which 0: (phi - phi_ref, 0); which 1: (u_c,x, u_c,y).
__global__ void __launch_bounds__(RB)
k_spec_load(const float* __restrict__ phi, const float* __restrict__ mac, long long N, int b,
            int which, const DevParams* __restrict__ prm, double2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const double d = phi[b * N + i];
    if (which == 0) {
        out[i] = make_double2(d, 0.0);
    } else {
        const double pv = (double)prm[b].phi_ref + d;
        const float* m = mac + 8 * b * N;
        const double ucx = pv * m[i] + (1.0 - pv) * m[2 * N + i];
        const double ucy = pv * m[N + i] + (1.0 - pv) * m[3 * N + i];
        out[i] = make_double2(ucx, ucy);
    }
}

// Forward DFT of each row (length L, `rows` rows) in place, in shared memory.
// Power-of-two L: iterative radix-2 (bit-reversed load, butterflies);
// otherwise the direct O(L^2) sum.  Twiddles exp(-2 pi i j k / L) from sincospi.
__global__ void __launch_bounds__(RB) k_fft_rows(double2* __restrict__ data, int L) {
    extern __shared__ double2 sh[];
    double2* row = data + (long long)blockIdx.x * L;
    const bool pow2 = (L & (L - 1)) == 0;
    if (pow2) {
        int lg = 0;
        while ((1 << lg) < L) ++lg;
        for (int j = threadIdx.x; j < L; j += RB) {
            const int r = lg == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - lg));
            sh[r] = row[j];
        }
        __syncthreads();
        for (int len = 2; len <= L; len <<= 1) {
            const int half = len >> 1;
            for (int t = threadIdx.x; t < L / 2; t += RB) {
                const int grp = t / half, pos = t - grp * half;
                const int i0 = grp * len + pos, i1 = i0 + half;
                double sn, cs;
                sincospi(-2.0 * (double)pos / (double)len, &sn, &cs);
                const double2 a = sh[i0], v = sh[i1];
                const double2 bw = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
                sh[i0] = make_double2(a.x + bw.x, a.y + bw.y);
                sh[i1] = make_double2(a.x - bw.x, a.y - bw.y);
            }
            __syncthreads();
        }
        for (int j = threadIdx.x; j < L; j += RB) row[j] = sh[j];
    } else {
        for (int j = threadIdx.x; j < L; j += RB) sh[j] = row[j];
        __syncthreads();
        for (int k = threadIdx.x; k < L; k += RB) {
            double sx = 0.0, sy = 0.0;
            for (int j = 0; j < L; ++j) {
                const long long jk = ((long long)j * k) % L;
                double sn, cs;
                sincospi(-2.0 * (double)jk / (double)L, &sn, &cs);
                const double2 v = sh[j];
                sx += v.x * cs - v.y * sn;
                sy += v.x * sn + v.y * cs;
            }
            row[k] = make_double2(sx, sy);  // each k written by one thread; reads use sh
        }
    }
}

// out[c][r] = in[r][c] for an R x C matrix, 32x32 tiles.
__global__ void k_transpose(const double2* __restrict__ in, double2* __restrict__ out, int R,
                            int C) {
    __shared__ double2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[dy][threadIdx.x] = in[(long long)r * C + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(long long)c * R + r] = tile[threadIdx.x][dy];
    }
}

// Signed FFT mode number of index j of an n-point transform (numpy fftfreq * n).
__device__ __forceinline__ int signed_mode(int j, int n) { return j <= (n - 1) / 2 ? j : j - n; }

// Shell of mode (jx, jy): floor(r + 1/2) with r = sqrt((mx m/nx)^2 + (my m/ny)^2),
// m = min(nx, ny), evaluated with separately rounded IEEE operations.
__device__ __forceinline__ int shell_of(int jx, int jy, int nx, int ny) {
    const int m = nx < ny ? nx : ny;
    const double tx = __ddiv_rn((double)signed_mode(jx, nx) * m, (double)nx);
    const double ty = __ddiv_rn((double)signed_mode(jy, ny) * m, (double)ny);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)));
    return (int)floor(__dadd_rn(r, 0.5));
}

// Shell histogram of |z|^2 * scale over the transposed spectrum T[jx][jy]
// (nx rows of ny).  which 0 drops the k = 0 mode.  Per-block partials of
// n_shell + 1 entries; the last entry is the all-mode total.
__global__ void __launch_bounds__(RB)
k_shell_bin(const double2* __restrict__ T, int nx, int ny, int n_shell, double scale,
            int which, int counts_only, double* __restrict__ part) {
    extern __shared__ double hist[];
    for (int k = threadIdx.x; k <= n_shell; k += RB) hist[k] = 0.0;
    __syncthreads();
    const long long N = (long long)nx * ny;
    double total = 0.0;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const int jx = (int)(i / ny), jy = (int)(i % ny);
        double val;
        if (counts_only) {
            val = 1.0;
        } else {
            const double2 z = T[i];
            val = (z.x * z.x + z.y * z.y) * scale;
            if (which == 0 && jx == 0 && jy == 0) val = 0.0;
        }
        total += val;
        const int sh = shell_of(jx, jy, nx, ny);
        if (sh < n_shell) atomicAdd(&hist[sh], val);
    }
    double v[1] = {total};
    block_sum<1>(v);
    for (int k = threadIdx.x; k < n_shell; k += RB)
        part[(long long)blockIdx.x * (n_shell + 1) + k] = hist[k];
    if (threadIdx.x == 0) part[(long long)blockIdx.x * (n_shell + 1) + n_shell] = v[0];
}

__global__ void __launch_bounds__(RB)
k_shell_finish(const double* __restrict__ part, int nparts, int n_shell, double* __restrict__ out) {
    for (int k = blockIdx.x * RB + threadIdx.x; k <= n_shell; k += gridDim.x * RB) {
        double s = 0.0;
        for (int j = 0; j < nparts; ++j) s += part[(long long)j * (n_shell + 1) + k];
        out[k] = s;
    }
}

// ---------------------------------------------------------- correlations
// Correlated quantity of instance b as complex doubles (ny rows of nx):
// TF_CORR_U (u_c,x, u_c,y), TF_CORR_OMEGA (omega_c, 0), TF_CORR_Q (Q_xx, Q_xy).
__global__ void __launch_bounds__(RB)
k_corr_load(const float* __restrict__ phi, const float* __restrict__ Q,
            const float* __restrict__ mac, int nx, int ny, int b, int which,
            const DevParams* __restrict__ prm, double2* __restrict__ out) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const double c = prm[b].phi_ref;
    if (which == TF_CORR_U)
        out[i] = make_double2(mixture_u(phi, mac, N, b, c, 0, i), mixture_u(phi, mac, N, b, c, 1, i));
    else if (which == TF_CORR_OMEGA)
        out[i] = make_double2(mixture_vorticity(phi, mac, nx, ny, b, c, i), 0.0);
    else
        out[i] = make_double2((double)Q[2 * b * N + i], (double)Q[(2 * b + 1) * N + i]);
}

// Power of the (one or two) real components packed in z = a + i b:
// |a_hat(k)|^2 + |b_hat(k)|^2 = (|Z(k)|^2 + |Z(-k)|^2) / 2, written as (P, 0)
// in the same [jx][jy] layout (nx rows of ny).  centred: drop k = 0.
__global__ void __launch_bounds__(RB)
k_corr_power(const double2* __restrict__ T, int nx, int ny, int centred,
             double2* __restrict__ out) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const int jx = (int)(i / ny), jy = (int)(i % ny);
    const int mx = jx == 0 ? 0 : nx - jx, my = jy == 0 ? 0 : ny - jy;
    const double2 z = T[i], w = T[(long long)mx * ny + my];
    double p = 0.5 * ((z.x * z.x + z.y * z.y) + (w.x * w.x + w.y * w.y));
    if (centred && jx == 0 && jy == 0) p = 0.0;
    out[i] = make_double2(p, 0.0);
}

// Shell of displacement (rx, ry) (array positions): floor(|r| + 1/2) with the
// minimum image r, separately rounded IEEE operations.
__device__ __forceinline__ int rshell_of(int rx, int ry, int nx, int ny) {
    const double tx = (double)signed_mode(rx, nx), ty = (double)signed_mode(ry, ny);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)));
    return (int)floor(__dadd_rn(r, 0.5));
}

// Shell sums of Re R(r) and displacement counts over R[ry][rx] (ny rows of nx):
// per-block partials [2 * n_shell] (sums, then counts).
__global__ void __launch_bounds__(RB)
k_rshell_bin(const double2* __restrict__ R, int nx, int ny, int n_shell,
             double* __restrict__ part) {
    extern __shared__ double hist[];
    for (int k = threadIdx.x; k < 2 * n_shell; k += RB) hist[k] = 0.0;
    __syncthreads();
    const long long N = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const int ry = (int)(i / nx), rx = (int)(i % nx);
        const int sh = rshell_of(rx, ry, nx, ny);
        if (sh < n_shell) {
            atomicAdd(&hist[sh], R[i].x);
            atomicAdd(&hist[n_shell + sh], 1.0);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * n_shell; k += RB)
        part[(long long)blockIdx.x * 2 * n_shell + k] = hist[k];
}

// out[m] = (shell-m sum / shell-m count) / R(0), partials summed in block order.
__global__ void __launch_bounds__(RB)
k_rshell_finish(const double* __restrict__ part, int nparts, int n_shell,
                const double2* __restrict__ R, double* __restrict__ out) {
    const double r0 = R[0].x;
    for (int k = blockIdx.x * RB + threadIdx.x; k < n_shell; k += gridDim.x * RB) {
        double s = 0.0, n = 0.0;
        for (int j = 0; j < nparts; ++j) {
            s += part[(long long)j * 2 * n_shell + k];
            n += part[(long long)j * 2 * n_shell + n_shell + k];
        }
        out[k] = n > 0.0 && r0 != 0.0 ? s / n / r0 : 0.0;
    }
}

// Snapshot of instance b: u_c,x, u_c,y, omega_c, Q_xx, Q_xy (FP32 planes).
__global__ void __launch_bounds__(RB)
k_snapshot(const float* __restrict__ phi, const float* __restrict__ Q,
           const float* __restrict__ mac, int nx, int ny, int b,
           const DevParams* __restrict__ prm, float* __restrict__ snap) {
    const long long N = (long long)nx * ny;
    const long long i = (long long)blockIdx.x * RB + threadIdx.x;
    if (i >= N) return;
    const double c = prm[b].phi_ref;
    float* o = snap + 5 * b * N;
    o[i] = (float)mixture_u(phi, mac, N, b, c, 0, i);
    o[N + i] = (float)mixture_u(phi, mac, N, b, c, 1, i);
    o[2 * N + i] = (float)mixture_vorticity(phi, mac, nx, ny, b, c, i);
    o[3 * N + i] = Q[2 * b * N + i];
    o[4 * N + i] = Q[(2 * b + 1) * N + i];
}

// Sums of a(snapshot) . a(now) and |a(snapshot)|^2 for u_c, omega_c, Q:
// partials [6] = (uu', uu, ww', ww, QQ', QQ).
__global__ void __launch_bounds__(RB)
k_timecorr(const float* __restrict__ phi, const float* __restrict__ Q,
           const float* __restrict__ mac, const float* __restrict__ snap, int nx, int ny, int b,
           const DevParams* __restrict__ prm, double* __restrict__ part) {
    const long long N = (long long)nx * ny;
    const double c = prm[b].phi_ref;
    const float* o = snap + 5 * b * N;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const double ax = o[i], ay = o[N + i], aw = o[2 * N + i], aq = o[3 * N + i],
                     bq = o[4 * N + i];
        const double ux = mixture_u(phi, mac, N, b, c, 0, i), uy = mixture_u(phi, mac, N, b, c, 1, i);
        const double w = mixture_vorticity(phi, mac, nx, ny, b, c, i);
        const double qa = Q[2 * b * N + i], qb = Q[(2 * b + 1) * N + i];
        v[0] += ax * ux + ay * uy;
        v[1] += ax * ax + ay * ay;
        v[2] += aw * w;
        v[3] += aw * aw;
        v[4] += aq * qa + bq * qb;
        v[5] += aq * aq + bq * bq;
    }
    block_sum<6>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = v[k];
}

// ---------------------------------------------------------------- defects
// Winding of the doubled director angle, i.e. of the vector (Q_xx, Q_xy),
// along one edge a -> b turned by its smallest rotation: +1 when that
// rotation crosses the positive x half-axis counter-clockwise, -1 clockwise.
// a.y*b.x and a.x*b.y are exact in FP64 for FP32 inputs and the sign of
// their difference is exact, so the decision is exact.  An antiparallel pair
// (cross product 0) contributes nothing.
__device__ __forceinline__ int edge_crossing(double ax, double ay, double bx, double by) {
    const double cr = ax * by - ay * bx;
    if (ay < 0.0 && by >= 0.0 && cr > 0.0) return 1;
    if (by < 0.0 && ay >= 0.0 && cr < 0.0) return -1;
    return 0;
}

// Counts of plaquette charges +1/2, -1/2 and other nonzero (partials [3]).
__global__ void __launch_bounds__(RB)
k_defects(const float* __restrict__ Q, int nx, int ny, int b, double* __restrict__ part) {
    const long long N = (long long)nx * ny;
    const float* qa = Q + 2 * b * N;
    const float* qb = qa + N;
    double v[3] = {0, 0, 0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N;
         i += (long long)gridDim.x * RB) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const int xp = x + 1 < nx ? x + 1 : 0, yp = y + 1 < ny ? y + 1 : 0;
        const long long c[4] = {(long long)y * nx + x, (long long)y * nx + xp,
                                (long long)yp * nx + xp, (long long)yp * nx + x};
        int w = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long p = c[k], q = c[(k + 1) & 3];
            w += edge_crossing(qa[p], qb[p], qa[q], qb[q]);
        }
        // w winds the doubled angle: the charge is w / 2
        if (w == 1) v[0] += 1.0;
        else if (w == -1) v[1] += 1.0;
        else if (w != 0) v[2] += 1.0;
    }
    block_sum<3>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = v[k];
}

inline unsigned nblk(long long N) { return (unsigned)((N + RB - 1) / RB); }

}  // namespace

// ======================================================================
cudaError_t tf_launch_zero_state(tf_ctx* ctx) {
    const DevBuffers& d = ctx->d;
    const size_t N = (size_t)ctx->N, B = (size_t)ctx->batch;
    for (int k = 0; k < 2; ++k) {
        cudaMemsetAsync(d.f[k], 0, 18 * B * N * tf_pop_bytes(ctx->storage), ctx->stream);
        cudaMemsetAsync(d.phi[k], 0, B * N * sizeof(float), ctx->stream);
        cudaMemsetAsync(d.Q[k], 0, 2 * B * N * sizeof(float), ctx->stream);
        cudaMemsetAsync(d.u[k], 0, 4 * B * N * sizeof(float), ctx->stream);
    }
    return cudaGetLastError();
}

cudaError_t tf_launch_init(tf_ctx* ctx, int inst, uint64_t seed, double phi0, double dphi,
                           double S0) {
    const int b0 = inst < 0 ? 0 : inst, b1 = inst < 0 ? ctx->batch : inst + 1;
    const DevBuffers& d = ctx->d;
    k_init<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.f[ctx->fcur], d.phi[ctx->pcur],
                                                 d.Q[ctx->pcur], ctx->N, b0, b1, seed, phi0, dphi,
                                                 S0, d.prm, ctx->storage);
    return cudaGetLastError();
}

cudaError_t tf_launch_write_field(tf_ctx* ctx, int inst, int field, const double* dsrc) {
    const DevBuffers& d = ctx->d;
    k_write<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.f[ctx->fcur], d.phi[ctx->pcur],
                                                  d.Q[ctx->pcur], dsrc, ctx->nx, ctx->ny, inst,
                                                  field, d.prm, ctx->storage);
    return cudaGetLastError();
}

cudaError_t tf_launch_set_equilibrium(tf_ctx* ctx, int inst, const double* du1,
                                      const double* du2) {
    k_set_eq<<<nblk(ctx->N), RB, 0, ctx->stream>>>(ctx->d.f[ctx->fcur], du1, du2, ctx->nx,
                                                   ctx->ny, inst, ctx->d.prm, ctx->storage);
    return cudaGetLastError();
}

cudaError_t tf_launch_read_field(tf_ctx* ctx, int inst, int field, double* ddst) {
    const DevBuffers& d = ctx->d;
    if ((field >= TF_FIELD_U1X && field <= TF_FIELD_RHO2) || field == TF_FIELD_MU ||
        (field >= TF_FIELD_E_KIN && field <= TF_FIELD_OMEGA_C)) {
        cudaError_t e = tf_launch_macro(ctx, d.macro);
        if (e != cudaSuccess) return e;
    }
    k_read<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.f[ctx->fcur], d.phi[ctx->pcur], d.Q[ctx->pcur],
                                                 d.macro, d.mu, ddst, ctx->nx, ctx->ny, inst,
                                                 field, d.prm, ctx->storage);
    return cudaGetLastError();
}

cudaError_t tf_launch_conserved(tf_ctx* ctx, int inst, double* dout8) {
    const DevBuffers& d = ctx->d;
    cudaError_t e = tf_launch_macro(ctx, d.macro);
    if (e != cudaSuccess) return e;
    k_conserved<<<ctx->red_blocks, RB, 0, ctx->stream>>>(d.f[ctx->fcur], d.phi[ctx->pcur],
                                                        d.Q[ctx->pcur], d.macro, ctx->N, inst,
                                                        d.red_part, ctx->storage);
    k_finish<8><<<1, RB, 0, ctx->stream>>>(d.red_part, ctx->red_blocks, dout8);
    return cudaGetLastError();
}

cudaError_t tf_launch_phase_difference(tf_ctx* ctx, int inst, double* dout6) {
    const DevBuffers& d = ctx->d;
    cudaError_t e = tf_launch_macro(ctx, d.macro);
    if (e != cudaSuccess) return e;
    k_phase<<<ctx->red_blocks, RB, 0, ctx->stream>>>(d.phi[ctx->pcur], d.macro, ctx->nx, ctx->ny,
                                                    inst, d.prm, d.red_part);
    k_finish<6><<<1, RB, 0, ctx->stream>>>(d.red_part, ctx->red_blocks, dout6);
    return cudaGetLastError();
}

cudaError_t tf_launch_nonfinite_scan(tf_ctx* ctx) {
    const DevBuffers& d = ctx->d;
    const long long n = (long long)ctx->batch * ctx->N;
    long long blocks = (7 * n + RB * 8 - 1) / (RB * 8);
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    k_scan_nonfinite<<<(int)blocks, RB, 0, ctx->stream>>>(d.phi[ctx->pcur], n, d.Q[ctx->pcur],
                                                         2 * n, d.u[ctx->ucur], 4 * n, d.flags);
    ctx->launches += 1;
    return cudaGetLastError();
}

cudaError_t tf_launch_phi_stats(tf_ctx* ctx, int inst, double* dout2) {
    const DevBuffers& d = ctx->d;
    k_phi_moments<<<ctx->red_blocks, RB, 0, ctx->stream>>>(d.phi[ctx->pcur], ctx->N, inst,
                                                          d.red_part);
    k_finish<2><<<1, RB, 0, ctx->stream>>>(d.red_part, ctx->red_blocks, dout2);
    return cudaGetLastError();
}

static cudaError_t fft2d_to_transposed(tf_ctx* ctx) {
    // cbuf[0]: ny rows of nx  ->  cbuf[1]: nx rows of ny, fully transformed.
    const DevBuffers& d = ctx->d;
    const int nx = ctx->nx, ny = ctx->ny;
    k_fft_rows<<<ny, RB, nx * sizeof(double2), ctx->stream>>>(d.cbuf[0], nx);
    dim3 tb(32, 8), tg((nx + 31) / 32, (ny + 31) / 32);
    k_transpose<<<tg, tb, 0, ctx->stream>>>(d.cbuf[0], d.cbuf[1], ny, nx);
    k_fft_rows<<<nx, RB, ny * sizeof(double2), ctx->stream>>>(d.cbuf[1], ny);
    return cudaGetLastError();
}

cudaError_t tf_launch_spectrum(tf_ctx* ctx, int inst, int which) {
    const DevBuffers& d = ctx->d;
    if (which == 1) {
        cudaError_t e = tf_launch_macro(ctx, d.macro);
        if (e != cudaSuccess) return e;
    }
    k_spec_load<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.phi[ctx->pcur], d.macro, ctx->N, inst,
                                                      which, d.prm, d.cbuf[0]);
    cudaError_t e = fft2d_to_transposed(ctx);
    if (e != cudaSuccess) return e;
    const double invN = 1.0 / (double)ctx->N;
    const double scale = (which == 0 ? 1.0 : 0.5) * invN * invN;
    const size_t shm = (size_t)(ctx->n_shell + 1) * sizeof(double);
    k_shell_bin<<<ctx->shell_blocks, RB, shm, ctx->stream>>>(d.cbuf[1], ctx->nx, ctx->ny,
                                                             ctx->n_shell, scale, which, 0,
                                                             d.shell_part);
    k_shell_finish<<<(ctx->n_shell + RB) / RB, RB, 0, ctx->stream>>>(
        d.shell_part, ctx->shell_blocks, ctx->n_shell, d.shell_out);
    return cudaGetLastError();
}

cudaError_t tf_launch_shell_counts(tf_ctx* ctx) {
    const DevBuffers& d = ctx->d;
    const size_t shm = (size_t)(ctx->n_shell + 1) * sizeof(double);
    k_shell_bin<<<ctx->shell_blocks, RB, shm, ctx->stream>>>(d.cbuf[1], ctx->nx, ctx->ny,
                                                             ctx->n_shell, 1.0, 0, 1,
                                                             d.shell_part);
    k_shell_finish<<<(ctx->n_shell + RB) / RB, RB, 0, ctx->stream>>>(
        d.shell_part, ctx->shell_blocks, ctx->n_shell, d.shell_out);
    return cudaGetLastError();
}

// 2-D forward DFT: `in` holds `rows` rows of `cols`; the result lands in
// `out` as cols rows of `rows` (transposed).
static cudaError_t fft2d(cudaStream_t st, double2* in, double2* out, int rows, int cols) {
    k_fft_rows<<<rows, RB, cols * sizeof(double2), st>>>(in, cols);
    dim3 tb(32, 8), tg((cols + 31) / 32, (rows + 31) / 32);
    k_transpose<<<tg, tb, 0, st>>>(in, out, rows, cols);
    k_fft_rows<<<cols, RB, rows * sizeof(double2), st>>>(out, rows);
    return cudaGetLastError();
}

cudaError_t tf_launch_correlation(tf_ctx* ctx, int inst, int which, double* dout) {
    const DevBuffers& d = ctx->d;
    const int nx = ctx->nx, ny = ctx->ny;
    if (which != TF_CORR_Q) {
        cudaError_t e = tf_launch_macro(ctx, d.macro);
        if (e != cudaSuccess) return e;
    }
    k_corr_load<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.phi[ctx->pcur], d.Q[ctx->pcur], d.macro,
                                                      nx, ny, inst, which, d.prm, d.cbuf[0]);
    // cbuf[0] (ny x nx) -> cbuf[1] = spectrum [jx][jy]
    cudaError_t e = fft2d(ctx->stream, d.cbuf[0], d.cbuf[1], ny, nx);
    if (e != cudaSuccess) return e;
    k_corr_power<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.cbuf[1], nx, ny, which != TF_CORR_Q,
                                                       d.cbuf[0]);
    // The power is even in k, so its forward transform is N^2 R(r):
    // cbuf[0] (nx x ny) -> cbuf[1] = [ry][rx]
    e = fft2d(ctx->stream, d.cbuf[0], d.cbuf[1], nx, ny);
    if (e != cudaSuccess) return e;
    const size_t shm = (size_t)(2 * ctx->n_shell) * sizeof(double);
    k_rshell_bin<<<ctx->shell_blocks, RB, shm, ctx->stream>>>(d.cbuf[1], nx, ny, ctx->n_shell,
                                                              d.shell_part);
    k_rshell_finish<<<(ctx->n_shell + RB - 1) / RB, RB, 0, ctx->stream>>>(
        d.shell_part, ctx->shell_blocks, ctx->n_shell, d.cbuf[1], dout);
    return cudaGetLastError();
}

cudaError_t tf_launch_snapshot(tf_ctx* ctx, int inst) {
    const DevBuffers& d = ctx->d;
    cudaError_t e = tf_launch_macro(ctx, d.macro);
    if (e != cudaSuccess) return e;
    k_snapshot<<<nblk(ctx->N), RB, 0, ctx->stream>>>(d.phi[ctx->pcur], d.Q[ctx->pcur], d.macro,
                                                     ctx->nx, ctx->ny, inst, d.prm, d.snap);
    return cudaGetLastError();
}

cudaError_t tf_launch_time_correlation(tf_ctx* ctx, int inst, double* dout6) {
    const DevBuffers& d = ctx->d;
    cudaError_t e = tf_launch_macro(ctx, d.macro);
    if (e != cudaSuccess) return e;
    k_timecorr<<<ctx->red_blocks, RB, 0, ctx->stream>>>(d.phi[ctx->pcur], d.Q[ctx->pcur], d.macro,
                                                       d.snap, ctx->nx, ctx->ny, inst, d.prm,
                                                       d.red_part);
    k_finish<6><<<1, RB, 0, ctx->stream>>>(d.red_part, ctx->red_blocks, dout6);
    return cudaGetLastError();
}

cudaError_t tf_launch_defects(tf_ctx* ctx, int inst, double* dout3) {
    const DevBuffers& d = ctx->d;
    k_defects<<<ctx->red_blocks, RB, 0, ctx->stream>>>(d.Q[ctx->pcur], ctx->nx, ctx->ny, inst,
                                                      d.red_part);
    k_finish<3><<<1, RB, 0, ctx->stream>>>(d.red_part, ctx->red_blocks, dout3);
    return cudaGetLastError();
}

cudaError_t tf_configure_observe_kernels() {
    // The row FFT and the shell histogram may need more than 48 KB of
    // dynamic shared memory (rows up to 8192 points, up to 8192 shells).
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * (int)sizeof(double2));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rshell_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * 8193 * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_shell_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                8193 * (int)sizeof(double));
}
