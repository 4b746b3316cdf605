/*
 * twofluid.h -- C ABI of the GB300 two-fluid active-nematic / passive-fluid
 * lattice solver (Ahmed, Lin & Qu, "Phase separation dynamics and active
 * turbulence in a binary fluid mixture", arXiv 2511.00445).
 *
 * One coupled lattice time step (Sec. II model, Sec. III scheme):
 *   - forces from phi^n, Q^n: chemical potential mu = A_ch f'(phi) - kappa
 *     lap(phi) (Eq. 2), molecular field H (Eq. 7-8), elastic stress (Sec. II
 *     display after Eq. 6), active force div(zeta phi Q), capillary force
 *     mu grad(phi) - grad(phi mu) (Eq. 10);
 *   - two D2Q9 BGK lattice-Boltzmann fluids with Guo forcing, coupled by the
 *     drag gamma phi (1-phi)(u2 - u1) (Eq. 4-5), taken implicitly inside the
 *     Guo half-force velocity (a 2x2 solve per site);
 *   - n_sub forward-Euler finite-difference sub-steps (Sec. III: five per
 *     lattice step) of Cahn-Hilliard (Eq. 1/3) and Beris-Edwards (Eq. 11-12)
 *     with the step's velocities frozen;
 *   - periodic boundaries in x and y for every field.
 *
 * Conventions for every entry point:
 *   - Lattice units: dx = dt_LBM = 1, c_s^2 = 1/3; the FD sub-steps advance
 *     by dt_fd = dt / n_sub each (tf_params.dt, 1 for lattice units).
 *   - A context holds `batch` independent instances (e.g. a parameter sweep)
 *     that share nx, ny and n_sub; each instance has its own tf_params.
 *   - Host arrays are row-major (y, x): element (x, y) at index y*nx + x, in
 *     double precision, nx*ny entries, caller-owned.
 *   - Device memory: the caller allocates ONE device workspace of at least
 *     tf_workspace_bytes() bytes (256-byte aligned) and keeps it alive until
 *     tf_destroy().  The library never allocates or frees device memory.
 *   - `stream` is a cudaStream_t passed as void*; all device work of a
 *     context is ordered on it.  tf_step() is asynchronous; entry points that
 *     fill host arrays synchronise the stream before returning.
 *   - Every function returns TF_OK (0) or a negative TF_ERR_* code; the
 *     message of the last failure is available from tf_last_error().  No
 *     C++ exception crosses this boundary and no kernel traps.
 *   - A context (and an ensemble, a surrogate) is used by one host thread at
 *     a time; different contexts may be used from different threads.
 */
#ifndef TWOFLUID_H
#define TWOFLUID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TF_OK             0
#define TF_ERR_ARG       (-1)  /* invalid argument (sizes, ids, null pointers)   */
#define TF_ERR_CUDA      (-2)  /* a CUDA runtime call or kernel launch failed    */
#define TF_ERR_NONFINITE (-3)  /* NaN or Inf found in the state                  */
#define TF_ERR_TIMEOUT   (-4)  /* a bounded device wait ran out                  */
#define TF_ERR_IO        (-5)  /* checkpoint file could not be read or written   */
#define TF_ERR_WORKSPACE (-6)  /* workspace missing, too small or misaligned     */
#define TF_ERR_TOO_LARGE (-7)  /* input larger than a fixed-footprint entry point accepts */
#define TF_ERR_BOUNDS    (-8)  /* an index check of the bounds-check build failed
                                  (libtwofluid_bc.so only; see tf_sync)          */

/* ---- field ids for tf_read_field / tf_write_field -------------------- */
#define TF_FIELD_PHI   0   /* concentration phi of the active fluid (r/w)        */
#define TF_FIELD_QXX   1   /* Q_xx (Q is traceless symmetric, Q_yy = -Q_xx) (r/w) */
#define TF_FIELD_QXY   2   /* Q_xy (r/w)                                         */
#define TF_FIELD_U1X   3   /* Guo velocity of fluid 1 (read only, derived)      */
#define TF_FIELD_U1Y   4
#define TF_FIELD_U2X   5   /* Guo velocity of fluid 2 (read only, derived)      */
#define TF_FIELD_U2Y   6
#define TF_FIELD_RHO1  7   /* density of fluid 1 (read only, derived)            */
#define TF_FIELD_RHO2  8   /* density of fluid 2 (read only, derived)            */
#define TF_FIELD_MU    9   /* chemical potential mu (read only, derived)         */
/* Energy and flow maps of Sec. IV (Fig. 6), read only, derived; u_c = phi u1 +
 * (1 - phi) u2, central differences, FP64 from the stored FP32 state: */
#define TF_FIELD_E_ELASTIC 10 /* K/2 |grad Q|^2 over all four entries of Q          */
#define TF_FIELD_E_KIN     11 /* 1/2 (rho1 + rho2) |u_c|^2, local densities         */
#define TF_FIELD_UC_MAG    12 /* |u_c|                                              */
#define TF_FIELD_OMEGA_C   13 /* omega_c = d_x u_c,y - d_y u_c,x                    */
#define TF_FIELD_F1   16   /* + i (i = 0..8): pre-collision population f_i of fluid 1 (r/w) */
#define TF_FIELD_F2   32   /* + i (i = 0..8): pre-collision population f_i of fluid 2 (r/w) */
/* D2Q9 direction order: c0 = (0,0); c1..c4 = (1,0), (0,1), (-1,0), (0,-1);
 * c5..c8 = (1,1), (-1,1), (-1,-1), (1,-1). */

/* ---- storage precision of the populations ---------------------------- */
/* The device keeps each population as its deviation d_i = f_i - w_i from the
 * rest equilibrium of unit density (w_i the D2Q9 weights).  All arithmetic
 * is FP32 whatever the storage; only the stored value is rounded.  The paper
 * (Sec. III) computes in one precision throughout; the 16-bit modes have no
 * counterpart there. */
#define TF_STORE_F32   0   /* FP32 d_i                                              */
#define TF_STORE_F16   1   /* FP16 of d_i * 2^12 (round to nearest even); the
                              exact power-of-two scale keeps |d_i| from 1.5e-8 up
                              in the normal range; |d_i| must stay below 16      */
#define TF_STORE_BF16  2   /* BF16 of d_i (round to nearest even)                  */

/* Per-instance parameters (Sec. III parameter list; lattice units). */
typedef struct tf_params {
    int    nx, ny;      /* grid size, >= 1 each; identical for all instances    */
    int    n_sub;       /* FD sub-steps per lattice step (Sec. III: 5), 1..64   */
    int    storage;     /* TF_STORE_*                                           */
    double tau1, tau2;  /* BGK relaxation times (> 1/2); nu_k = (tau_k - 1/2)/3 */
    double rho1, rho2;  /* rest densities of the initial equilibrium           */
    double gamma;       /* drag coefficient (Eq. 4-5)                          */
    double zeta;        /* activity (F_active = div(zeta phi Q))               */
    double lambda;      /* tumbling parameter (Eq. 12, elastic stress)         */
    double K;           /* Frank elastic constant (Eq. 8)                      */
    double Gamma_Q;     /* rotational diffusion Gamma (Eq. 11)                 */
    double A_Q, C_Q;    /* Landau-de Gennes coefficients (Eq. 8; B drops in 2D)*/
    double M;           /* Cahn-Hilliard mobility (Eq. 1)                      */
    double A_ch;        /* double-well prefactor: f -> A_ch phi^2 (1-phi)^2    */
    double kappa;       /* eps^2 of Eq. (2)                                    */
    double phi_ref;     /* reference value phi is stored relative to (use the
                           mean concentration, e.g. 0.5)                        */
    double dt;          /* duration of one lattice step in the time unit of the
                           Cahn-Hilliard and Beris-Edwards rates; each of the
                           n_sub sub-steps advances them by dt / n_sub (Sec.
                           III: five FD updates per lattice step).  1 reads the
                           rates in lattice units (the default reading); the
                           printed dt = 0.02 is the literal one.  > 0, finite */
    int    check_every; /* 0: off.  k > 0: tf_step scans the latest phi, Q and
                           velocity planes after every k-th lattice step (counted
                           by tf_step_count) for NaN / Inf and records
                           TF_ERR_NONFINITE in the context's device status word,
                           which the next tf_sync returns; no host
                           synchronisation, no device trap.  Taken from params[0]
                           for the whole context.                              */
} tf_params;

typedef struct tf_ctx tf_ctx;   /* opaque, library-owned host object */

/* Bytes of device workspace needed for `batch` instances described by
 * params[0..batch-1].  Returns 0 when the parameters are invalid. */
size_t tf_workspace_bytes(const tf_params* params, int batch);

/* Create a context over caller-owned device memory.  `params` holds `batch`
 * entries (copied).  `d_workspace` must be 256-byte aligned and at least
 * tf_workspace_bytes(params, batch) bytes.  The state starts zeroed (all
 * populations at the rest equilibrium w_i, phi = phi_ref, Q = 0). */
int tf_create(const tf_params* params, int batch, void* d_workspace,
              size_t workspace_bytes, void* stream, tf_ctx** out);
int tf_destroy(tf_ctx* ctx);
const char* tf_last_error(const tf_ctx* ctx);

/* Initial condition of Sec. III with the director form of Eq. (9):
 * phi = phi0 + dphi (2U - 1), theta = pi U', Q_xx = S0 cos 2theta,
 * Q_xy = S0 sin 2theta, populations at the rest equilibrium (u = 0) with
 * densities rho1, rho2.  U, U' are SplitMix64 counter draws keyed by
 * (seed, field id 0 / 1, site index y*nx + x).  inst = -1: all instances,
 * each with the same seed.  Asynchronous. */
int tf_init_fields(tf_ctx* ctx, int inst, uint64_t seed, double phi0,
                   double dphi, double S0);

/* Overwrite a stored field of one instance from a host array (synchronous).
 * Writable: TF_FIELD_PHI, QXX, QXY and the 18 populations.  Values are
 * rounded to FP32 and, for a population under a 16-bit storage mode, then
 * to that mode (the population arrays hold f_i itself, not d_i). */
int tf_write_field(tf_ctx* ctx, int inst, int field, const double* host);

/* Set both fluids' populations to the equilibrium with rest densities
 * rho1, rho2 and the given velocities (host arrays of 2*nx*ny doubles laid
 * out as [component x/y][y][x]; NULL means zero).  Synchronous. */
int tf_set_equilibrium(tf_ctx* ctx, int inst, const double* u1, const double* u2);

/* Read one field of one instance into a host array of nx*ny doubles.
 * Derived fields (velocities, densities, mu) are evaluated on the current
 * state exactly as the next step would evaluate them.  A population reads
 * back as w_i + (its stored deviation widened to FP32).  Synchronous. */
int tf_read_field(tf_ctx* ctx, int inst, int field, double* host);

/* Advance every instance by n >= 0 coupled lattice steps.  Asynchronous on
 * the context stream; launch errors are returned, execution errors are
 * reported by the next synchronising call. */
int tf_step(tf_ctx* ctx, int64_t n);

/* Kernel of the steady-state steps (five sub-steps per step).  Both compute
 * bitwise the same trajectory; they differ in schedule:
 *   TF_KERNEL_TILE:  one CTA per 2-D tile (up to 40 x 30 sites) with a 12-site
 *                    halo, the five sub-steps on shrinking neighbourhoods;
 *   TF_KERNEL_STRIP: one CTA per column strip (up to 96 columns) and row
 *                    segment, walked down in blocks of 8 rows with the five
 *                    sub-steps pipelined two rows apart (needs nx % 4 == 0);
 *   TF_KERNEL_AUTO:  the strip kernel when the context's 32 x 32 tiles exceed
 *                    one wave of resident CTAs, nx % 4 == 0 and its strips x
 *                    row segments (segments of at least 32 rows) fill at
 *                    least 90% of one wave (e.g. 1024^2, 2048^2, 4 x 512^2),
 *                    else the tile kernel.
 * tf_set_step_kernel takes effect from the next step (TF_ERR_ARG for an
 * unknown kind, or TF_KERNEL_STRIP on a context it cannot step);
 * tf_step_kernel returns TF_KERNEL_TILE or TF_KERNEL_STRIP, the kernel the
 * next steady-state step launches (planning it if needed), or a negative
 * TF_ERR_* code. */
#define TF_KERNEL_AUTO  0
#define TF_KERNEL_TILE  1
#define TF_KERNEL_STRIP 2
int tf_set_step_kernel(tf_ctx* ctx, int kind);
int tf_step_kernel(tf_ctx* ctx);

/* Wait for the context stream; returns TF_ERR_CUDA on an execution error,
 * else the device status word if a kernel set it since the last tf_sync
 * (TF_ERR_TIMEOUT: a bounded device wait ran out; TF_ERR_NONFINITE: the
 * check_every scan found NaN or Inf), clearing it. */
int tf_sync(tf_ctx* ctx);

/* Number of lattice steps taken since the last init / load. */
int64_t tf_step_count(const tf_ctx* ctx);

/* Number of CUDA kernels this context has launched so far (all entry points). */
int64_t tf_kernel_launches(const tf_ctx* ctx);

/* FP64 global sums of one instance (8 doubles, synchronous):
 *   [0] sum phi, [1] sum rho1, [2] sum rho2,
 *   [3] sum (m1 + m2)_x, [4] sum (m1 + m2)_y   (bare momenta sum_i c_i f_i),
 *   [5] sum (G1 + G2)_x, [6] sum (G1 + G2)_y   (non-drag forces of this state),
 *   [7] number of non-finite stored values.
 * Guo forcing gives sum m(n+1) - sum m(n) = sum G(n) exactly.
 * Returns TF_ERR_NONFINITE (after filling out) when [7] > 0. */
#define TF_NCONS 8
int tf_conserved(tf_ctx* ctx, int inst, double out[TF_NCONS]);

/* Spectral observables of one instance (Sec. IV).  Transforms are
 * g_hat(k) = (1/(nx ny)) sum_x g(x) exp(-i k.x), k = 2 pi (n_x/nx, n_y/ny);
 * shell m collects modes with |k|/k0 in [m - 1/2, m + 1/2), k0 = 2 pi /
 * min(nx, ny), m = 0 .. tf_n_shell()-1 (corner modes beyond are dropped).
 * All arithmetic in FP64.  Synchronous. */
int tf_n_shell(const tf_ctx* ctx);
/* out[m] = number of modes in shell m. */
int tf_shell_counts(tf_ctx* ctx, double* out, int n_shell);
/* S[m] = shell sum of |phi_hat|^2 of phi - <phi> (Eq. 24; Phi(k) of Eq. 27 is S/2). */
int tf_structure_factor(tf_ctx* ctx, int inst, double* S, int n_shell);
/* L = sum_{m>=1} Phi_m / sum_{m>=1} k_m Phi_m, k_m = m k0 (Eq. 27). */
int tf_length_scale(tf_ctx* ctx, int inst, double* L);
/* E[m] = 1/2 shell sum of |u_c_hat|^2 (Eq. 22), u_c = phi u1 + (1-phi) u2;
 * *E_total = 1/2 sum over all modes = <|u_c|^2>/2 (Eq. 29). */
int tf_energy_spectrum(tf_ctx* ctx, int inst, double* E, int n_shell, double* E_total);

/* Inter-phase differences and RMS values (Sec. IV, Fig. 8), 6 doubles:
 * [0] rms|u1 - u2|, [1] rms(w1 - w2), [2] rms|u1|, [3] rms|u_c|,
 * [4] rms w1, [5] rms w_c; w = d_x u_y - d_y u_x (central differences). */
int tf_phase_difference(tf_ctx* ctx, int inst, double out[6]);

/* Standard deviation Delta of phi (Sec. IV, Fig. 3) and its mean. */
int tf_phi_stats(tf_ctx* ctx, int inst, double* mean, double* stddev);

/* Spatial correlation functions (Sec. IV) of
 *   TF_CORR_U: delta u_c = u_c - <u_c>,  TF_CORR_OMEGA: delta omega_c,
 *   TF_CORR_Q: Q, with a(0) . a(r) = Q(0):Q(r) (uncentred).
 * C[m] = mean over the displacements r of shell m of R(r) / R(0), with
 * R(r) = <a(x) . a(x + r)>_x; r is the minimum image in lattice units and
 * shell m collects floor(|r| + 1/2) = m, m = 0 .. tf_n_shell()-1 (longer
 * displacements are dropped).  FP64 through the FFT (Wiener-Khinchin).
 * Synchronous; n_shell must equal tf_n_shell(). */
#define TF_CORR_U     0
#define TF_CORR_OMEGA 1
#define TF_CORR_Q     2
int tf_correlation(tf_ctx* ctx, int inst, int which, double* C, int n_shell);

/* Temporal correlation functions (Sec. IV).  tf_snapshot keeps u_c, omega_c
 * and Q of one instance (FP32, in the workspace) as the reference time tau;
 * tf_time_correlation returns out = [C_uu(t), C_ww(t), C_QQ(t)] =
 * <a(tau) . a(tau + t)> / <|a(tau)|^2> (uncentred) against the current
 * state; TF_ERR_ARG when the instance has no snapshot.  Synchronous. */
int tf_snapshot(tf_ctx* ctx, int inst);
int tf_time_correlation(tf_ctx* ctx, int inst, double out[3]);

/* Topological defects of the director field (Sec. IV, winding number
 * method): around every plaquette (x, y) -> (x+1, y) -> (x+1, y+1) ->
 * (x, y+1) the director turns along each edge by its smallest rotation (a
 * headless line: angles within (-pi/2, pi/2)); the total over 2 pi is the
 * charge.  out = [number of +1/2, number of -1/2, number of other nonzero
 * charges (only exact ties)]; the defect density is (out[0] + out[1]) /
 * (nx ny).  Decided exactly: only signs of FP64 products of the stored FP32
 * Q values enter.  Synchronous. */
int tf_defects(tf_ctx* ctx, int inst, int64_t out[3]);

/* Reynolds number of Sec. IV: Re = rho_c u_c,rms L_a / eta_c with
 * rho_c = rho1 + rho2 (rest densities), eta_c = eta1 + eta2, eta_k =
 * rho_k (tau_k - 1/2) / 3 (lattice units) and L_a = sqrt(K / |zeta|);
 * zeta = 0 gives Re = L_a = +inf.  The coarsening-arrest scale L_c is the
 * caller's time average of tf_length_scale.  Synchronous. */
int tf_reynolds(tf_ctx* ctx, int inst, double* Re, double* L_a);

/* Raw state (populations, phi, Q of every instance) as one byte blob in
 * the device storage layout.  tf_state_bytes() gives its size. */
size_t tf_state_bytes(const tf_ctx* ctx);

/* End-to-end entry point with HOST buffers: copy the raw state from
 * `h_in` (ideally pinned; NULL keeps the device state), advance n steps,
 * copy the raw state to `h_out` (NULL skips), and synchronise.  Both buffers
 * hold tf_state_bytes(ctx) bytes.  On a batch of several instances with
 * n_sub = 5 the call is pipelined per instance: the upload of instance b + 1
 * and the download of instance b - 1 overlap the steps of instance b, on
 * streams the context owns (forked from and joined back to its stream).  An
 * instance's piece of `h_in` is read before its piece of `h_out` is written,
 * so the two may be one buffer.  Results are bitwise those of the
 * unpipelined sequence. */
int tf_advance_host(tf_ctx* ctx, const void* h_in, int64_t n, void* h_out);

/* Checkpoint / resume of the whole context (header + raw state), bitwise. */
int tf_save(tf_ctx* ctx, const char* path);
int tf_load(tf_ctx* ctx, const char* path);

/* Tile plan of the fused per-context kernel (n_sub = 5); host-side only, no
 * device call.  For `batch` instances of nx x ny sites and `slots` resident
 * CTAs (SMs x CTAs per SM; contexts take it from the occupancy of the narrow
 * kernel, two per SM on GB300) it writes out[0] = 1 for the wide geometry
 * (tiles of at most 40 x 30 sites, used when the 32 x 32 tiles of all
 * instances exceed one wave) or 0 for the narrow one (at most 32 x 32),
 * out[1] = tile columns and out[2] = tile rows per instance.  Tile row r
 * spans rows [r ny / out[2], (r + 1) ny / out[2]) (integer division); column
 * tile k spans [col_start[k], col_start[k + 1]).  `col_start` may be NULL;
 * otherwise it must hold cap >= out[1] + 1 entries.  TF_ERR_ARG on a bad
 * argument. */
int tf_plan_tiles(int nx, int ny, int batch, long long slots, int out[3], int* col_start,
                  int cap);

/* ---- ensembles: several contexts stepped together ----------------------- */
/* The paper explores its parameters (activity zeta, tumbling lambda, Frank
 * constant K; Sec. IV) through many separate runs; it has no counterpart to
 * this batching layer.  An ensemble steps several contexts ("groups", each a
 * batch of instances sharing one grid size) together, in one of three launch
 * shapes its autotuner chooses from (tf_ensemble_autotune): a persistent
 * cooperative kernel over a ragged work-list of tiles that CTAs take in turn
 * from an atomic counter, one launch running many steps separated by a grid
 * barrier (every wait in it is bounded; a wait that runs out stops the launch
 * and reports TF_ERR_TIMEOUT through the members' tf_sync); one launch per
 * step over the tiles of every group; or each group's own per-context
 * launches, the groups on parallel branches (streams forked from and joined
 * back to the ensemble's stream), so that their launches overlap.  A launch
 * shape seen before is replayed from a cached CUDA graph.
 *
 * The ensemble does not own the members' state: between ensemble calls the
 * members' own entry points (tf_read_field, observables, tf_save, ...) see
 * the current state, and reads complete pending sub-steps exactly as for a
 * context stepped alone (trajectories are bitwise the same either way).
 * Members must not be stepped through tf_step or tf_advance_host, nor
 * destroyed, while the ensemble exists. */
typedef struct tf_ensemble tf_ensemble;
#define TF_ENS_MAX_GROUPS 64
#define TF_ENS_CANDIDATES 9    /* autotuner candidates, see tf_ensemble_autotune */

/* Device workspace bytes for an ensemble of n_groups (1..64) groups; 0 when
 * n_groups is out of range. */
size_t tf_ensemble_workspace_bytes(int n_groups);

/* Group n_groups contexts.  Every member must use n_sub = 5 (the fused
 * step), the same storage mode, and `stream` as its stream.  Pending
 * sub-steps of the members are completed first.  `d_workspace`: at least
 * tf_ensemble_workspace_bytes(n_groups) bytes, 256-byte aligned, caller-owned,
 * alive until tf_ensemble_destroy.  Starts with tile height 32 and two CTAs
 * per SM. */
int tf_ensemble_create(tf_ctx* const* groups, int n_groups, void* d_workspace,
                       size_t workspace_bytes, void* stream, tf_ensemble** out);
int tf_ensemble_destroy(tf_ensemble* ens);
const char* tf_ensemble_last_error(const tf_ensemble* ens);

/* Advance every member instance by n >= 0 steps: an LBM-only first pass
 * when the members hold a completed state, then the remaining steps as one
 * persistent launch (candidates 0..5 of tf_ensemble_autotune), as one launch
 * per step covering every tile of every group (candidates 6, 7), or as each
 * group's own per-context launches (candidate 8), up to 1024 steps per launch
 * or per recorded graph.  Asynchronous on the ensemble's stream. */
int tf_ensemble_step(tf_ensemble* ens, int64_t n);

/* Wait for the ensemble's work and report the members' device status
 * (TF_ERR_TIMEOUT after a bounded wait ran out). */
int tf_ensemble_sync(tf_ensemble* ens);

/* Launch-shape autotuner over TF_ENS_CANDIDATES candidates.  Candidate
 * k = 0..5: one persistent cooperative launch for all steps (a grid barrier
 * between steps, populations read through L2), tile shape (columns x rows)
 * {32 x 32, 32 x 24, 40 x 30}[k/2] with {2, 1}[k%2] resident CTAs per SM.
 * Candidates 6 and 7: one launch per step with one CTA per tile of every
 * group (populations read through L1, as in per-context stepping), tile
 * shape 32 x 32 and 40 x 30.  40-column tiles cut columns at multiples of 4,
 * up to 40 wide.  Candidate 8: per step, each group's own per-context launch
 * (the strip or tile kernel its plan picks, see tf_set_step_kernel), recorded
 * into the same graph.  Each candidate runs `steps_per_candidate` (1..1024) real
 * steps timed with CUDA events; the fastest becomes the configuration.  Every
 * candidate computes bitwise the same trajectory, so the tuning steps are
 * ordinary steps: the ensemble advances by TF_ENS_CANDIDATES *
 * steps_per_candidate steps (plus the first pass if one is due).
 * Synchronous. */
int tf_ensemble_autotune(tf_ensemble* ens, int steps_per_candidate);

/* Current configuration: tile height (30 means the 40 x 30 shape; 0 for
 * candidate 8), CTAs per SM, grid size of one launch (of the persistent
 * launch, tiles per step for candidates 6, 7, all groups' CTAs per step for
 * candidate 8), tiles per step; us_per_step (may be NULL) receives the
 * TF_ENS_CANDIDATES autotuner timings in microseconds per step (0 before
 * tf_ensemble_autotune).  *graphs = 1 when launches replay CUDA graphs, 0
 * when they are issued directly (stream capture unavailable). */
int tf_ensemble_config(const tf_ensemble* ens, int* tile_y, int* ctas_per_sm, int* grid,
                       int64_t* tiles_per_step, double* us_per_step, int* graphs);

/* Kernel launches issued by this ensemble so far (a graph replay counts the
 * kernels it holds). */
int64_t tf_ensemble_launches(const tf_ensemble* ens);

/* The candidate in use (0 .. TF_ENS_CANDIDATES - 1, see tf_ensemble_autotune;
 * 0 after tf_ensemble_create), or TF_ERR_ARG for a null ensemble. */
int tf_ensemble_candidate(const tf_ensemble* ens);

/* Use candidate `candidate` from the next tf_ensemble_step on (results do not
 * depend on it).  TF_ERR_ARG when it is out of range. */
int tf_ensemble_select(tf_ensemble* ens, int candidate);

/* Failure-detection drill for the persistent launch's grid barrier (candidates
 * 0..5; launches of candidates 6..8 have no grid barrier) (no fault
 * is injected on the device: a CTA just leaves early).  From the next
 * tf_ensemble_step on, the barrier gives up after `barrier_polls` polls of
 * ~128 ns each (0 restores the default of about one second) and, when
 * held_cta >= 0, that CTA of each steady-state launch of two or more steps
 * returns at the first grid barrier without arriving (it has no bulk copy in
 * flight there).  The other CTAs' bounded waits then run out: they record
 * TF_ERR_TIMEOUT in the first member's status word, raise the launch's abort
 * word and return, so tf_ensemble_sync reports TF_ERR_TIMEOUT and the members'
 * state is left partly stepped (initialise or load it again).  The drill
 * stays on until called again with (0, -1).  TF_ERR_ARG for held_cta < -1. */
int tf_ensemble_fault_drill(tf_ensemble* ens, uint32_t barrier_polls, int held_cta);

/* ---- learned surrogate: a U-Net that advances a state by many steps ---- */
/* The paper has no learned component; this layer is a convolutional
 * surrogate of the coupled step: from (phi, Q_xx, Q_xy, u1, u2) at time t of
 * one instance (plus its activity zeta as a constant input plane) it predicts
 * the fields at t + horizon, trained on pairs the solver itself produces,
 * with the plain method as the reference for its error (observables above).
 *
 * Network (NHWC activations in BF16, FP32 master weights and accumulation):
 * `levels` U-Net levels with C_l = base_channels * 2^l channels; per level two
 * 3x3 convolutions with circular padding (the lattice is periodic) + ReLU;
 * 2x2 average pooling down, nearest-neighbour upsampling up, skip
 * concatenation [upsampled, skip], and a 1x1 head to 7 outputs.  Inputs:
 * 8 channels, the 7 fields normalised per channel by the dataset's mean and
 * standard deviation and zeta / max|zeta|; outputs: the 7 increments
 * x(t + horizon) - x(t), normalised the same way.  The 3x3 convolutions,
 * their input gradients and their weight gradients run as tcgen05 tensor-
 * core GEMMs; Adam updates the FP32 weights.  Loss: mean squared error of the
 * normalised increments.
 *
 * Flat parameter vector (tf_sur_set_weights / tf_sur_get_weights /
 * tf_sur_gradients): for every 3x3 convolution in order (encoder level 0 ..
 * levels-1, two each; then decoder level levels-2 .. 0, two each) its weights
 * W[out][ky][kx][in] (tap (ky, kx) reads the input at (y + ky - 1,
 * x + kx - 1)) and biases b[out]; then the head W[7][C_0] and b[7]. */
typedef struct tf_surrogate tf_surrogate;
typedef struct tf_sur_config {
    int levels;         /* 1..5                                                  */
    int base_channels;  /* C_0: 16, 32 or 64                                     */
    int nx, ny;         /* lattice size: multiples of 8 * 2^(levels-1)           */
    int max_batch;      /* minibatch capacity, >= 1                              */
    int max_pairs;      /* training-pair capacity, >= 1                          */
    int horizon;        /* lattice steps one prediction spans, >= 1              */
} tf_sur_config;
#define TF_SUR_IN   8   /* phi - phi_ref, Q_xx, Q_xy, u1x, u1y, u2x, u2y, zeta */
#define TF_SUR_OUT  7

size_t tf_sur_workspace_bytes(const tf_sur_config* cfg);   /* 0 if cfg is invalid */
int tf_sur_create(const tf_sur_config* cfg, void* d_workspace, size_t workspace_bytes,
                  void* stream, tf_surrogate** out);
int tf_sur_destroy(tf_surrogate* s);
const char* tf_sur_last_error(const tf_surrogate* s);
int64_t tf_sur_num_params(const tf_surrogate* s);

/* Weights: He-normal initialisation from a seeded SplitMix64 stream, or a
 * copy of `n` FP32 values in the flat order above (host arrays). */
int tf_sur_init_weights(tf_surrogate* s, uint64_t seed);
int tf_sur_set_weights(tf_surrogate* s, const float* host, int64_t n);
int tf_sur_get_weights(tf_surrogate* s, float* host, int64_t n);

/* Direct access for checks: `x` holds batch x ny x nx x 8 normalised inputs
 * (host, FP32, rounded to BF16 on upload), `target` batch x ny x nx x 7.
 * tf_sur_forward writes the batch x ny x nx x 7 outputs; tf_sur_gradients the
 * loss and the flat gradient of the loss with respect to the weights.
 * Synchronous. */
int tf_sur_forward(tf_surrogate* s, const float* x, int batch, float* out);
int tf_sur_gradients(tf_surrogate* s, const float* x, const float* target, int batch,
                     double* loss, float* grad, int64_t n);

/* Training data from a solver context with the same nx, ny (it must share
 * the surrogate's stream): which = 0 stores instance `inst`'s current fields
 * as the input of pair `slot`, which = 1 as its target; the caller advances
 * the context by `horizon` steps in between.  tf_sur_fit_normalisation
 * derives the per-channel statistics from pairs 0 .. n_pairs-1. */
int tf_sur_add_pair(tf_surrogate* s, int slot, tf_ctx* ctx, int inst, int which);
int tf_sur_fit_normalisation(tf_surrogate* s, int n_pairs);

/* `steps` Adam steps (learning rate lr, betas 0.9 / 0.999) on minibatches of
 * `batch` pairs drawn from 0 .. n_pairs-1 by a seeded SplitMix64 stream;
 * losses[i] (may be NULL) receives the loss of step i.  Synchronous. */
int tf_sur_train(tf_surrogate* s, int n_pairs, int steps, int batch, double lr, uint64_t seed,
                 double* losses);

/* Advance instance `inst` of `ctx` (inst = -1: every instance, predicted as
 * one batch of at most max_batch) by `horizon` steps with the network: phi
 * and Q are replaced by the prediction and the populations by the
 * equilibrium of the rest densities and the predicted u1, u2.  The context's
 * step count (one counter for all its instances) is unchanged.  Asynchronous
 * on the shared stream. */
int tf_sur_predict(tf_surrogate* s, tf_ctx* ctx, int inst);

/* Prediction judged by the plain method: instance `inst` of `ctx` is copied
 * into the same instance of `shadow` (a context of the same shape and
 * storage on the same stream), `shadow` advances every instance by
 * `horizon` plain steps, and `ctx`'s instance is predicted.  The relative
 * errors of the prediction against the solver, err_L = |L_pred - L| / L (Eq. 27)
 * and err_E = sum_m |E_pred(m) - E(m)| / sum_m E(m) (Eq. 22), decide: above
 * max_err_L or max_err_E the instance falls back to the solver's state.
 * out = [err_L, err_E, L_pred, L]; *fell_back = 1 after a fallback, else 0.
 * The judge costs a plain run of `horizon` steps: call it for a sample of the
 * predictions.  Synchronous. */
int tf_sur_judged_predict(tf_surrogate* s, tf_ctx* ctx, tf_ctx* shadow, int inst,
                          double max_err_L, double max_err_E, double out[4], int* fell_back);

/* ---- fixed-footprint entry point ------------------------------------- */
/* The paper has no counterpart to this call; it exists for integration.
 *
 * Every other entry point works inside the workspace the caller handed to
 * tf_create.  Some callers cannot provide device memory at the moment they
 * need an answer: a plug-in living inside a host application whose memory
 * pool owns the whole device, or a time-critical loop where cudaMalloc (which
 * may synchronise the device, and fails once a framework's caching allocator
 * has reserved the memory) is not allowed.  tf_phi_stats_noalloc gives such
 * callers the concentration statistics of tf_phi_stats without any allocation:
 * it calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Input: d_values, a device array of n FP32 values v_i (for example the
 * stored deviations phi - phi_ref of a concentration field).  Output: d_out, a
 * device array of 2 doubles receiving mean = phi_ref + <v> and the standard
 * deviation sqrt(<(v - <v>)^2>) of v, in FP64: every block of 4096 values
 * contributes its mean and its sum of squared deviations (two passes), and
 * these are merged pairwise in a fixed order (Chan, Golub & LeVeque), so v
 * need not be centred.  The call only enqueues work on `stream` (a
 * cudaStream_t passed as void*); synchronise before reading d_out.
 *
 * Scratch: the library keeps TF_NOALLOC_MAX_BLOCKS x 2 doubles (16 KiB) of
 * per-block partials in one statically allocated device array, held by every
 * GPU that loads the library until the process exits.  n is limited to
 * TF_NOALLOC_MAX_ELEMS (4 194 304, e.g. one 2048 x 2048 field); larger n
 * returns TF_ERR_TOO_LARGE, n <= 0 or a null pointer TF_ERR_ARG.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * may load the library's device code there, so make it before any stream
 * capture.  All calls share the array: two calls whose kernels overlap on
 * the GPU (different streams, or different host threads on one device) race
 * and may return wrong values. */
#define TF_NOALLOC_MAX_BLOCKS 1024
#define TF_NOALLOC_MAX_ELEMS  (4096LL * TF_NOALLOC_MAX_BLOCKS)
int tf_phi_stats_noalloc(const float* d_values, long long n, double phi_ref,
                         double* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TWOFLUID_H */
