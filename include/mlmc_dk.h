/*
 * mlmc_dk.h -- C-ABI of the GB300 (sm_103a) Multilevel Monte Carlo library for
 * the 2-D Dean--Kawasaki equation (Cornalba & Fischer, arXiv 2311.08872).
 *
 * What the library computes
 * -------------------------
 * For levels l = 0..L_max with n_l = n0 2^l cells per axis, h_l = length/n_l,
 * tau_l = tau_0 4^-l and M_l = M_0 4^l fine steps (Eq. cfl_preserved, Section
 * 7.2), one *sample* of level l is the pair of paths of Eq. (FullyDiscreteDK)
 * with b0 = 0, b1 = 1 (explicit Euler--Maruyama, Section 7.2):
 *     rho^{m+1} = rho^m + tau/2 Delta_h rho^m
 *                 + N^{-1/2} div_h( h^{-1} sqrt([rho^m]^+) dbeta^m ),
 * on the fine grid (h_l, tau_l) and -- for l >= 1 -- on the coarse grid
 * (h_{l-1}, tau_{l-1}) driven by the Right-Most Nearest-Neighbour coupled
 * increments of Section 3.2 (each coarse increment is 1/2 x the sum of the
 * 2x2 fine increments to its right, summed over the 4 fine steps inside one
 * coarse step).  Each path is reduced at T to Y_k = (rho^T, I_h phi_k)_h and to
 *     P = N (Y_j - Ybar_j)(Y_k - Ybar_k)          (Eq. eqn_MLMCLevels, psi = x^2;
 *                                                    j = k unless `products`),
 * where Ybar is the discrete mean field (the noise-free scheme), and the
 * library accumulates per level the moment sums of dP = P_f - P_c (P_c = 0 on
 * level 0) that the estimator of Eq. (MLMCEstimator) telescopes.
 * mlmc_dk_estimate runs Algorithm 1 (Section 7.1) with the sample allocation
 * of Eq. (opt_M_ell) and the stopping test of Eq. (convergence_criterion).
 *
 * Noise: dbeta = sqrt(tau) Z, Z from Philox4x32-10 + Box--Muller.  Sample i of
 * level l in stream s is a pure function of (seed, l, s, i): for the fine cell
 * pair p = (i1 n + i2)/2 and fine step m the counter is
 *     (p, m, i & 0xffffffff, (l+1) | s << 8 | ((i >> 32) & 0xffff) << 16),
 * key (seed & 0xffffffff, seed >> 32); words (x0,x1) feed cell 2p and (x2,x3)
 * cell 2p+1 with u = (x0+1) 2^-32, theta = 2 pi (x1 + 1/2) 2^-32,
 * Z_1 = sqrt(-2 ln u) cos theta, Z_2 = sqrt(-2 ln u) sin theta.  Stream 0 is
 * the coupled MLMC stream, stream 1 plain single-level Monte Carlo.
 *
 * Grids up to 256^2 keep each sample's state in registers for the whole run;
 * larger grids (512^2, 1024^2) stream the state of a wave of samples through
 * global memory with one launch per fine step (same arithmetic, same results).
 *
 * Grids are row-major, point (i1, i2) at (i1 h, i2 h), flat index i1 n + i2;
 * component r = 1 of the noise flux is along i1.  The library only sees the
 * caller's samples of rho-bar_0 and phi_k: sampled at (i1 + 1/2, i2 + 1/2) h
 * instead (cell-centred grids), each coarse point is the centre of its coupled
 * 2x2 block and the same kernels run the symmetric variant of the coupling
 * (Remark avoid_right_bias).
 *
 * Precision: the state is 32-bit fixed point, rho = q 2^-S_l, with S_l in
 * [16, 40] chosen per level at init as large as the initial range and the
 * expected per-cell fluctuation sqrt(rho/(N h^2)) allow.  Each step adds per-edge diffusion
 * fluxes and per-cell noise transfers (computed in FP32, rounded to integers)
 * exactly, so the mass (rho, 1)_h is conserved bit for bit and every rounding
 * error enters in divergence form; observables and moment sums are FP64.
 *
 * Ownership and errors
 * --------------------
 * The context owns all device memory it allocates and frees it in
 * mlmc_dk_free.  The caller owns every struct and array it passes (they are
 * copied or only read during the call).  Every function returning int returns
 * MLMC_DK_OK (0) on success, MLMC_DK_NOT_CONVERGED (1) when Algorithm 1 hit
 * L_max without passing the stopping test (the result is still filled), or a
 * negative MLMC_DK_ERR_* code; mlmc_dk_last_error gives the message.  No call
 * aborts the process.  All device work runs on the context's stream; calls on
 * one context must not overlap.
 */
#ifndef MLMC_DK_H
#define MLMC_DK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLMC_DK_OK 0
#define MLMC_DK_NOT_CONVERGED 1
#define MLMC_DK_ERR_INVALID (-1)     /* bad argument or configuration */
#define MLMC_DK_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define MLMC_DK_ERR_RANGE (-3)       /* |rho| reached 2^(30-S_l): the level's fixed-point range */
#define MLMC_DK_ERR_UNSUPPORTED (-4) /* grid size without a kernel variant */
#define MLMC_DK_ERR_STATE (-5)       /* checkpoint buffer does not match */
#define MLMC_DK_ERR_TIMEOUT (-6)     /* a kernel's bounded wait for another CTA's progress gave up (band, persistent streamed and tensor-core GEMM kernels) */

#define MLMC_DK_MAX_LEVELS 16
#define MLMC_DK_MAX_OBS 4
#define MLMC_DK_MAX_QUANT 10          /* 4 observables with all products j <= k */
#define MLMC_DK_NSUM 12               /* per-quantity device sums, see below */

/* Configuration (read during mlmc_dk_init, then not referenced again). */
typedef struct {
    double length;          /* torus side (1.0, or 2 pi for the paper's setting) */
    int32_t n0;             /* level-0 cells per axis: a power of two in [4, 1024] */
    int32_t L_max;          /* finest level index, n0 << L_max <= 1024 */
    double T;               /* final time */
    double cfl_mu;          /* nominal tau/h^2 (<= 1/2 for the explicit scheme): M_0 = ceil(T/(mu h0^2)),
                               tau_0 = T/M_0 */
    int32_t M0;             /* > 0: use this M_0 instead (tau_0 = T/M_0) */
    double N;               /* particle number; 0 switches the noise off */
    const double* const* rho0; /* [L_max+1] host arrays: rho0[l] = I_{h_l} rho-bar_0, n_l^2 values */
    int32_t n_obs;          /* number of test functions, 1..4 */
    const double* const* phi;  /* [(L_max+1) * n_obs] host arrays: phi[l*n_obs+k] = I_{h_l} phi_k */
    int32_t products;       /* 0: one quantity per phi_k; 1: all pairs j <= k (n_obs(n_obs+1)/2) */
    int32_t pilot;          /* Algorithm 1 initial samples per level (0 -> 256) */
    int32_t L_start;        /* Algorithm 1 initial finest level (0 -> 2, capped at L_max) */
    void* cuda_stream;      /* cudaStream_t for all device work, or NULL (legacy default stream) */
    int32_t stream_from_n;  /* 0: stream the state only where no register kernel exists (n >= 512);
                               k > 0: also for every level with n >= k (n a multiple of 64) */
    double theta_b0;        /* implicit weight b0 in [0, 1] of Eq. (FullyDiscreteDK), b1 = 1 - b0
                               (Definition 2.1): (I - b0 tau/2 Delta_h) rho^m = (I + b1 tau/2 Delta_h)
                               rho^(m-1) + noise.  0: explicit Euler--Maruyama (Section 7.2).  b0 > 0
                               runs every level on the theta-scheme kernel (n0 2^L_max <= 128, no
                               stream_from_n; a 128^2 level runs on clusters of 4 CTAs per sample); cfl_mu may then exceed 1/2 up to the scheme's
                               stability bound 1 / (2 (b1 - b0)) (none for b0 >= 1/2), with
                               b0 cfl_mu <= 10 */
    int32_t theta_kernel;   /* 1: run b0 = 0 on the theta-scheme kernel too (the same integer
                               arithmetic as the explicit kernels); 0: default */
    int32_t coupling;       /* 0: Right-Most Nearest-Neighbour coupling (Section 3.2), h_{l-1} = 2 h_l,
                               tau_{l-1} = 4 tau_l; 1: Fourier coupling (Section 3.1), h_{l-1} = 3 h_l,
                               tau_{l-1} = 9 tau_l: the coarse noise of a coarse step carries every
                               Fourier mode of the summed fine noise that the coarse grid resolves (the
                               coarse Nyquist mode takes its two fine aliases with weight 2^-1/2 each).
                               Fourier: n0 = 6, L_max <= 3 (grids 6^2, 18^2, 54^2, 162^2; a 162^2
                               level runs on clusters of 6 CTAs per sample), explicit scheme,
                               level n_l = n0 3^l, M_l = M_0 9^l; rho0 / phi arrays on those grids */
    int32_t state_repr;     /* representation of the fixed-point state (Eq. FullyDiscreteDK is linear apart
                               from sqrt([rho]^+), so both give the same scheme):
                               1: absolute, q = rho 2^S_l;
                               2: fluctuation about the noise-free path, q = (rho - rho-bar^m) 2^S_l, with
                                  rho-bar^m (m = 0..M_l - 1) kept in a per-level FP32 table on the device and the
                                  transfers G = rint(c 2^S sqrt([rho-bar^m + q 2^-S]^+) Z); S_l then only has to
                                  cover 12 standard deviations of the per-cell fluctuation, i.e. many more
                                  fraction bits at large N.  Explicit hierarchies with N > 0: NN with grids up
                                  to 128^2 (register kernels), Fourier with grids up to 54^2 (one CTA per
                                  sample); tables <= 512 MB; else MLMC_DK_ERR_UNSUPPORTED;
                               0: automatic -- fluctuation where it is supported and gains at least 3 bits on
                                  every level, absolute otherwise */
} mlmc_dk_config;

/* Per-level description returned by mlmc_dk_level_info. */
typedef struct {
    int32_t level, n, M;    /* fine cells per axis and fine steps */
    double h, tau;          /* fine mesh size and step */
    double ybar_f[MLMC_DK_MAX_OBS];  /* (rho-bar^T, phi_k)_h on the fine grid */
    double ybar_c[MLMC_DK_MAX_OBS];  /* same on the coarse grid (level >= 1) */
    double cost;            /* cell-steps per coupled sample: n_l^2 M_l + n_{l-1}^2 M_{l-1} */
    double cost_mc;         /* cell-steps per plain MC sample: n_l^2 M_l */
    int64_t next_sample;    /* first sample id the next mlmc_dk_run_level call uses */
    int64_t h2d_bytes;      /* bytes mlmc_dk_init uploaded for all levels (pinned staging) */
    int32_t frac_bits;      /* S_l: the level's fixed-point state is rho 2^S_l */
    int32_t n_variants;     /* kernel variants (lane-block shapes, cluster sizes) for this grid size */
    int32_t variant_single, variant_coupled;  /* variants in use for the fine-only and the coupled kernel */
    int32_t lane_cols, lane_rows, cluster;    /* the level's main kernel: C x R coarse cells per lane, cluster */
    int32_t streamed;       /* 1: grid too large for registers; state streamed through global memory */
    int32_t in_flight;      /* streamed path: samples advanced together (their state fits L2); on a
                               split-capable level, those of its streamed share */
    int32_t tile_rows;      /* streamed path: fine rows per CTA tile of the variant in use (tiles are
                               tile_rows x 64 fine cells); 0 for the register kernels */
    int32_t split_capable;  /* 1: a register level (n >= 256, 8-SM clusters) whose batch samples can be
                               shared with the streamed kernels (mlmc_dk_set_batch_split) */
    double split_fraction;  /* share of this level's batch samples run on the streamed kernels */
    int64_t batch_streamed; /* samples of the last multi-level batch that ran on the streamed kernels */
    int32_t theta;          /* 1: the level runs on the theta-scheme kernel */
    double theta_b0;        /* its implicit weight b0 */
    int32_t cheb_steps;     /* Chebyshev steps per implicit solve (0: none) */
    int32_t coupling;       /* 0: NN, 1: Fourier (as configured) */
    int32_t fluct;          /* 1: fluctuation state (frac_bits is then the fluctuation's S_l) */
    int32_t band;           /* 1: the level's kernel in use spreads each sample over `bands` CTAs (full-width
                               bands of coarse rows in registers, band edges exchanged through global memory;
                               in_flight samples per launch) */
    int32_t bands;
    int32_t persistent;     /* 1: the level's streamed kernel in use runs each wave of in_flight samples as one
                               launch whose CTAs take (tile, step) items in order from a counter and wait, with
                               bounded polls, for the items they read from; 0: one launch per step */
    int32_t pdl;            /* 1: the level's streamed kernel in use launches each step as a programmatic dependent
                               launch of the previous one (its Philox words are drawn before it waits for it) */
} mlmc_dk_level_desc;

/* Host-side moment sums of one quantity on one level (accumulated into). */
typedef struct {
    int64_t n;                    /* samples */
    double dp1, dp2, dp3, dp4;    /* sum of dP, dP^2, dP^3, dP^4 (dP = P_f - P_c) */
    double pf1, pf2;              /* sum of P_f, P_f^2 */
    double pc1, pc2;              /* sum of P_c, P_c^2 (0 on level 0 and for plain MC) */
    double yf1, yf2;              /* sum of (Y_f - Ybar_f), its square (first observable of the quantity) */
    double yc1, yc2;              /* same for the coarse path */
    double max_mass_err;          /* max |(rho^T,1)_h - (rho^0,1)_h| over the samples (exactly 0 expected) */
    double cost;                  /* cell-steps performed */
    double wall_s;                /* wall time of the calls that produced the samples */
    double kernel_s;              /* device time of their level kernels (CUDA events on the launching stream) */
    int64_t launches;             /* kernels launched (level kernel + fixed-order reduction per call) */
    int64_t d2h_bytes;            /* bytes read back to the host (sums and the device error word) */
} mlmc_dk_level_sums;

/* Result of Algorithm 1. */
typedef struct {
    double estimate;              /* mu_MLMC of the first quantity, Eq. (MLMCEstimator) */
    double variance;              /* sum_l V_l / M_l */
    double eps_abs;               /* absolute RMSE target used */
    int32_t L;                    /* finest level reached */
    int32_t converged;            /* 1 if the stopping test passed */
    int64_t M[MLMC_DK_MAX_LEVELS];
    double V[MLMC_DK_MAX_LEVELS], E[MLMC_DK_MAX_LEVELS], C[MLMC_DK_MAX_LEVELS];
    double estimates[MLMC_DK_MAX_QUANT];   /* mu_MLMC of every quantity */
    double sample_steps;          /* coupled sample-steps performed (sum of M_l x fine steps) */
    double cell_steps;            /* fine + coarse cell-steps performed */
    double wall_s;
    double kernel_s[MLMC_DK_MAX_LEVELS];   /* device time of each level's kernels */
    double var_pf[MLMC_DK_MAX_LEVELS];     /* sample variance of P_l from the level-l fine paths */
    int64_t launches;             /* kernels launched */
    int64_t d2h_bytes;            /* bytes read back to the host */
} mlmc_dk_result;

typedef struct mlmc_dk_ctx mlmc_dk_ctx;   /* opaque */

/* Validate `cfg`, build the level table, compute on the host the discrete
 * mean field rho-bar^T of every level (FFT diagonalisation of the noise-free
 * scheme) and its pairings with phi, and upload the per-level tables (fixed
 * point initial states and mean fields, FP32 test functions) to the device.
 * Errors: MLMC_DK_ERR_INVALID (mu > 1/2, n0 not a power of two, sizes out of
 * range, |rho0| >= 64, null arrays), MLMC_DK_ERR_CUDA.  On error *out is NULL
 * and the message is available from mlmc_dk_last_error(NULL). */
int mlmc_dk_init(const mlmc_dk_config* cfg, mlmc_dk_ctx** out);

/* Release all device and host memory of the context (NULL is a no-op). */
void mlmc_dk_free(mlmc_dk_ctx* ctx);

/* Message of the last failed call on ctx (ctx == NULL: last failure of
 * mlmc_dk_init in this thread).  Owned by the library, valid until the next
 * call on the same context. */
const char* mlmc_dk_last_error(const mlmc_dk_ctx* ctx);

/* Fill *out with the level table entry of `level` (0..L_max). */
int mlmc_dk_level_info(const mlmc_dk_ctx* ctx, int32_t level, mlmc_dk_level_desc* out);

/* Run n_samples coupled samples of level `level` (P_l - P_{l-1}; P_0 on level
 * 0) with ids next_sample .. next_sample+n_samples-1 under `seed`, and add
 * their moment sums into sums[q] for every quantity q (caller-allocated host
 * array of n_quant structs).  Advances next_sample.  Synchronous: returns
 * after the device work and the copy of the sums to the host. */
int mlmc_dk_run_level(mlmc_dk_ctx* ctx, int32_t level, int64_t n_samples, uint64_t seed,
                      mlmc_dk_level_sums* sums);

/* Same for plain single-level Monte Carlo samples of P_l (stream 1, fine
 * path only; sample ids 0..n_samples-1 after the previous MC call on that
 * level). */
int mlmc_dk_run_mc(mlmc_dk_ctx* ctx, int32_t level, int64_t n_samples, uint64_t seed,
                   mlmc_dk_level_sums* sums);

/* Device-resident batch: samples first_sample .. first_sample+n_samples-1 of
 * `level` in `stream_tag` (0 coupled, 1 plain MC) under `seed`.  Writes (not
 * accumulates) into device memory:
 *   sums_dev:    double[2 + n_quant * MLMC_DK_NSUM]: [0] sample count,
 *                [1] max mass error, then per quantity
 *                {dp1..dp4, pf1, pf2, pc1, pc2, yf1, yf2, yc1, yc2};
 *   samples_dev: NULL, or double[n_samples][2 n_obs + 2]: Y_f-Ybar_f (n_obs),
 *                Y_c-Ybar_c (n_obs, 0 without a coarse path), mass_f, mass_c.
 * Both must be 8-byte aligned device pointers.  Asynchronous on `cuda_stream`
 * (NULL: the context's stream); does not touch next_sample.  The scratch it
 * needs (per-slot partial sums) is owned by the context. */
int mlmc_dk_run_level_dev(mlmc_dk_ctx* ctx, int32_t level, int32_t stream_tag,
                          int64_t first_sample, int64_t n_samples, uint64_t seed,
                          double* sums_dev, double* samples_dev, void* cuda_stream);

/* Multi-level batch: counts[l] coupled samples of every level l = 0..L_max
 * (0 skips the level), sample ids first_sample.. on every level, under
 * `seed`.  The levels run concurrently, each on its own stream and scratch,
 * finest level first with the most urgent launch priority so that its
 * thread-block clusters are placed before the coarser levels fill the SMs the
 * clusters leave free; the whole fork/join is captured into a CUDA graph and
 * replayed (re-instantiated only when the batch's shape changes).  Writes
 * sums_dev[l * (2 + n_quant*MLMC_DK_NSUM) ...] for every level in the layout of
 * mlmc_dk_run_level_dev (zeros for skipped levels).  Asynchronous on
 * cuda_stream (NULL: the context's stream); does not touch next_sample; must
 * not be called while cuda_stream is being captured. */
int mlmc_dk_run_batch_dev(mlmc_dk_ctx* ctx, const int64_t* counts, int64_t first_sample, uint64_t seed,
                          double* sums_dev, void* cuda_stream);

/* Device time (ms) of each level's kernels in the last completed multi-level
 * batch, from CUDA events recorded on that level's stream inside the graph
 * (ms[0..L_max]; 0 for levels the batch skipped or never ran).  On a split
 * level this is the register kernels' share only. */
int mlmc_dk_batch_level_ms(mlmc_dk_ctx* ctx, double* ms);

/* Batch split.  The 8-SM thread-block clusters of the 256^2 (and larger
 * register) levels cannot use every SM (152 SMs hold 15 such clusters), and
 * once the coarser levels of a batch are done those SMs idle.  With
 * `fraction` > 0 the multi-level batch runs the last floor(fraction *
 * counts[level]) sample ids of `level` on the streamed-state kernels (same
 * samples, same fixed-point paths) on the least urgent stream beside the
 * graph, and adds their sums to the level's (entry 1 by max).  level in
 * 1..L_max, fraction in [0, 1/2]; MLMC_DK_ERR_UNSUPPORTED unless
 * level_info.split_capable (fraction 0 is always accepted). */
int mlmc_dk_set_batch_split(mlmc_dk_ctx* ctx, int32_t level, double fraction);

/* Autotuner of the batch split: on the finest split-capable level with
 * counts[l] > 1, times the whole batch `counts` (sample ids from 0, results
 * discarded; CUDA events on the context's stream; one untimed warm-up run,
 * then `repeats` timed runs per candidate) for fractions 0, 0.04, 0.06, 0.08,
 * 0.10, 0.12 and keeps the fastest (a larger share only when it is at least
 * 1% faster).  Tune on the batch that will run: the best share depends on its
 * size.  *fraction and *seconds (optional) receive the choice and the tuning
 * time. */
int mlmc_dk_tune_batch(mlmc_dk_ctx* ctx, const int64_t* counts, int32_t repeats, double* fraction, double* seconds);

/* Host form of the multi-level batch: ids start at the largest next_sample
 * over the levels (then next_sample = that + counts[l] on every level run);
 * sums[l * n_quant + q] receives level l, quantity q.  Synchronous. */
int mlmc_dk_run_batch(mlmc_dk_ctx* ctx, const int64_t* counts, uint64_t seed, mlmc_dk_level_sums* sums);

/* Same batch as mlmc_dk_run_level_dev, for callers that must not allocate
 * device memory when they run it: processes that hand out all of their GPU
 * memory from a pool reserved at start-up and may not allocate afterwards,
 * and latency-critical loops in which cudaMalloc/cudaFree (which synchronise
 * the device) are not allowed.  This call allocates nothing and uses none of
 * the context's device buffers except its read-only level tables: the per-slot
 * partial sums go to a statically allocated device array of 4 MiB that every
 * GPU loading the library keeps until the process exits.  The paper has no
 * counterpart of this entry point.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, with the device current); make that first call
 *     before any stream capture on that device.
 *   - All calls share the array and it keeps the last call's contents; the
 *     kernel overwrites every entry it later reads, so nothing needs clearing.
 *     Calls that overlap on the GPU (other streams, other host threads, other
 *     contexts) race on the array and corrupt each other's sums: serialise them.
 *   - The grid is limited to the sample slots whose partial sums fit the array
 *     (at least one CTA's worth; otherwise MLMC_DK_ERR_INVALID), so a call may
 *     keep fewer samples in flight than mlmc_dk_run_level_dev.  Per-sample
 *     values are identical; the sums agree up to FP64 summation order.
 *   - err_dev: NULL, or a caller-owned device word that receives the range
 *     error bit (1) by atomic OR; with NULL, range errors are not reported.
 * Outputs and alignment as mlmc_dk_run_level_dev; asynchronous on cuda_stream
 * (NULL: the context's stream); the context is not modified. */
int mlmc_dk_run_level_static(const mlmc_dk_ctx* ctx, int32_t level, int32_t stream_tag, int64_t first_sample,
                             int64_t n_samples, uint64_t seed, double* sums_dev, double* samples_dev,
                             unsigned int* err_dev, void* cuda_stream);

/* Failure-detection test of the band kernel's bounded waits (the paper has no
 * counterpart): one sample of `level` (>= 1) over at most 64 fine steps on the
 * band kernel, with every wait limited to `polls` polls and band `stall_band`
 * never publishing its edges, so that its neighbours' waits run out.  The
 * kernel records the timeout, every CTA stops stepping, and the call returns
 * MLMC_DK_ERR_TIMEOUT; the context stays usable.  MLMC_DK_ERR_UNSUPPORTED
 * when the level does not run on the band kernel. */
int mlmc_dk_band_wait_test(mlmc_dk_ctx* ctx, int32_t level, uint32_t polls, int32_t stall_band);

/* Failure-detection test of the persistent streamed kernel's bounded waits
 * (the paper has no counterpart): one sample of streamed `level` over at most
 * 64 fine steps on the persistent streamed kernel, with every wait limited to
 * `polls` polls and fine tile `stall_tile` never reporting its step 1, so that
 * the waits for it run out.  The kernel records the timeout, every CTA stops
 * at its next item, and the call returns MLMC_DK_ERR_TIMEOUT; the context
 * stays usable.  MLMC_DK_ERR_UNSUPPORTED when the level is not streamed. */
int mlmc_dk_stream_wait_test(mlmc_dk_ctx* ctx, int32_t level, uint32_t polls, int32_t stall_tile);

/* Algorithm 1 (Section 7.1): start at L = L_start with `pilot` samples on
 * levels 0..L; repeat {run the missing samples (all levels of a round at once
 * through the multi-level batch, ids continuing each level's range from 0),
 * re-estimate V_l, set targets by
 * Eq. (opt_M_ell), once no level needs samples apply Eq.
 * (convergence_criterion) with alpha = 2 and add a level if it fails}.  The
 * first quantity drives the allocation; eps is absolute, or relative to the
 * pilot estimate |mu| when `relative` is nonzero (frozen after the pilot).
 * Returns MLMC_DK_OK, MLMC_DK_NOT_CONVERGED (L_max reached) or an error. */
int mlmc_dk_estimate(mlmc_dk_ctx* ctx, double eps, int32_t relative, uint64_t seed,
                     mlmc_dk_result* out);

/* Algorithm 1 over several processes, host-only (no context, no GPU needed).
 * The same algorithm as mlmc_dk_estimate (which runs it on one process with
 * the multi-level batch): start at L = L_start with `pilot` (>= 2) samples on
 * levels 0..L; every round, the missing samples of level l, ids
 * next_l .. target_l - 1, are cut into `world` contiguous pieces and piece
 * `rank` is run here by
 *     run_round(user, L, first, count, sums):
 *         count[l] samples of level l with ids first[l].. (0 <= l <= L_max;
 *         count 0 for levels to skip); write their sums into sums
 *         [(L_max + 1) * (2 + 12 n_quant)] in the layout of
 *         mlmc_dk_run_level_dev (zeros for skipped levels; the buffer arrives
 *         zeroed); return 0, or nonzero to stop with MLMC_DK_ERR_INVALID;
 * then, with world > 1,
 *     reduce(user, sums, L_max + 1, 2 + 12 n_quant):
 *         combine the round's sums over all processes in place (sum; entry 1
 *         of each level, the mass error, by max); return 0 on success.
 * Every process then takes the same decisions (Eq. opt_M_ell with the
 * costs cost[l] of one sample of level l, Eq. convergence_criterion with
 * alpha = 2 and mesh ratio `ratio`), so the result does not depend on the
 * number of processes up to FP64 summation order.  eps is absolute, or
 * relative to the pilot estimate when `relative` is nonzero.  Fills
 * estimate(s), variance, eps_abs, L, converged, M, E, V, C, cell_steps,
 * var_pf and wall_s of *out.  Returns MLMC_DK_OK, MLMC_DK_NOT_CONVERGED
 * (L_max reached) or MLMC_DK_ERR_INVALID. */
typedef int (*mlmc_dk_round_fn)(void* user, int32_t L, const int64_t* first, const int64_t* count, double* sums);
typedef int (*mlmc_dk_reduce_fn)(void* user, double* sums, int64_t n_levels, int64_t stride);
int mlmc_dk_algorithm1(int32_t L_max, int32_t L_start, int64_t pilot, int32_t n_quant, const double* cost,
                       double ratio, double eps, int32_t relative, int32_t rank, int32_t world,
                       mlmc_dk_round_fn run_round, mlmc_dk_reduce_fn reduce, void* user, mlmc_dk_result* out);

/* Choose kernel variant `variant` (0 .. n_variants-1, see mlmc_dk_level_info)
 * for level `level`'s coupled (coupled = 1, level >= 1) or fine-only kernel.
 * All variants compute the same fixed-point paths bit for bit (hence equal
 * masses); the observables differ only by the order of their FP32 partial
 * sums.  Variants differ in how many cells a lane owns and how many SMs share
 * a sample; on streamed levels, in the resident CTAs per SM of the fine-step
 * kernel (4, or 5 with at most 48 registers per thread). */
int mlmc_dk_set_variant(mlmc_dk_ctx* ctx, int32_t level, int32_t coupled, int32_t variant);

/* Autotuner: for every level and kernel with more than one variant, time each
 * variant (CUDA events, `repeats` timed launches of two full waves of sample
 * slots after a warm-up launch -- on streamed levels one wave of samples in
 * flight over 64 fine steps; sample ids from 0, results discarded) and keep
 * the fastest per sample.  *seconds (optional) receives the tuning time. */
int mlmc_dk_tune(mlmc_dk_ctx* ctx, int32_t repeats, double* seconds);

/* ---- Learned level below level 0 (an addition; the paper has no such level).
 * Features of a level-0 sample: its normals projected on the 32 lowest real
 * orthonormal grid modes e_j (cosine and sine per wave vector, ordered by
 * |k|^2), weighted by the noise-free scheme's per-step factor g_j on each mode
 * carried to T: F_(j,r) = sum_m g_j^(M-1-m) <Z^m_(.,r), e_j>, standardised by
 * their exact standard deviation (they are i.i.d. N(0, sum_i g_j^(2i))).  A
 * 64-256-256-256-K ReLU perceptron (K = n_obs outputs; BF16 tensor-core
 * GEMMs, FP32 accumulation and master weights) maps them to
 * That_k ~ sqrt(N) (Y_0k - Ybar_0k); S_jl = That_j That_l stands in for the
 * quantity P_0,jl (j = l without `products`).  The estimate telescopes
 *     E[P_L] = E[S] + E[P_0 - S] + sum_{l>=1} E[P_l - P_{l-1}],
 * where the level below 0 draws its standardised features directly as
 * standard normals (stream 2, level tag 0) and the correction level evaluates
 * S on the features of the very noise that drives its level-0 path; the sum is
 * unbiased for any network.  Requires a level-0 grid of 8^2..32^2 (so not the
 * Fourier coupling's 6^2).  With the theta-scheme g_j is its factor
 * (1 - b1 lam_j)/(1 + b0 lam_j); the constant factor 1/(1 + b0 lam_j) through
 * which each step's noise reaches the mode cancels in the standardisation.
 * Parameters: flat FP32 vector of 148224 + 257 K values
 * (mlmc_dk_surrogate_info), per layer W [out][in] row-major then b [out]. */
int mlmc_dk_surrogate_init(mlmc_dk_ctx* ctx, uint64_t seed);   /* He-uniform weights, zero biases */
int mlmc_dk_surrogate_params(mlmc_dk_ctx* ctx, float* theta_out, const float* theta_in);  /* get and/or set */
/* Number of network parameters and outputs (K = n_obs) of an initialised learned level. */
int mlmc_dk_surrogate_info(const mlmc_dk_ctx* ctx, int32_t* n_params, int32_t* n_outputs);
/* Standardised features (host float[n][64], n <= 65536) of samples first..
 * of level 0 in stream `stream_tag` (direct = 0), or the direct draws of the
 * level below 0 (direct = 1). */
int mlmc_dk_surrogate_features(mlmc_dk_ctx* ctx, int32_t direct, int32_t stream_tag, int64_t first, int64_t n,
                               uint64_t seed, float* X_host);
/* Network outputs y_host[n][K] of the feature rows X_host[n][64] (n <= 65536). */
int mlmc_dk_surrogate_forward(mlmc_dk_ctx* ctx, const float* X_host, int64_t n, float* y_host);
/* Squared error of the network on (X, T) (T [B][K], B <= 4096 rows), summed
 * over the outputs and averaged over the rows, and its gradient (host float
 * [n_params], same layout as the parameters). */
int mlmc_dk_surrogate_loss_grad(mlmc_dk_ctx* ctx, const float* X_host, const float* T_host, int32_t B, double* loss,
                                float* grad_host);
/* Train on n_pairs level-0 paths of the training stream (3): targets
 * sqrt(N)(Y_0k - Ybar_0k), Adam (beta 0.9, 0.999), cosine-decayed step size,
 * minibatches of `batch` (a multiple of 64, <= 4096), the last 1/16 held out.
 * Outputs the last batch's and the held-out errors (the loss above). */
int mlmc_dk_surrogate_train(mlmc_dk_ctx* ctx, int64_t n_pairs, int32_t epochs, int32_t batch, double lr, uint64_t seed,
                            double* train_mse, double* val_mse, double* seconds);
/* n samples of the level below 0 (part = -1: dP = S) or of the correction
 * level (part = 0: dP = P_0 - S, P_f = P_0, P_c = S), added into
 * sums[0 .. n_quant-1], one per quantity (consecutive sample ids per part). */
int mlmc_dk_run_surrogate(mlmc_dk_ctx* ctx, int32_t part, int64_t n_samples, uint64_t seed, mlmc_dk_level_sums* sums);
/* Algorithm 1 over {level below 0, correction level, levels 1..L}, costs =
 * measured device seconds per sample, allocation by the first quantity;
 * result arrays index 0 = correction level, l = level l; estimates[q] per
 * quantity; the level below 0's sums of the first quantity go to
 * *surrogate_level. */
int mlmc_dk_estimate_surrogate(mlmc_dk_ctx* ctx, double eps, int32_t relative, uint64_t seed, mlmc_dk_result* out,
                               mlmc_dk_level_sums* surrogate_level);

/* Host-only planning step of Algorithm 1 for levels 0..L: from per-level
 * sample counts n[l], sums s1[l] = sum dP and s2[l] = sum dP^2 and costs
 * cost[l], compute target[l] by Eq. (opt_M_ell) (never below n[l]) and
 * *converged by Eq. (convergence_criterion) with alpha = 2.  Needs n[l] >= 2. */
int mlmc_dk_plan(int32_t L, const int64_t* n, const double* s1, const double* s2,
                 const double* cost, double eps, int64_t* target, int32_t* converged);

/* The same for a level hierarchy with mesh ratio `ratio` (> 1): the stopping
 * test max_t ratio^(-t alpha) |E_{L-t}| / (ratio^alpha - 1) < eps / sqrt 2 (the
 * printed test has ratio 2; the Fourier coupling's levels refine by 3).
 * mlmc_dk_estimate uses the context's ratio. */
int mlmc_dk_plan_ratio(int32_t L, const int64_t* n, const double* s1, const double* s2, const double* cost,
                       double eps, double ratio, int64_t* target, int32_t* converged);

/* Host-only discrete mean field: the noise-free scheme with mesh h and step
 * tau iterated M times from rho0 (n x n, n even), in FP64: by FFT
 * diagonalisation when n is a power of two, by M direct stencil steps
 * otherwise (the Fourier coupling's grids).  out may alias rho0. */
int mlmc_dk_mean_field_host(int32_t n, double h, double tau, int64_t M, const double* rho0, double* out);

/* The same for the theta-scheme's weights (b0, 1 - b0) of Eq. (FullyDiscreteDK):
 * every discrete Fourier mode is multiplied by (1 - b1 lam)/(1 + b0 lam) per
 * step (n a power of two). */
int mlmc_dk_mean_field_theta_host(int32_t n, double h, double tau, int64_t M, double b0, const double* rho0,
                                  double* out);

/* Host-only Chebyshev schedule of the theta-scheme's implicit solve
 * (I + alpha L) u = b, L = -h^2 Delta_h, alpha = b0 tau / (2 h^2): *K steps
 * (the first with 1/T_K((1+4 alpha)/(4 alpha)) <= 2^-27; 0 for alpha = 0) and the
 * direction recurrence d <- c1[k] d + c2[k] r (c1, c2: caller arrays of 64
 * floats) of Chebyshev acceleration, started with u = 0, r = b,
 * d = r / (1 + 4 alpha).  MLMC_DK_ERR_UNSUPPORTED if K would exceed 64. */
int mlmc_dk_chebyshev_schedule_host(double alpha, int32_t* K, float* c1, float* c2);

/* Host-only restriction matrix of the Fourier coupling (Section 3.1) along one
 * axis: P1 [n/3][n] (caller array, row-major) with the coarse normal field of
 * a coarse step P1 S P1^T / 3 for S the sum of its 9 fine normal fields; n a
 * multiple of 6. */
int mlmc_dk_fourier_restriction_host(int32_t n, float* P1);

/* Checkpoint: the per-level next sample ids (coupled and MC).  With
 * buf == NULL, *len receives the size needed.  Results stay a pure function
 * of (seed, level, stream, sample id), so a restored context continues the
 * same sample sequence bit for bit. */
int mlmc_dk_save_state(const mlmc_dk_ctx* ctx, void* buf, size_t* len);
int mlmc_dk_load_state(mlmc_dk_ctx* ctx, const void* buf, size_t len);

/* The standard normals Z of fine step m of sample `sample` on an n x n grid
 * (n even), exactly as the level kernel generates them in registers (see the
 * counter layout above; Definition 2.1 asks for independent increments per
 * cell and component).  z_dev: NULL or device float[n*n][2]; raw_dev: NULL or
 * device uint32[n*n/2][4], the Philox4x32-10 words of each cell pair.  Both
 * 16-byte aligned.  Asynchronous on cuda_stream.  Needs no context. */
int mlmc_dk_noise_dev(uint64_t seed, int32_t level, int32_t stream_tag, int64_t sample, int32_t m, int32_t n,
                      float* z_dev, uint32_t* raw_dev, void* cuda_stream);

/* Number of quantities (n_obs, or n_obs(n_obs+1)/2 with products). */
int32_t mlmc_dk_num_quantities(const mlmc_dk_ctx* ctx);

/* Library version string (static). */
const char* mlmc_dk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_DK_H */
