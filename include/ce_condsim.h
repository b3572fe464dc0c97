/*
 * ce_condsim.h -- C ABI of the GB300 (sm_103a) library for circulant-embedding
 * conditional simulation of a stationary Gaussian field on a regular grid,
 * given noisy observations at irregularly spaced sites.
 *
 * Method: Bailey, Bandyopadhyay & Nychka, "Adapting conditional simulation
 * using circulant embedding for irregularly spaced spatial data"
 * (arXiv 2109.11044).  Section 2 gives the five-step algorithm; Section 2.1
 * local Kriging and Section 2.2 nearest-neighbour Kriging for the off-grid
 * sites; Eq. (condmvn) in Section 3 the conditional law; Section 3.3 the Matern
 * covariance; Section 3.6 the sparse off-grid weights.
 *
 * Conventions used by every entry point:
 *  - Grid node (i, j), 0 <= i, j < m, sits at (x0 + j h, y0 + i h); its flat
 *    index is g = i m + j.  Fields are float32, realization-major R x m x m,
 *    row-major (out[r][i][j]).
 *  - Observation sites are (x, y) pairs of float64 in host memory, n x 2.
 *  - Realization r (global index r_offset + local index) draws its noise from
 *    Philox4x32-10 keyed by the 64-bit seed; results depend only on
 *    (seed, global index), so ranges of realizations can be computed in pieces.
 *    r_offset must be even (realizations come in pairs from one complex FFT).
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is asynchronous on that stream.  Pointers named *_dev are
 *    device pointers owned by the caller; the library never frees them.
 *  - The library owns all other device memory through the context.
 *  - Every function returns a ce_status.  Argument errors are detected on the
 *    host before any work is queued.  ce_last_error() returns a message for the
 *    most recent failure on that context.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef CE_CONDSIM_H
#define CE_CONDSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CE_OK = 0,
  CE_ERR_ARG = 1,      /* invalid argument (sizes, ranges, sites outside the grid) */
  CE_ERR_EMBED = 2,    /* embedding still indefinite after max_growth doublings     */
  CE_ERR_NOT_SPD = 3,  /* a covariance matrix was not positive definite           */
  CE_ERR_CUDA = 4,     /* a CUDA runtime call failed                              */
  CE_ERR_TIMEOUT = 5,  /* a bounded device wait gave up                           */
  CE_ERR_OOM = 6,      /* device allocation failed                                */
  CE_ERR_STATE = 7     /* call out of order (e.g. condsim before krige_weights)   */
} ce_status;

typedef enum { CE_LOCAL = 0, CE_NN = 1 } ce_mode;

/* Arithmetic of the Kriging correction (the grid x site contraction).
 * CE_PREC_FP32: FP32 CUDA-core products and sums (the plain form).
 * CE_PREC_F16X3: tensor cores (tcgen05, kind::f16) on fp16 hi/lo splits of both
 *   operands, three products hi*hi + hi*lo + lo*hi accumulated in FP32: one
 *   low-precision product plus one refinement pass for its residual.
 * CE_PREC_BF16X3: the same with bf16 splits.
 * CE_PREC_TF32X3: the same with tf32 splits (kind::tf32, 32 sites per chunk;
 *   FP32's exponent range, so neither operand needs a scale).
 * In every tensor-core form each accumulator in tensor memory sums at most 512
 * sites before its partial sum joins an FP32 running sum.
 * CE_PREC_FP64: FP64 CUDA-core evaluation, products and sums (site coordinates in
 *   FP64 where local Kriging keeps them); the field stays FP32.  A comparison form
 *   (FP64 runs far below FP32 here), with the FP32 form's compensated solve. */
typedef enum { CE_PREC_FP32 = 0, CE_PREC_F16X3 = 1, CE_PREC_BF16X3 = 2, CE_PREC_TF32X3 = 3, CE_PREC_FP64 = 4 } ce_precision;

typedef struct {
  int m;            /* grid side, 8 <= m <= 4096                                  */
  double x0, y0;    /* coordinates of node (0, 0)                                 */
  double h;         /* node spacing, > 0                                          */
} ce_grid;

typedef struct {
  double sigma;     /* marginal standard deviation; C(0) = sigma^2               */
  double range;     /* Matern range theta > 0                                     */
  double nu;        /* smoothness, 0.5 or 1.5 (Section 3.3 closed forms)          */
  double tau2;      /* nugget variance tau^2 >= 0                                 */
} ce_cov;

typedef struct {
  int mode;         /* ce_mode                                                    */
  int np;           /* local Kriging: neighbourhood order, window (2 np)^2 nodes, 1..4 */
  int k;            /* NN Kriging: nearest grid nodes per site, 1..8              */
  int prec;         /* ce_precision of the correction                             */
} ce_nbhd;

typedef struct {
  int m, P;               /* grid side and embedding side actually used           */
  int n;                  /* number of sites                                     */
  int n_obs;              /* rows of the solve: n (local) or n_N surrogates (NN)  */
  int K;                  /* off-grid weights per site: (2 np)^2 (local) or 1 (NN) */
  int growth;             /* embedding doublings taken                           */
  long long clipped;      /* eigenvalues set to zero                             */
  double lambda_min;      /* smallest eigenvalue before clipping                 */
  double lambda_max;      /* largest eigenvalue                                  */
  double clipped_mass;    /* sum of the clipped (negative) eigenvalues' moduli    */
  double logdet;          /* log det of the prediction matrix A                  */
  size_t device_bytes;    /* device memory held by the context                   */
  int launches;           /* kernels queued by the most recent ce_condsim         */
  int solve_tc;           /* the solve form (ce_solve_form): 1 on the tensor cores  */
} ce_info;

typedef struct ce_ctx ce_ctx;

/* ---------------------------------------------------------------------------
 * ce_setup -- circulant embedding of the grid covariance (Section 1, Wood &
 * Chan; Section 2.1 step (a)).  Builds the first row of the block-circulant
 * matrix on a P x P torus, P the smallest power of two >= 2m, takes its 2-D
 * DFT in FP64 on the device, and doubles P (at most max_growth times, 0..3)
 * while lambda_min < -1e-6 lambda_max; remaining negative eigenvalues are set
 * to 0 and counted.  Stores sqrt(lambda / P^2) in FP32.  Synchronises the
 * stream.  Returns CE_ERR_EMBED when the embedding stays indefinite.
 * *out receives a new context; free it with ce_destroy.
 * ------------------------------------------------------------------------- */
int ce_setup(ce_ctx** out, const ce_grid* grid, const ce_cov* cov, int max_growth, void* stream);

/* ---------------------------------------------------------------------------
 * ce_krige_weights -- off-grid set-up for n sites (obs_xy: host float64 n x 2,
 * 1 <= n <= 65536, every site inside the grid's bounding box, else CE_ERR_ARG).
 * CE_LOCAL (Section 2.1, Section 3.6): per site the (2 np)^2 window of grid
 * nodes around its grid box (shifted inward at the edges), the weights
 * W_1 = K_21 K_11^-1, gamma = sigma^2 - K_21 K_11^-1 K_12 and the nugget
 * phi^2 = tau^2 + gamma, all in FP64 on the device; the prediction matrix is
 * A = K_oo + tau^2 I.
 * CE_NN (Section 2.2, Section 3.2): the union J_N of each site's k nearest grid
 * nodes, the surrogate-data map K_No A^-1, the surrogate variances sigma_N^2 and
 * the prediction matrix K_NN + tau^2 I + diag(sigma_N^2).
 * The prediction matrix is factored by an FP64 Cholesky on the device
 * (CE_ERR_NOT_SPD if that fails) and inverted in FP64; the inverse is kept as
 * an FP32 pair (hi + lo).  Synchronises the stream.  May be called again to
 * replace the sites.
 * ------------------------------------------------------------------------- */
int ce_krige_weights(ce_ctx* ctx, const double* obs_xy, int n, const ce_nbhd* nb);

/* Geometric anisotropy (the paper's Section 5: circulant embedding extends to
 * anisotropic covariances): the covariance of an offset (dx, dy) becomes
 * C(|A (dx, dy)|) with A = diag(1, 1/ratio) Rot(-angle), i.e. the range is the
 * context's range along the direction at `angle` (radians, from the x axis
 * towards y) and range * ratio across it; ratio = 1, angle = 0 is the isotropic
 * model.  Every covariance the library forms follows it: the embedding (whose
 * first row is made even at the torus lag P/2 by the mean with its mirror, so
 * that the eigenvalues stay real; the grid uses no such lag), the Kriging
 * windows and weights, the prediction matrix, the corrections and ce_se_map.
 * Nearest-neighbour selection stays Euclidean in grid units.  Recomputes the
 * embedding on `stream` (it may grow, or fail with CE_ERR_EMBED) and discards
 * the off-grid set-up: call ce_krige_weights again.  If the new embedding fails
 * (CE_ERR_EMBED, CE_ERR_OOM) the previous covariance and its embedding are
 * restored and the error is returned.  ce_condsim_grad returns CE_ERR_STATE
 * while it is anisotropic.  Synchronous; ratio must be positive and finite
 * (CE_ERR_ARG). */
int ce_set_anisotropy(ce_ctx* ctx, double ratio, double angle, void* stream);

/* Change the correction arithmetic (ce_precision) without redoing the set-up. */
int ce_set_precision(ce_ctx* ctx, int prec);

/* Form of the solve B = A^-1 E (Eq. (condmvn)) in ce_condsim, ce_solve and the batch
 * calls (no counterpart in the paper).  CE_SOLVE_FP32 (default): FP32 products with the
 * hi + lo pair of the FP64 inverse, summed with error-free transformations; B is within
 * about 1e-7 of the FP64 solve.  CE_SOLVE_TENSOR: tcgen05 tensor cores, A^-1 and E each
 * split into f16 hi + lo (power-of-two scaled), three products, FP32 accumulation drained
 * every 512 sites, K split over work items whose partial products are joined in a fixed
 * order (deterministic); B is within about 1e-6 of the FP64 solve, at a fraction of the
 * time for thousands of rows.  Because the correction K_go B cancels (its sum of
 * magnitudes is 500 to 2400 times the result on clustered stations), a draw with the
 * tensor-core solve is accurate to about 1e-3, not 1e-5.  The first tensor-core solve of
 * a set-up converts A^-1 (n_obs^2 x 4 bytes more device memory).  CE_ERR_ARG for an
 * unknown form. */
enum ce_solve_form { CE_SOLVE_FP32 = 0, CE_SOLVE_TENSOR = 1 };
int ce_set_solve_form(ce_ctx* ctx, int form);

/* Bound on each wait of the tensor-core correction's epilogue for an accumulator
 * (no counterpart in the paper): the number of mbarrier try_wait rounds (each of
 * which suspends the waiting thread for at most 2 us, less when the accumulator
 * becomes ready) before the wait gives up, records CE_ERR_TIMEOUT, and the launch aborts; the launch then
 * lets its bulk copies and tensor-core work finish, frees its tensor memory and
 * returns, and ce_sync_status reports CE_ERR_TIMEOUT (once: the status word is
 * cleared as it is read).  The output of such a call is invalid.  Default 2^22
 * rounds (at most about 8 s); 0 makes every such wait give up at once, which exercises the
 * abort path without a fault.  Applies to later calls on this context, and to the
 * shared correction launch of a batch (ce_condsim_batch, ce_batch_create) whose
 * first joined event, in the caller's order, it is; that launch reports its status
 * on the same context. */
int ce_set_wait_limit(ce_ctx* ctx, unsigned iterations);

/* How the Kriging correction K_gN B (step 5) is formed in NN mode.
 * CE_NN_DIRECT: the Matern covariance evaluated tile by tile and contracted
 *   (as for local Kriging; follows ce_set_precision).
 * CE_NN_CIRCULANT: the surrogate nodes lie on the grid, so K_gN B is the 2-D
 *   circular convolution of the embedding row c with B scattered onto the
 *   P x P torus, exact for every lag inside the grid (Section 2.1 (a),
 *   Section 2.2): F^-1(lambda . F(b)), two realizations per complex transform,
 *   with the stored (clipped) eigenvalues; FP32 FFTs, independent of
 *   ce_set_precision.
 * Returns CE_ERR_STATE unless the context holds NN Kriging weights. */
enum { CE_NN_DIRECT = 0, CE_NN_CIRCULANT = 1 };
int ce_set_nn_correction(ce_ctx* ctx, int method);

/* Linear mean model (Section 2: z_i = x(s_i)^T beta + y(s_i) + eps_i, beta by
 * generalized least squares).  degree -1: zero mean (the default); 0: a
 * constant, x(s) = [1]; 1: a plane, x(s) = [1, u, v] with u, v the grid-unit
 * coordinates centred on the grid and divided by m.  ce_condsim then draws
 * v_r = y_r + yhat(z - z*_r) with the universal Kriging predictor
 * yhat(w) = X_g beta(w) + K_go A^-1 (w - X beta(w)), beta(w) = (X^T A^-1 X)^-1
 * X^T A^-1 w: per realization beta_r from the residuals (FP64), B_r reduced by
 * A^-1 X beta_r before the correction, X_g beta_r added after it.  Local Kriging
 * only (CE_ERR_STATE otherwise), after ce_krige_weights (a new call of it
 * resets the model); forms A^-1 X and the GLS map once in FP64 on the host and
 * synchronises.  The single-step entry points and ce_condsim_grad do not apply
 * it (the latter returns CE_ERR_STATE while a trend is set). */
int ce_set_trend(ce_ctx* ctx, int degree);

/* Joint draw of sites that share a grid box (the multivariate form of step (b)
 * of local Kriging, Section 2.1; Section 3.6).  on = 1: sites in one grid box
 * (the floor of their grid coordinates) share the box's window S_b and their
 * synthetic observations carry noise L_b eps_b, L_b = chol(Gamma_b + tau^2 I)
 * with Gamma_b = K(s_b, s_b) - K(s_b, S_b) K_11^-1 K(S_b, s_b) their conditional
 * covariance given the window (FP64 set-up, FP32 rows), taken over the box's
 * sites in ascending caller index, eps_b their own nugget draws; a site alone in
 * its box keeps phi_i eps_i, so its draws do not change.  on = 0: every site
 * independently (the default, the algorithm the paper studies).  Prediction
 * still uses A = K_oo + tau^2 I.  *n_boxes (may be NULL) receives the number of
 * boxes with more than one site.  Local Kriging only (CE_ERR_STATE otherwise),
 * after ce_krige_weights (a new call of it resets the choice); CE_ERR_ARG for a
 * box with more than 8 sites, CE_ERR_NOT_SPD for a box whose factor does not
 * exist (coincident sites with tau^2 = 0).  Synchronises.  Applies to
 * ce_condsim, the host entry points and ce_residuals; ce_condsim_grad returns
 * CE_ERR_STATE while it is on. */
int ce_set_box_joint(ce_ctx* ctx, int on, int* n_boxes);

/* Closed-form prediction standard errors at every grid node, without drawing
 * (Section 3.4: SE_E, SE_L, SE_N).  se_exact_dev (M = m*m floats, row-major
 * grid, may be NULL): sqrt of the diagonal of Eq. (condmvn)'s conditional
 * covariance, sigma^2 - k_g^T (K_oo + tau^2 I)^-1 k_g; local mode only
 * (CE_ERR_STATE in NN mode).  se_approx_dev (M floats, may be NULL): the
 * standard deviation of the draws ce_condsim makes on this context, i.e. the
 * diagonal of (I - W_2 S) K_gg (I - W_2 S)^T + W_2 D W_2^T (Section 3.1) with
 * S = W_1 and D the synthetic-noise covariance (diag phi^2, or the grid-box
 * blocks of ce_set_box_joint) in local mode, and the surrogate model's
 * sigma^2 - k_g^T A_N^-1 k_g (Section 3.2) in NN mode.  FP64 covariance
 * evaluation, FP32 products with the stored inverse pair, FP64 sums per node.
 * CE_ERR_STATE while a trend is set.  Cost in local mode: two FP32 products of
 * M x n by n x n, plus n^2 K^2 / 2 FP64 multiply-adds to form Q (K = (2 np)^2
 * window nodes; about 4 ms at n = 2000, K = 36, but minutes at n = 10000,
 * K = 64).  Allocates its work buffers (about 300 MB
 * at most, plus n x n pairs and an m x (2m - 1) table) and synchronises `stream`. */
int ce_se_map(ce_ctx* ctx, float* se_exact_dev, float* se_approx_dev, void* stream);

/* Ensemble moments at every grid node (the ensemble mean estimate and its
 * standard error of the paper's application, Section 4).  ce_ensemble_moments:
 * sum_dev[g] and sumsq_dev[g] (M = m*m doubles each, device) receive the sum and
 * the sum of squares over the R realizations of v_dev (R x m x m floats, device,
 * the layout ce_condsim writes): compensated FP32 sums within the call (within a
 * few FP32 units of the sum of magnitudes), joined to the FP64 buffers; accumulate = 1 adds to what they hold,
 * so calls, batches and ranks combine by addition.  ce_ensemble_stats: mean_dev
 * and sd_dev (M floats each, either may be NULL) receive sum / count and the
 * sample standard deviation sqrt((sumsq - count mean^2) / (count - 1)) (0 for
 * count = 1).  Asynchronous on `stream`. */
int ce_ensemble_moments(ce_ctx* ctx, const float* v_dev, int R, double* sum_dev, double* sumsq_dev, int accumulate,
                        void* stream);
int ce_ensemble_stats(ce_ctx* ctx, const double* sum_dev, const double* sumsq_dev, double count, float* mean_dev,
                      float* sd_dev, void* stream);

/* Measurement support for the rooflines (no counterpart in the paper): the
 * special-function and FP32 FMA throughput of the current GPU, measured by
 * chains of dependent operations on every SM (8 chains per thread, 8 blocks of
 * 256 threads per SM; best of three timed launches).  ex2_per_s: base-2
 * exponentials per second; sqrt_per_s: square roots per second;
 * matern_evals_per_s: evaluations per second of ex2(-sqrt(d2)), the two
 * special-function operations one closed-form Matern covariance takes in the
 * Kriging correction; fma_per_s: FP32 fused multiply-adds per second (two flops
 * each).  Allocates 1.2 MB per call and synchronises `stream`. */
int ce_unit_rates(double* ex2_per_s, double* sqrt_per_s, double* matern_evals_per_s, double* fma_per_s, void* stream);

/* ---------------------------------------------------------------------------
 * ce_condsim -- the whole hot path for R realizations (Section 2, steps 1-5):
 * unconditional CE fields, off-grid values, nugget-perturbed residuals
 * e_r = z - z*_r, B = A^-1 E, and v_r = y_r + K_go B[:, r] on every node.
 * z_dev: device float32 data at the n sites (caller's site order).
 * out_dev: device float32 R x m x m, receives v.  1 <= R <= 4096.
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int ce_condsim(ce_ctx* ctx, const float* z_dev, int R, uint64_t seed, uint64_t r_offset,
               float* out_dev, void* stream);

/* Allocate, ahead of time, every device work buffer that ce_condsim needs for
 * up to R realizations on this context, so that later calls with R or fewer
 * realizations allocate nothing (for example before capturing them into a
 * CUDA graph).  Synchronous. */
int ce_condsim_prepare(ce_ctx* ctx, int R);

/* ce_condsim with host buffers: copies z (n floats) to the device, runs
 * ce_condsim into a context-owned buffer and copies R x m x m floats back
 * to out_host.  Pinned host memory gives full copy bandwidth.  Returns after
 * the copy-back has completed. */
int ce_condsim_host(ce_ctx* ctx, const float* z_host, int R, uint64_t seed, uint64_t r_offset,
                    float* out_host, void* stream);

/* ce_condsim_host_async -- the same draws (Section 2, steps 1-5) with host
 * buffers, pipelined across calls: the data copy and the computation are
 * queued on `stream`, the copy of the fields back to out_host on a stream of
 * the context, and the call returns at once.  Two device staging buffers are
 * used in turn, so the copy-back of one call overlaps the computation of the
 * next.  z_host must stay unchanged, and out_host unread, until ce_host_wait
 * returns; both should be pinned (pageable memory makes the copies
 * synchronous).  Calls on one context must use one stream.  The first call,
 * and a call with a larger R than before, allocate the staging buffers and
 * synchronise.  Argument errors return synchronously; device errors are
 * reported by ce_host_wait. */
int ce_condsim_host_async(ce_ctx* ctx, const float* z_host, int R, uint64_t seed, uint64_t r_offset,
                          float* out_host, void* stream);

/* Waits until every copy-back queued by ce_condsim_host_async on ctx has
 * reached host memory, then returns as ce_sync_status does. */
int ce_host_wait(ce_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Single steps of the path, for testing and timing.  Same conventions.
 * ce_unconditional: step 2 on the grid (Section 2.1 (a)) -- y_dev R x m x m.
 * ce_residuals: steps 3-4 data side -- E_dev R x n_obs float32,
 *   E[r][q] = z_eff[q] - (S y_r)[q] - phi[q] eps*_r[q], with S the local
 *   weights (Section 3.6) or the surrogate selection J_N, in the caller's site
 *   order (NN: increasing surrogate node index).
 * ce_solve: B_dev (R x n_obs) = (A^-1 E^T)^T, same orders.
 * ce_correct: y_dev (R x m x m) += (K_go B)^T in place (step 5).
 * ------------------------------------------------------------------------- */
int ce_unconditional(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y_dev, void* stream);
int ce_residuals(ce_ctx* ctx, const float* y_dev, const float* z_dev, int R, uint64_t seed,
                 uint64_t r_offset, float* E_dev, void* stream);
int ce_solve(ce_ctx* ctx, const float* E_dev, int R, float* B_dev, void* stream);
int ce_correct(ce_ctx* ctx, const float* B_dev, int R, float* y_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Batches of independent events (many grids, site sets and covariance models
 * at once).  Each event is a context set up by ce_setup + ce_krige_weights;
 * the contexts of one batch must be distinct (each owns its work buffers).
 * ce_condsim_batch: queues the draws of every event on `nstreams` (1..16)
 * internal streams forked from and joined back into `stream`, so that events
 * too small to fill the GPU run side by side.  The events whose correction uses
 * the tensor cores (the operand kind of the first such event, an isotropic
 * covariance, the direct correction, R <= 128) run up to the solve on those
 * streams, and after the join their corrections share ONE persistent launch on
 * `stream` (at most 64 events per launch): its blocks take the tiles of all
 * these events from a device work queue (an atomic counter), largest events
 * first, with bounded waits (ce_set_wait_limit); the shared launch's status is
 * reported on the first such event's context.  Other events run whole
 * ce_condsim calls on the internal streams.  Arrays have `count` entries:
 * z_devs[i] (n_i floats), Rs[i], seeds[i], r_offsets[i] (even), outs[i]
 * (R_i x m_i x m_i floats, device).  Asynchronous on `stream`.
 * ce_batch_create: the same schedule captured once into a CUDA graph (the
 * arrays are copied; the pointers must stay valid); ce_batch_launch replays
 * it with one graph launch on `stream` (same seeds: the same draws);
 * ce_batch_destroy frees it.
 * ------------------------------------------------------------------------- */
int ce_condsim_batch(ce_ctx* const* ctxs, const float* const* z_devs, const int* Rs, const uint64_t* seeds,
                     const uint64_t* r_offsets, float* const* outs, int count, int nstreams, void* stream);
typedef struct ce_batch ce_batch;
int ce_batch_create(ce_batch** out, ce_ctx* const* ctxs, const float* const* z_devs, const int* Rs,
                    const uint64_t* seeds, const uint64_t* r_offsets, float* const* outs, int count, int nstreams);
int ce_batch_launch(ce_batch* batch, void* stream);
void ce_batch_destroy(ce_batch* batch);

/* ce_autotune: times, with R realizations on this context (on scratch buffers it
 * allocates and frees), the unconditional ensemble for each L2 budget of one
 * chunk of its FFT intermediate (32, 64, 96 MB: how many realization pairs the
 * column pass hands to the row pass at a time) and, for the tensor-core forms,
 * the correction for each producer-warp configuration (8 or 16 warps), and keeps
 * the fastest of each for later calls.  Synchronises. */
int ce_autotune(ce_ctx* ctx, int R, void* stream);

/* ---------------------------------------------------------------------------
 * ce_unconditional_static -- ce_unconditional that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory at call time (a host application that gives its whole
 * GPU memory budget to its own pool up front, or a latency-critical loop where
 * cudaMalloc/cudaFree would synchronise the device).  The caller passes the
 * context (set up earlier by ce_setup) and the output y_dev (R x m x m); the
 * per-pair FFT intermediate lives in a fixed device array of
 * CE_STATIC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * the library until the process exits.  Grids whose one realization pair needs
 * more (P x m complex floats, 8 P m bytes) are rejected with CE_ERR_ARG and a
 * message.  ce_setup looks up the array's device address (cudaGetSymbolAddress,
 * which also loads the module that holds it) for the device current at set-up,
 * so a call on that device allocates and loads nothing; on a device where no
 * ce_setup ran, the first call does the lookup itself with that device current:
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (nothing in it needs clearing: the row
 * pass writes all that the column pass reads); calls whose work overlaps on the
 * GPU race on it.  Results are bit-identical to those of ce_unconditional.
 * ------------------------------------------------------------------------- */
#define CE_STATIC_SCRATCH_BYTES (16u << 20)
int ce_unconditional_static(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y_dev, void* stream);

/* ---------------------------------------------------------------------------
 * ce_condsim_grad -- ce_condsim (local Kriging) plus the pathwise gradient, at
 * the same noise, of
 *   L = (1/R) sum_r mean_{(i,j) in W} v_r[i][j]^2 + l,
 *   l = -z^T A^-1 z / 2 - log det A / 2 - (n/2) log(2 pi),  A = K_oo + tau^2 I
 * (the Gaussian log-likelihood of the data under the model of Eq. (condmvn)).
 * window: host int[4] = {i0, i1, j0, j1}, the half-open rows and columns of W.
 * out_dev receives v (R x m x m); grad_theta (host double[3]) receives
 * dL/d(sigma, range, tau^2); grad_z_dev (device float, n) receives dL/dz in the
 * caller's site order; *loss receives L.  1 <= R <= 128.  The first call sets
 * up the derivatives of the spectral weights and of the off-grid weights (FP64).
 * Synchronises the stream.
 * ------------------------------------------------------------------------- */
int ce_condsim_grad(ce_ctx* ctx, const float* z_dev, int R, uint64_t seed, uint64_t r_offset, const int* window,
                    float* out_dev, double* grad_theta, float* grad_z_dev, double* loss, void* stream);

/* ---------------------------------------------------------------------------
 * ce_loglik -- the Gaussian log-likelihood of the data under the model of
 * Eq. (condmvn) (z ~ N(0, A), A = K_oo + tau^2 I):
 *   *out = -z^T A^-1 z / 2 - log det A / 2 - (n/2) log(2 pi).
 * z_dev: device float32, n values in the caller's site order.  Uses the FP64
 * log-determinant of the set-up's Cholesky factor and the stored inverse pair
 * (hi + lo), with the quadratic form summed in FP64 on the device.  Local
 * Kriging set-up only and no trend (CE_ERR_STATE otherwise: the NN context
 * factors its surrogate matrix instead of A).  Allocates a buffer of n floats
 * for the call and synchronises `stream`.
 * ------------------------------------------------------------------------- */
int ce_loglik(ce_ctx* ctx, const float* z_dev, double* out, void* stream);

/* Raw Philox4x32-10 words: out_dev[4 i + w] = word w of the generator at counter
 * (ctr_dev[4 i .. 4 i + 3]) and key (seed & 0xffffffff, seed >> 32); count >= 0. */
int ce_philox(const uint32_t* ctr_dev, int count, uint64_t seed, uint32_t* out_dev, void* stream);

/* Box-Muller normals from the same words: out_dev[4 i .. 4 i + 3] = the normals
 * of counter i (pairs (w0, w1) and (w2, w3)). */
int ce_normals(const uint32_t* ctr_dev, int count, uint64_t seed, float* out_dev, void* stream);

/* Context facts (sizes, embedding diagnostics, memory). */
int ce_get_info(const ce_ctx* ctx, ce_info* info);

/* Copy set-up arrays to host memory for inspection, `bytes` = capacity of dst:
 *  CE_ARR_SQRT_LAMBDA  float32 P x P   sqrt(lambda / P^2)
 *  CE_ARR_IDX          int32 n x K     window node indices (local; caller's order)
 *  CE_ARR_W            float32 n x K   W_1 (local; caller's order)
 *  CE_ARR_PHI          float32 n_obs   nugget standard deviations (caller's order)
 *  CE_ARR_J            int32 n_obs     surrogate nodes J_N (NN)                   */
enum { CE_ARR_SQRT_LAMBDA = 0, CE_ARR_IDX = 1, CE_ARR_W = 2, CE_ARR_PHI = 3, CE_ARR_J = 4 };
int ce_copy_array(const ce_ctx* ctx, int which, void* dst, size_t bytes);

/* Per-stage timing of ce_condsim with CUDA events recorded on the call's stream.
 * ce_profile(ctx, 1) starts recording (and clears earlier records), 0 stops.
 * ce_profile_read waits for the recorded calls and writes the summed
 * milliseconds of the CE_NSTAGES stages (unconditional fields, residuals,
 * solve, correction) into ms[], and the number of calls into *calls. */
#define CE_NSTAGES 4
int ce_profile(ce_ctx* ctx, int enable);
int ce_profile_read(ce_ctx* ctx, double* ms, int* calls);

/* Wait for the context's queued work and report errors recorded by kernels. */
int ce_sync_status(ce_ctx* ctx);

/* Message for the last failure on ctx (or the last global failure if ctx is NULL). */
const char* ce_last_error(const ce_ctx* ctx);

/* Free every device buffer of the context.  NULL is ignored. */
void ce_destroy(ce_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CE_CONDSIM_H */
