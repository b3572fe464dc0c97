// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ce_condsim.h"

struct ce_ctx {
  // grid and covariance
  int m = 0;
  double x0 = 0, y0 = 0, h = 0;
  double sigma = 0, range = 0, nu = 0, tau2 = 0;
  // geometric anisotropy (identity map when off)
  double aniso_ratio = 1.0, aniso_angle = 0.0;
  int max_growth = 3;
  // embedding
  int P = 0, growth = 0;
  long long clipped = 0;
  double lambda_min = 0, lambda_max = 0, clipped_mass = 0;
  float* sqrt_lam = nullptr;   // P x P, sqrt(max(lambda, 0) / P^2)
  float* sqrt_lam_t = nullptr; // its transpose, read by the column passes (== sqrt_lam when isotropic)
  float2* twiddle = nullptr;   // P entries e^{-2 pi i k / P}
  float2* tw32 = nullptr;      // P >= 1024: 32 x 32 entries, [k][t] = e^{-2 pi i t k / 1024}
  // off-grid set-up (internal "q" order: Morton order of the observation points)
  int mode = -1, np = 0, knn = 0, prec = CE_PREC_FP32;
  int n = 0;          // sites
  int nobs = 0;       // rows of the solve
  int K = 0;          // weights per row
  int nobs_pad = 0;   // nobs rounded up for the tensor-core tiles
  int* perm = nullptr;      // q -> caller index (local: site; NN: position in J_N)
  int* idx = nullptr;       // nobs x K node indices (internal order)
  float* W = nullptr;       // nobs x K weights
  float* phi = nullptr;     // nobs nugget sd
  int* J = nullptr;         // NN: surrogate nodes, caller (sorted) order
  float* WN = nullptr;      // NN: nobs x n surrogate-data map, internal rows, caller columns
  float4* obs = nullptr;    // nobs points in grid units (int part, frac part) x, y; internal order
  float* Ainv_hi = nullptr; // nobs x nobs, internal order
  float* Ainv_lo = nullptr;
  double logdet = 0;
  // gradient set-up (local mode), computed on first use
  double* sites64 = nullptr;  // nobs x 2 FP64 site coordinates, internal order
  float* dW = nullptr;        // nobs x K: d W_1 / d theta
  float* dphi = nullptr;      // nobs x 3: d phi / d (sigma, theta, tau^2)
  float* ds_theta = nullptr;  // P x P: d sqrt(lambda / N) / d theta
  float* grad_buf = nullptr;  // gradient work buffers
  size_t grad_bytes = 0;
  // sites that share a grid box, drawn jointly (local mode; none while off)
  int box_joint = 0;          // boxes holding more than one site
  int* box_cnt = nullptr;     // nobs: 0 for a site alone in its box, else its position in the box + 1
  int* box_mem = nullptr;     // nobs x kBoxMax: caller indices of the box's sites up to this one
  float* box_L = nullptr;     // nobs x kBoxMax: this site's row of the box's noise factor
  // per-call work buffers (grown on demand)
  int Rcap = 0;
  float* zint = nullptr;    // nobs
  float* E = nullptr;       // Rcap x nobs (internal order)
  float* Bpart = nullptr;   // kSolveKSplit x Rcap x nobs partial (sum, compensation) pairs of the solve
  float* Bm = nullptr;      // Rpad x nobs_pad (internal order), padded for the MMA tiles
  void* Bsplit = nullptr;   // tensor-core operands of B (hi/lo halves)
  size_t bsplit_bytes = 0;
  // the solve on the tensor cores (ce_set_solve_form): A^-1 as f16 hi/lo blocks of 128
  // rows x 64 columns (built on first use), then the bits of max |A^-1|; per-call partial
  // products of the K parts
  int solve_form = CE_SOLVE_FP32;
  uint8_t* ainv_blk = nullptr;
  float* solve_part = nullptr;
  size_t solve_part_bytes = 0;
  int tc_producer_warps = 16;  // producer warps of the tensor-core correction (8 or 16)
  float2* T = nullptr;      // FFT intermediate: pairs_chunk x P x m
  int fft_chunk_mb = 64;    // L2 budget of one chunk of the intermediate (ce_autotune)
  int Tpairs = 0;
  float* host_out = nullptr;    // device buffer used by ce_condsim_host
  size_t host_out_bytes = 0;
  // ce_condsim_host_async: two device staging buffers used in turn, a copy
  // stream for the copies back, and per buffer the events "computed" (on the
  // caller's stream) and "copied" (on the copy stream).
  // linear mean model (ce_set_trend): p regressors, F = A^-1 X (n x p), G (p x n),
  // and per realization the GLS coefficients beta (up to 4096 x 3), FP64
  int trend_p = 0;
  double* trend_F = nullptr;
  double* trend_G = nullptr;
  double* trend_beta = nullptr;
  float* trend_kf = nullptr;     // per realization: the plane k0 + k1 j + k2 i in FP32
  // NN Kriging correction by circulant convolution (ce_set_nn_correction): the
  // P x P complex buffers of one chunk of realization pairs.
  bool nn_circulant = false;
  float2* Xc = nullptr;
  int circ_pairs = 0;
  float* async_out[2] = {nullptr, nullptr};
  size_t async_out_bytes = 0;
  float* async_z[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_computed[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  int async_slot = 0;
  float* zdev_tmp = nullptr;
  int* dev_status = nullptr;    // device-side error word
  unsigned* queue = nullptr;    // work-queue counter of the tensor-core correction (beside the status word)
  unsigned wait_limit = 1u << 22;  // bound on the correction's accumulator waits (ce_set_wait_limit)
  cudaStream_t setup_stream = nullptr;
  size_t device_bytes = 0;
  std::unordered_map<void*, size_t> allocs;
  // optional per-stage timing of ce_condsim: 5 events per call
  int launches = 0;             // kernels queued by the last ce_condsim
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;
  std::string err;
};

// Allocate every per-call work buffer of R realizations ahead of time (ce_api.cu).
extern "C" int ce_condsim_prepare(ce_ctx* ctx, int R);

namespace ce {

// K-range splits of the per-call FP32 solve (more blocks in flight; a second kernel adds the partials).
constexpr int kSolveKSplit = 16;
// Most sites in one grid box that can be drawn jointly.
constexpr int kBoxMax = 8;

// Record a message on ctx (or the global slot) and return the status.
int fail(ce_ctx* ctx, int status, const std::string& msg);
void* dalloc(ce_ctx* ctx, size_t bytes);   // tracked cudaMalloc, nullptr on failure
void dfree(ce_ctx* ctx, void* p);

// ce_api.cu: allocate the per-call work buffers of R realizations ahead of time
int ensure_fft_buffer(ce_ctx* ctx, int R);
int ensure_bsplit(ce_ctx* ctx, int R);

// ce_eigs.cu
int eigs_setup(ce_ctx* ctx, int max_growth, cudaStream_t s);
// Frees the off-grid set-up (weights, inverse, trend, boxes, work buffers); mode becomes -1.
void release_offgrid(ce_ctx* ctx);

int eigs_dsqrt_dtheta(ce_ctx* ctx, float* ds, cudaStream_t s);

// ce_fft.cu
int fft_unconditional(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s);
// The circulant NN correction at P = 1024 in register passes (on ctx->Xc).
int circulant_correct_1024(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);
// The same passes with the intermediate in a caller-supplied buffer; allocates nothing.
int fft_unconditional_into(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s, void* T,
                           size_t T_bytes);
void launch_philox(const uint32_t* ctr, int count, uint64_t seed, uint32_t* out, cudaStream_t s);
void launch_normals(const uint32_t* ctr, int count, uint64_t seed, float* out, cudaStream_t s);

// ce_noalloc.cu: device address of the allocation-free entry point's scratch array,
// looked up (once per device) for the current device.
int static_scratch_resolve();

// ce_linalg.cu
// FP64 Cholesky of A (n x n, device, destroyed) and A^-1: into ctx->Ainv_hi/lo
// (and ctx->logdet) when inv_out is null, else returned in FP64 (caller frees).
int chol_inverse_f64(ce_ctx* ctx, double* A, int n, cudaStream_t s, double** inv_out);
void gemm64_nn_sub(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N, int K,
                   cudaStream_t s);
void launch_solve(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s);
// The context's solve form is the tensor-core one.
bool solve_on_tensor_cores(const ce_ctx* ctx);
// B = A^-1 E on the tensor cores (f16 hi/lo operands, FP32 accumulation drained every 512
// sites, K split into parts joined in a fixed order); *launches counts its kernels.
int launch_solve_tc(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s, int* launches);
// The solve of a conditional-simulation call in the form the context selects; returns
// the status, *launches the kernels it launched.
int solve_condsim(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s, int* launches);
// out (R x n, row stride ldo) = E (R x n) times the symmetric FP32 pair hi + lo (n x n,
// row stride lda, a multiple of 128), through kSolveKSplit partial products in part
// (kSolveKSplit x R x n float pairs).  compensated: TwoSum accumulation (the solve
// that feeds the correction); otherwise per-chunk FP32 sums joined by Kahan compensation.
void launch_gemm_hilo(const float* E, int R, int n, const float* hi, const float* lo, int lda, float* part, float* out,
                      int ldo, cudaStream_t s, bool compensated);
void launch_gemv_f32(const float* Amat, const float* x, float* y, int rows, int cols, cudaStream_t s);

// ce_krige.cu
int check_sites(ce_ctx* ctx, const double* xy, int n);
int krige_local_setup(ce_ctx* ctx, const double* xy_host, int n, int np, cudaStream_t s);
int krige_nn_setup(ce_ctx* ctx, const double* xy_host, int n, int k, cudaStream_t s);
int krige_local_derivatives(ce_ctx* ctx, cudaStream_t s);
void launch_residuals(ce_ctx* ctx, const float* y, const float* zint, int R, uint64_t seed,
                      uint64_t r_offset, float* E, cudaStream_t s);
void launch_permute_rows(const float* src, float* dst, const int* perm, int R, int nobs,
                         int ld_src, int ld_dst, bool to_caller, cudaStream_t s);

// ce_correct.cu, ce_correct_tc.cu
struct MaternF;
int launch_correct(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);
int launch_correct_tc(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);
// Split weights and site records of Rc <= Npad <= 128 realizations of B (rows of stride
// nobs_pad) into the context's operand buffer, for a later batched launch.
int correct_tc_prepare(ce_ctx* ctx, const float* B, int Rc, int Npad, cudaStream_t s);
// One persistent tensor-core launch over the tiles of many prepared events (same operand
// kind, isotropic): y_e += K_go B_e; the queue counter, wait bound and status word of
// `owner` serve it.
int correct_tc_batch(ce_ctx* owner, ce_ctx* const* ctxs, const int* Rs, float* const* ys, int count, int Npad,
                     cudaStream_t s);
// ce_condsim up to and including the solve (steps 2-4 and B = A^-1 E, with the GLS
// reduction of B when a trend is set): the fields in out, B in ctx->Bm.
int condsim_front(ce_ctx* ctx, const float* z, int R, uint64_t seed, uint64_t r_offset, float* out, cudaStream_t s);
int ensure_circulant_buffer(ce_ctx* ctx, int R);
void free_trend(ce_ctx* ctx);
void launch_trend_solve(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s);
void launch_trend_add(ce_ctx* ctx, int R, float* y, cudaStream_t s);
int launch_correct_circulant(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);

}  // namespace ce
