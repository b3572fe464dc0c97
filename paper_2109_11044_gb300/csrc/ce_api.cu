// C ABI of the library: argument checks, context and buffer management, and
// the order of the steps of the conditional simulation (Section 2, steps 1-5).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace {
thread_local std::string tl_err;
}

namespace ce {

int fail(ce_ctx* ctx, int status, const std::string& msg) {
  tl_err = msg;
  if (ctx) ctx->err = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  tl_err = buf;
  return e == cudaErrorMemoryAllocation ? CE_ERR_OOM : CE_ERR_CUDA;
}

void* dalloc(ce_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  ctx->allocs[p] = bytes;
  ctx->device_bytes += bytes;
  return p;
}

void dfree(ce_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->allocs.find(p);
  if (it != ctx->allocs.end()) {
    ctx->device_bytes -= it->second;
    ctx->allocs.erase(it);
  }
  cudaFree(p);
}

}  // namespace ce

using namespace ce;

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int ensure_work(ce_ctx* ctx, int R) {
  if (R <= ctx->Rcap) return CE_OK;
  dfree(ctx, ctx->E);
  dfree(ctx, ctx->Bm);
  dfree(ctx, ctx->Bpart);
  ctx->E = nullptr;
  ctx->Bm = nullptr;
  ctx->Bpart = nullptr;
  ctx->Rcap = 0;
  const int Rpad = (R + 15) / 16 * 16;
  ctx->E = (float*)dalloc(ctx, sizeof(float) * (size_t)R * ctx->nobs);
  ctx->Bm = (float*)dalloc(ctx, sizeof(float) * (size_t)Rpad * ctx->nobs_pad);
  ctx->Bpart = (float*)dalloc(ctx, sizeof(float2) * kSolveKSplit * (size_t)R * ctx->nobs);   // (sum, compensation) pairs
  if (!ctx->E || !ctx->Bm || !ctx->Bpart) return fail(ctx, CE_ERR_OOM, "per-call buffers");
  CE_CUDA_TRY(cudaMemset(ctx->Bm, 0, sizeof(float) * (size_t)Rpad * ctx->nobs_pad));
  ctx->Rcap = R;
  return CE_OK;
}

int check_call(ce_ctx* ctx, int R, uint64_t r_offset) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (ctx->mode < 0) return fail(ctx, CE_ERR_STATE, "ce_krige_weights has not been called");
  if (!ctx->sqrt_lam) return fail(ctx, CE_ERR_STATE, "the context has no embedding");
  if (R < 1 || R > 4096) return fail(ctx, CE_ERR_ARG, "R must be in [1, 4096]");
  if (r_offset % 2) return fail(ctx, CE_ERR_ARG, "r_offset must be even");
  if (r_offset + (uint64_t)R > 0xffffffffull) return fail(ctx, CE_ERR_ARG, "realization index exceeds 32 bits");
  return CE_OK;
}

// zint[q] = z[perm[q]] (local) or (K_No A^-1 z)[q] (NN)
void data_to_internal(ce_ctx* ctx, const float* z, cudaStream_t s) {
  ctx->launches += 1;
  if (ctx->mode == CE_NN) launch_gemv_f32(ctx->WN, z, ctx->zint, ctx->nobs, ctx->n, s);
  else launch_permute_rows(z, ctx->zint, ctx->perm, 1, ctx->nobs, ctx->n, ctx->nobs, false, s);
}

}  // namespace

namespace ce {

int condsim_front(ce_ctx* ctx, const float* z, int R, uint64_t seed, uint64_t r_offset, float* out, cudaStream_t s) {
  int st = check_call(ctx, R, r_offset);
  if (st) return st;
  if (!z || !out) return fail(ctx, CE_ERR_ARG, "null pointer");
  if ((st = ensure_work(ctx, R))) return st;
  if ((st = fft_unconditional(ctx, R, seed, r_offset, out, s))) return st;   // step 2 on the grid
  data_to_internal(ctx, z, s);
  launch_residuals(ctx, out, ctx->zint, R, seed, r_offset, ctx->E, s);         // steps 3-4, data side
  int nl = 0;
  if ((st = solve_condsim(ctx, ctx->E, R, ctx->Bm, ctx->nobs_pad, s, &nl))) return st;   // B = A^-1 E
  launch_trend_solve(ctx, ctx->E, R, ctx->Bm, ctx->nobs_pad, s);              // linear mean: B -= F G E
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace ce

extern "C" {

int ce_setup(ce_ctx** out, const ce_grid* grid, const ce_cov* cov, int max_growth, void* stream) {
  tl_err.clear();
  if (!out || !grid || !cov) return fail(nullptr, CE_ERR_ARG, "null argument");
  *out = nullptr;
  if (grid->m < 8 || grid->m > 4096) return fail(nullptr, CE_ERR_ARG, "grid side m must be in [8, 4096]");
  if (!(grid->h > 0) || !std::isfinite(grid->h) || !std::isfinite(grid->x0) || !std::isfinite(grid->y0))
    return fail(nullptr, CE_ERR_ARG, "grid spacing must be positive and finite");
  if (!(cov->sigma > 0) || !(cov->range > 0) || !(cov->tau2 >= 0) || !std::isfinite(cov->sigma) ||
      !std::isfinite(cov->range) || !std::isfinite(cov->tau2))
    return fail(nullptr, CE_ERR_ARG, "covariance needs sigma > 0, range > 0, tau2 >= 0");
  if (cov->nu != 0.5 && cov->nu != 1.5) return fail(nullptr, CE_ERR_ARG, "nu must be 0.5 or 1.5");
  if (max_growth < 0 || max_growth > 3) return fail(nullptr, CE_ERR_ARG, "max_growth must be in [0, 3]");
  ce_ctx* ctx = new ce_ctx();
  ctx->m = grid->m;
  ctx->x0 = grid->x0;
  ctx->y0 = grid->y0;
  ctx->h = grid->h;
  ctx->sigma = cov->sigma;
  ctx->range = cov->range;
  ctx->nu = cov->nu;
  ctx->tau2 = cov->tau2;
  ctx->setup_stream = as_stream(stream);
  ctx->dev_status = (int*)dalloc(ctx, 4 * sizeof(int));   // the status word, then the work-queue counter
  if (!ctx->dev_status) { delete ctx; return fail(nullptr, CE_ERR_OOM, "status word"); }
  ctx->queue = reinterpret_cast<unsigned*>(ctx->dev_status + 1);
  if (cudaMemset(ctx->dev_status, 0, 4 * sizeof(int)) != cudaSuccess) {
    ce_destroy(ctx);
    return fail(nullptr, CE_ERR_CUDA, "status word");
  }
  ctx->max_growth = max_growth;
  int st = eigs_setup(ctx, max_growth, as_stream(stream));
  // the allocation-free entry point's scratch array: placed on this device now, not in its first call
  if (st == CE_OK) st = static_scratch_resolve();
  if (st != CE_OK) {
    const std::string msg = ctx->err.empty() ? tl_err : ctx->err;
    ce_destroy(ctx);
    return fail(nullptr, st, msg);
  }
  *out = ctx;
  return CE_OK;
}

int ce_krige_weights(ce_ctx* ctx, const double* obs_xy, int n, const ce_nbhd* nb) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!obs_xy || !nb) return fail(ctx, CE_ERR_ARG, "null argument");
  if (n < 1 || n > 65536) return fail(ctx, CE_ERR_ARG, "n must be in [1, 65536]");
  if (nb->prec < 0 || nb->prec > 4) return fail(ctx, CE_ERR_ARG, "unknown precision");
  for (int i = 0; i < 2 * n; ++i)
    if (!std::isfinite(obs_xy[i])) return fail(ctx, CE_ERR_ARG, "site coordinates must be finite");
  int st;
  ctx->mode = -1;
  if (nb->mode == CE_LOCAL) {
    if (nb->np < 1 || nb->np > 4) return fail(ctx, CE_ERR_ARG, "np must be in [1, 4]");
    st = krige_local_setup(ctx, obs_xy, n, nb->np, ctx->setup_stream);
  } else if (nb->mode == CE_NN) {
    if (nb->k < 1 || nb->k > 8) return fail(ctx, CE_ERR_ARG, "k must be in [1, 8]");
    st = krige_nn_setup(ctx, obs_xy, n, nb->k, ctx->setup_stream);
  } else {
    return fail(ctx, CE_ERR_ARG, "unknown mode");
  }
  if (st != CE_OK) { ctx->mode = -1; return st; }
  ctx->prec = nb->prec;
  CE_CUDA_TRY(cudaStreamSynchronize(ctx->setup_stream));
  return CE_OK;
}

int ce_set_precision(ce_ctx* ctx, int prec) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  if (prec < 0 || prec > 4) return fail(ctx, CE_ERR_ARG, "unknown precision");
  ctx->prec = prec;
  return CE_OK;
}

int ce_set_solve_form(ce_ctx* ctx, int form) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  if (form != CE_SOLVE_FP32 && form != CE_SOLVE_TENSOR) return fail(ctx, CE_ERR_ARG, "unknown solve form");
  ctx->solve_form = form;
  return CE_OK;
}

int ce_set_wait_limit(ce_ctx* ctx, unsigned iterations) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->wait_limit = iterations;
  return CE_OK;
}

int ce_unconditional(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y_dev, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!ctx->sqrt_lam) return fail(ctx, CE_ERR_STATE, "the context has no embedding");
  if (R < 1 || R > 4096) return fail(ctx, CE_ERR_ARG, "R must be in [1, 4096]");
  if (r_offset % 2) return fail(ctx, CE_ERR_ARG, "r_offset must be even");
  if (!y_dev) return fail(ctx, CE_ERR_ARG, "null output");
  return fft_unconditional(ctx, R, seed, r_offset, y_dev, as_stream(stream));
}

int ce_residuals(ce_ctx* ctx, const float* y_dev, const float* z_dev, int R, uint64_t seed, uint64_t r_offset, float* E_dev,
                 void* stream) {
  int st = check_call(ctx, R, r_offset);
  if (st) return st;
  if (!y_dev || !z_dev || !E_dev) return fail(ctx, CE_ERR_ARG, "null pointer");
  if ((st = ensure_work(ctx, R))) return st;
  cudaStream_t s = as_stream(stream);
  data_to_internal(ctx, z_dev, s);
  launch_residuals(ctx, y_dev, ctx->zint, R, seed, r_offset, ctx->E, s);
  launch_permute_rows(ctx->E, E_dev, ctx->perm, R, ctx->nobs, ctx->nobs, ctx->nobs, true, s);
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int ce_solve(ce_ctx* ctx, const float* E_dev, int R, float* B_dev, void* stream) {
  int st = check_call(ctx, R, 0);
  if (st) return st;
  if (!E_dev || !B_dev) return fail(ctx, CE_ERR_ARG, "null pointer");
  if ((st = ensure_work(ctx, R))) return st;
  cudaStream_t s = as_stream(stream);
  launch_permute_rows(E_dev, ctx->E, ctx->perm, R, ctx->nobs, ctx->nobs, ctx->nobs, false, s);
  int nl = 0;
  if ((st = solve_condsim(ctx, ctx->E, R, ctx->Bm, ctx->nobs_pad, s, &nl))) return st;
  launch_permute_rows(ctx->Bm, B_dev, ctx->perm, R, ctx->nobs, ctx->nobs_pad, ctx->nobs, true, s);
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int ce_correct(ce_ctx* ctx, const float* B_dev, int R, float* y_dev, void* stream) {
  int st = check_call(ctx, R, 0);
  if (st) return st;
  if (!B_dev || !y_dev) return fail(ctx, CE_ERR_ARG, "null pointer");
  if ((st = ensure_work(ctx, R))) return st;
  cudaStream_t s = as_stream(stream);
  launch_permute_rows(B_dev, ctx->Bm, ctx->perm, R, ctx->nobs, ctx->nobs, ctx->nobs_pad, false, s);
  return launch_correct(ctx, ctx->Bm, R, y_dev, s);
}

int ce_condsim_prepare(ce_ctx* ctx, int R) {
  int st = check_call(ctx, R, 0);
  if (st) return st;
  if ((st = ensure_work(ctx, R))) return st;
  if ((st = ensure_fft_buffer(ctx, R))) return st;
  if (ctx->mode == CE_NN && ctx->nn_circulant && (st = ensure_circulant_buffer(ctx, R))) return st;
  return ensure_bsplit(ctx, R);
}

int ce_set_nn_correction(ce_ctx* ctx, int method) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  if (method != CE_NN_DIRECT && method != CE_NN_CIRCULANT) return fail(ctx, CE_ERR_ARG, "unknown NN correction method");
  if (ctx->mode != CE_NN) return fail(ctx, CE_ERR_STATE, "the circulant correction needs NN Kriging (ce_krige_weights with CE_NN)");
  ctx->nn_circulant = method == CE_NN_CIRCULANT;
  return CE_OK;
}

int ce_condsim(ce_ctx* ctx, const float* z_dev, int R, uint64_t seed, uint64_t r_offset, float* out_dev, void* stream) {
  int st = check_call(ctx, R, r_offset);
  if (st) return st;
  if (!z_dev || !out_dev) return fail(ctx, CE_ERR_ARG, "null pointer");
  if ((st = ensure_work(ctx, R))) return st;
  cudaStream_t s = as_stream(stream);
  cudaEvent_t ev[CE_NSTAGES + 1] = {};
  if (ctx->profiling) {
    for (auto& e : ev) {
      CE_CUDA_TRY(cudaEventCreate(&e));
      ctx->prof_events.push_back(e);
    }
  }
  auto mark = [&](int i) { if (ctx->profiling) cudaEventRecord(ev[i], s); };
  ctx->launches = 0;
  mark(0);
  if ((st = fft_unconditional(ctx, R, seed, r_offset, out_dev, s))) return st;   // step 2 on the grid
  mark(1);
  data_to_internal(ctx, z_dev, s);
  launch_residuals(ctx, out_dev, ctx->zint, R, seed, r_offset, ctx->E, s);         // steps 3-4, data side
  mark(2);
  int nl = 0;
  if ((st = solve_condsim(ctx, ctx->E, R, ctx->Bm, ctx->nobs_pad, s, &nl))) return st;   // B = A^-1 E
  ctx->launches += 1 + nl;
  launch_trend_solve(ctx, ctx->E, R, ctx->Bm, ctx->nobs_pad, s);                  // linear mean: B -= F G E
  mark(3);
  st = launch_correct(ctx, ctx->Bm, R, out_dev, s);                               // step 5
  if (st == CE_OK) launch_trend_add(ctx, R, out_dev, s);                          // + X_g G E
  mark(4);
  return st;
}

int ce_profile(ce_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  CE_CUDA_TRY(cudaDeviceSynchronize());
  for (auto e : ctx->prof_events) cudaEventDestroy(e);
  ctx->prof_events.clear();
  ctx->profiling = enable != 0;
  return CE_OK;
}

int ce_profile_read(ce_ctx* ctx, double* ms, int* calls) {
  if (!ctx || !ms || !calls) return fail(nullptr, CE_ERR_ARG, "null argument");
  for (int i = 0; i < CE_NSTAGES; ++i) ms[i] = 0.0;
  const int per = CE_NSTAGES + 1;
  *calls = (int)(ctx->prof_events.size() / per);
  for (int c = 0; c < *calls; ++c) {
    CE_CUDA_TRY(cudaEventSynchronize(ctx->prof_events[(size_t)c * per + CE_NSTAGES]));
    for (int i = 0; i < CE_NSTAGES; ++i) {
      float t = 0.f;
      CE_CUDA_TRY(cudaEventElapsedTime(&t, ctx->prof_events[(size_t)c * per + i], ctx->prof_events[(size_t)c * per + i + 1]));
      ms[i] += t;
    }
  }
  return CE_OK;
}

int ce_condsim_host(ce_ctx* ctx, const float* z_host, int R, uint64_t seed, uint64_t r_offset, float* out_host, void* stream) {
  int st = check_call(ctx, R, r_offset);
  if (st) return st;
  if (!z_host || !out_host) return fail(ctx, CE_ERR_ARG, "null pointer");
  const size_t bytes = sizeof(float) * (size_t)R * ctx->m * ctx->m;
  if (ctx->host_out_bytes < bytes) {
    dfree(ctx, ctx->host_out);
    ctx->host_out = (float*)dalloc(ctx, bytes);
    ctx->host_out_bytes = ctx->host_out ? bytes : 0;
    if (!ctx->host_out) return fail(ctx, CE_ERR_OOM, "output staging buffer");
  }
  if (!ctx->zdev_tmp) {
    ctx->zdev_tmp = (float*)dalloc(ctx, sizeof(float) * ctx->n);
    if (!ctx->zdev_tmp) return fail(ctx, CE_ERR_OOM, "data staging buffer");
  }
  cudaStream_t s = as_stream(stream);
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->zdev_tmp, z_host, sizeof(float) * ctx->n, cudaMemcpyHostToDevice, s));
  if ((st = ce_condsim(ctx, ctx->zdev_tmp, R, seed, r_offset, ctx->host_out, stream))) return st;
  CE_CUDA_TRY(cudaMemcpyAsync(out_host, ctx->host_out, bytes, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  return CE_OK;
}

int ce_condsim_host_async(ce_ctx* ctx, const float* z_host, int R, uint64_t seed, uint64_t r_offset, float* out_host,
                          void* stream) {
  int st = check_call(ctx, R, r_offset);
  if (st) return st;
  if (!z_host || !out_host) return fail(ctx, CE_ERR_ARG, "null pointer");
  const size_t bytes = sizeof(float) * (size_t)R * ctx->m * ctx->m;
  if (!ctx->copy_stream) {
    CE_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      CE_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_computed[b], cudaEventDisableTiming));
      CE_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming));
    }
  }
  if (ctx->async_out_bytes < bytes) {
    CE_CUDA_TRY(cudaStreamSynchronize(ctx->copy_stream));   // earlier copies still read the old buffers
    CE_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    for (int b = 0; b < 2; ++b) {
      dfree(ctx, ctx->async_out[b]);
      ctx->async_out[b] = (float*)dalloc(ctx, bytes);
      if (!ctx->async_out[b]) {
        ctx->async_out_bytes = 0;
        return fail(ctx, CE_ERR_OOM, "output staging buffers");
      }
    }
    ctx->async_out_bytes = bytes;
  }
  for (int b = 0; b < 2; ++b) {
    if (!ctx->async_z[b]) {
      ctx->async_z[b] = (float*)dalloc(ctx, sizeof(float) * ctx->n);
      if (!ctx->async_z[b]) return fail(ctx, CE_ERR_OOM, "data staging buffers");
    }
  }
  cudaStream_t s = as_stream(stream);
  const int b = ctx->async_slot;
  ctx->async_slot ^= 1;
  // buffer b is free once the copy issued from it two calls ago has finished
  CE_CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_copied[b], 0));
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->async_z[b], z_host, sizeof(float) * ctx->n, cudaMemcpyHostToDevice, s));
  if ((st = ce_condsim(ctx, ctx->async_z[b], R, seed, r_offset, ctx->async_out[b], stream))) return st;
  CE_CUDA_TRY(cudaEventRecord(ctx->ev_computed[b], s));
  CE_CUDA_TRY(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_computed[b], 0));
  CE_CUDA_TRY(cudaMemcpyAsync(out_host, ctx->async_out[b], bytes, cudaMemcpyDeviceToHost, ctx->copy_stream));
  CE_CUDA_TRY(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
  return CE_OK;
}

int ce_host_wait(ce_ctx* ctx) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  if (ctx->copy_stream) CE_CUDA_TRY(cudaStreamSynchronize(ctx->copy_stream));
  return ce_sync_status(ctx);
}

int ce_philox(const uint32_t* ctr_dev, int count, uint64_t seed, uint32_t* out_dev, void* stream) {
  tl_err.clear();
  if (count < 0 || (count > 0 && (!ctr_dev || !out_dev))) return fail(nullptr, CE_ERR_ARG, "bad philox arguments");
  launch_philox(ctr_dev, count, seed, out_dev, as_stream(stream));
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int ce_normals(const uint32_t* ctr_dev, int count, uint64_t seed, float* out_dev, void* stream) {
  tl_err.clear();
  if (count < 0 || (count > 0 && (!ctr_dev || !out_dev))) return fail(nullptr, CE_ERR_ARG, "bad normals arguments");
  launch_normals(ctr_dev, count, seed, out_dev, as_stream(stream));
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int ce_set_anisotropy(ce_ctx* ctx, double ratio, double angle, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!(ratio > 0.0) || !std::isfinite(ratio) || !std::isfinite(angle)) {
    return fail(ctx, CE_ERR_ARG, "anisotropy ratio must be positive and finite, the angle finite");
  }
  CE_CUDA_TRY(cudaDeviceSynchronize());
  // every buffer whose size or contents depend on the embedding goes
  release_offgrid(ctx);
  if (ctx->sqrt_lam_t != ctx->sqrt_lam) dfree(ctx, ctx->sqrt_lam_t);
  ctx->sqrt_lam_t = nullptr;
  dfree(ctx, ctx->sqrt_lam); ctx->sqrt_lam = nullptr;
  dfree(ctx, ctx->twiddle); ctx->twiddle = nullptr;
  dfree(ctx, ctx->tw32); ctx->tw32 = nullptr;
  dfree(ctx, ctx->T); ctx->T = nullptr; ctx->Tpairs = 0;
  dfree(ctx, ctx->Xc); ctx->Xc = nullptr; ctx->circ_pairs = 0;
  const double old_ratio = ctx->aniso_ratio, old_angle = ctx->aniso_angle;
  ctx->aniso_ratio = ratio;
  ctx->aniso_angle = angle;
  const int st = eigs_setup(ctx, ctx->max_growth, as_stream(stream));
  if (st == CE_OK) return CE_OK;
  // keep the context usable: back to the previous covariance and its embedding
  const std::string msg = ctx->err;
  ctx->aniso_ratio = old_ratio;
  ctx->aniso_angle = old_angle;
  (void)cudaGetLastError();
  const int st2 = eigs_setup(ctx, ctx->max_growth, as_stream(stream));
  return fail(ctx, st, msg + (st2 == CE_OK ? " (the previous covariance is kept)" : " (no embedding left)"));
}

int ce_get_info(const ce_ctx* ctx, ce_info* info) {
  if (!ctx || !info) return fail(nullptr, CE_ERR_ARG, "null argument");
  info->m = ctx->m;
  info->P = ctx->P;
  info->n = ctx->n;
  info->n_obs = ctx->nobs;
  info->K = ctx->K;
  info->growth = ctx->growth;
  info->clipped = ctx->clipped;
  info->lambda_min = ctx->lambda_min;
  info->lambda_max = ctx->lambda_max;
  info->clipped_mass = ctx->clipped_mass;
  info->logdet = ctx->logdet;
  info->device_bytes = ctx->device_bytes;
  info->launches = ctx->launches;
  info->solve_tc = solve_on_tensor_cores(ctx) ? 1 : 0;
  return CE_OK;
}

int ce_copy_array(const ce_ctx* cctx, int which, void* dst, size_t bytes) {
  ce_ctx* ctx = const_cast<ce_ctx*>(cctx);
  if (!ctx || !dst) return fail(nullptr, CE_ERR_ARG, "null argument");
  CE_CUDA_TRY(cudaDeviceSynchronize());
  if (which == CE_ARR_SQRT_LAMBDA) {
    if (!ctx->sqrt_lam) return fail(ctx, CE_ERR_STATE, "the context has no embedding");
    const size_t need = sizeof(float) * (size_t)ctx->P * ctx->P;
    if (bytes < need) return fail(ctx, CE_ERR_ARG, "destination too small");
    CE_CUDA_TRY(cudaMemcpy(dst, ctx->sqrt_lam, need, cudaMemcpyDeviceToHost));
    return CE_OK;
  }
  if (ctx->mode < 0) return fail(ctx, CE_ERR_STATE, "no off-grid set-up");
  std::vector<int> perm(ctx->nobs);
  CE_CUDA_TRY(cudaMemcpy(perm.data(), ctx->perm, sizeof(int) * ctx->nobs, cudaMemcpyDeviceToHost));
  const int K = ctx->K, nob = ctx->nobs;
  if (which == CE_ARR_IDX || which == CE_ARR_W) {
    if (ctx->mode != CE_LOCAL) return fail(ctx, CE_ERR_STATE, "weights exist in local mode only");
    const size_t need = sizeof(float) * (size_t)nob * K;
    if (bytes < need) return fail(ctx, CE_ERR_ARG, "destination too small");
    std::vector<float> tmp((size_t)nob * K);
    CE_CUDA_TRY(cudaMemcpy(tmp.data(), which == CE_ARR_IDX ? (void*)ctx->idx : (void*)ctx->W, need, cudaMemcpyDeviceToHost));
    float* d = (float*)dst;
    for (int q = 0; q < nob; ++q) std::memcpy(d + (size_t)perm[q] * K, tmp.data() + (size_t)q * K, sizeof(float) * K);
    return CE_OK;
  }
  if (which == CE_ARR_PHI) {
    if (bytes < sizeof(float) * nob) return fail(ctx, CE_ERR_ARG, "destination too small");
    std::vector<float> tmp(nob);
    CE_CUDA_TRY(cudaMemcpy(tmp.data(), ctx->phi, sizeof(float) * nob, cudaMemcpyDeviceToHost));
    for (int q = 0; q < nob; ++q) ((float*)dst)[perm[q]] = tmp[q];
    return CE_OK;
  }
  if (which == CE_ARR_J) {
    if (ctx->mode != CE_NN) return fail(ctx, CE_ERR_STATE, "surrogate nodes exist in NN mode only");
    if (bytes < sizeof(int) * nob) return fail(ctx, CE_ERR_ARG, "destination too small");
    CE_CUDA_TRY(cudaMemcpy(dst, ctx->J, sizeof(int) * nob, cudaMemcpyDeviceToHost));
    return CE_OK;
  }
  return fail(ctx, CE_ERR_ARG, "unknown array");
}

int ce_sync_status(ce_ctx* ctx) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  CE_CUDA_TRY(cudaDeviceSynchronize());
  int st = 0;
  CE_CUDA_TRY(cudaMemcpy(&st, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    // reported once: the next calls start from a clear status word
    CE_CUDA_TRY(cudaMemset(ctx->dev_status, 0, sizeof(int)));
    return fail(ctx, st, "a kernel reported status " + std::to_string(st) +
                             (st == CE_ERR_TIMEOUT ? " (a bounded device wait gave up; the call's output is invalid)" : ""));
  }
  return CE_OK;
}

const char* ce_last_error(const ce_ctx* ctx) {
  if (ctx && !ctx->err.empty()) return ctx->err.c_str();
  return tl_err.c_str();
}

void ce_destroy(ce_ctx* ctx) {
  if (!ctx) return;
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
    for (int b = 0; b < 2; ++b) {
      cudaEventDestroy(ctx->ev_computed[b]);
      cudaEventDestroy(ctx->ev_copied[b]);
    }
  }
  for (auto e : ctx->prof_events) cudaEventDestroy(e);
  for (auto& kv : ctx->allocs) cudaFree(kv.first);
  ctx->allocs.clear();
  delete ctx;
}

}  // extern "C"
