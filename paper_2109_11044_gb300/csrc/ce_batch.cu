// Batches of independent events: a fork/join schedule of the per-event steps
// over internal streams with one persistent tensor-core correction launch for all
// events that can share it, optionally captured once into a CUDA graph and
// replayed with a single graph launch; and a small autotuner for the tensor-core
// correction's producer configuration.
#include <algorithm>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace {

constexpr int kMaxStreams = 16;

struct StreamSet {
  cudaStream_t s[kMaxStreams] = {};
  cudaEvent_t done[kMaxStreams] = {};
  cudaEvent_t fork = nullptr;
  int n = 0;
  int create(int want) {
    n = want;
    for (int i = 0; i < n; ++i) {
      CE_CUDA_TRY(cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking));
      CE_CUDA_TRY(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
    }
    CE_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    return CE_OK;
  }
  void destroy() {
    for (int i = 0; i < n; ++i) {
      if (s[i]) cudaStreamDestroy(s[i]);
      if (done[i]) cudaEventDestroy(done[i]);
    }
    if (fork) cudaEventDestroy(fork);
    n = 0;
  }
};

int check_batch(ce_ctx* const* ctxs, const float* const* z, const int* Rs, const uint64_t* seeds, const uint64_t* offs,
                float* const* outs, int count, int nstreams) {
  if (count < 1 || !ctxs || !z || !Rs || !seeds || !offs || !outs)
    return ce::fail(nullptr, CE_ERR_ARG, "batch: null array or count < 1");
  if (nstreams < 1 || nstreams > kMaxStreams) return ce::fail(nullptr, CE_ERR_ARG, "batch: nstreams must be in [1, 16]");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return ce::fail(nullptr, CE_ERR_ARG, "batch: null context");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return ce::fail(nullptr, CE_ERR_ARG, "batch: a context appears twice");
  }
  return CE_OK;
}

// Fork from `stream`, run event i on internal stream i % n, join back.  The events
// whose correction can share one launch (a tensor-core form, the same operand kind as
// the first such event, an isotropic covariance, no circulant NN correction, at most
// 128 realizations) run their steps up to the solve and their weight preparation on
// the internal streams; after the join one persistent tensor-core launch on `stream`
// takes the tiles of all of them from its work queue, largest events first.  The
// other events run whole ce_condsim calls on the internal streams.
int enqueue(StreamSet& ss, ce_ctx* const* ctxs, const float* const* z, const int* Rs, const uint64_t* seeds,
            const uint64_t* offs, float* const* outs, int count, cudaStream_t stream) {
  std::vector<int> joined;
  int prec = -1, Npad = 16;
  for (int e = 0; e < count; ++e) {
    const ce_ctx* c = ctxs[e];
    const bool tc = c->prec == CE_PREC_F16X3 || c->prec == CE_PREC_BF16X3 || c->prec == CE_PREC_TF32X3;
    const bool iso = c->aniso_ratio == 1.0 && c->aniso_angle == 0.0;
    if (tc && iso && !(c->mode == CE_NN && c->nn_circulant) && Rs[e] >= 1 && Rs[e] <= 128 && (prec < 0 || c->prec == prec)) {
      joined.push_back(e);
      prec = c->prec;
      Npad = std::max(Npad, (Rs[e] + 15) / 16 * 16);
    }
  }
  if (joined.size() < 2) joined.clear();   // a lone event keeps its own launch
  std::vector<char> in_batch(count, 0);
  for (int e : joined) in_batch[e] = 1;
  CE_CUDA_TRY(cudaEventRecord(ss.fork, stream));
  for (int i = 0; i < ss.n; ++i) CE_CUDA_TRY(cudaStreamWaitEvent(ss.s[i], ss.fork, 0));
  for (int e = 0; e < count; ++e) {
    cudaStream_t se = ss.s[e % ss.n];
    int st;
    if (in_batch[e]) {
      st = ce::condsim_front(ctxs[e], z[e], Rs[e], seeds[e], offs[e], outs[e], se);
      if (st == CE_OK) st = ce::correct_tc_prepare(ctxs[e], ctxs[e]->Bm, Rs[e], Npad, se);
    } else {
      st = ce_condsim(ctxs[e], z[e], Rs[e], seeds[e], offs[e], outs[e], se);
    }
    if (st != CE_OK) return st;
  }
  for (int i = 0; i < ss.n; ++i) {
    CE_CUDA_TRY(cudaEventRecord(ss.done[i], ss.s[i]));
    CE_CUDA_TRY(cudaStreamWaitEvent(stream, ss.done[i], 0));
  }
  if (!joined.empty()) {
    ce_ctx* owner = ctxs[joined.front()];   // the first joined event in the caller's order
    auto cost = [&](int e) { return (double)ctxs[e]->m * ((ctxs[e]->m + 127) / 128) * ctxs[e]->nobs_pad; };
    std::stable_sort(joined.begin(), joined.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<ce_ctx*> bc;
    std::vector<int> br;
    std::vector<float*> by;
    for (int e : joined) {
      bc.push_back(ctxs[e]);
      br.push_back(Rs[e]);
      by.push_back(outs[e]);
    }
    const int st = ce::correct_tc_batch(owner, bc.data(), br.data(), by.data(), (int)bc.size(), Npad, stream);
    if (st != CE_OK) return st;
    for (int e : joined) ce::launch_trend_add(ctxs[e], Rs[e], outs[e], stream);   // + X_g G E (no-op without a trend)
    CE_CUDA_TRY(cudaGetLastError());
  }
  return CE_OK;
}

thread_local StreamSet tl_streams;

}  // namespace

struct ce_batch {
  std::vector<ce_ctx*> ctxs;
  std::vector<const float*> z;
  std::vector<int> R;
  std::vector<uint64_t> seeds, offs;
  std::vector<float*> outs;
  StreamSet ss;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int ce_condsim_batch(ce_ctx* const* ctxs, const float* const* z_devs, const int* Rs, const uint64_t* seeds,
                     const uint64_t* r_offsets, float* const* outs, int count, int nstreams, void* stream) {
  int st = check_batch(ctxs, z_devs, Rs, seeds, r_offsets, outs, count, nstreams);
  if (st) return st;
  // work buffers first: an allocation inside the fork would serialise the streams
  for (int e = 0; e < count; ++e)
    if ((st = ce_condsim_prepare(ctxs[e], Rs[e]))) return st;
  if (tl_streams.n != nstreams) {
    tl_streams.destroy();
    if ((st = tl_streams.create(nstreams))) return st;
  }
  return enqueue(tl_streams, ctxs, z_devs, Rs, seeds, r_offsets, outs, count, reinterpret_cast<cudaStream_t>(stream));
}

int ce_batch_create(ce_batch** out, ce_ctx* const* ctxs, const float* const* z_devs, const int* Rs, const uint64_t* seeds,
                    const uint64_t* r_offsets, float* const* outs, int count, int nstreams) {
  if (!out) return ce::fail(nullptr, CE_ERR_ARG, "null output");
  *out = nullptr;
  int st = check_batch(ctxs, z_devs, Rs, seeds, r_offsets, outs, count, nstreams);
  if (st) return st;
  for (int e = 0; e < count; ++e)
    if ((st = ce_condsim_prepare(ctxs[e], Rs[e]))) return st;
  ce_batch* b = new ce_batch();
  b->ctxs.assign(ctxs, ctxs + count);
  b->z.assign(z_devs, z_devs + count);
  b->R.assign(Rs, Rs + count);
  b->seeds.assign(seeds, seeds + count);
  b->offs.assign(r_offsets, r_offsets + count);
  b->outs.assign(outs, outs + count);
  if ((st = b->ss.create(nstreams))) { ce_batch_destroy(b); return st; }
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    ce_batch_destroy(b);
    return ce::fail(nullptr, CE_ERR_CUDA, "capture stream");
  }
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = enqueue(b->ss, b->ctxs.data(), b->z.data(), b->R.data(), b->seeds.data(), b->offs.data(), b->outs.data(), count,
                 cap);
    const cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
    if (st == CE_OK && e2 != cudaSuccess) st = ce::cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    if (st == CE_OK) {
      const cudaError_t e3 = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e3 != cudaSuccess) st = ce::cuda_fail(e3, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
  } else {
    st = ce::cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  }
  cudaStreamDestroy(cap);
  if (st != CE_OK) { ce_batch_destroy(b); return st; }
  *out = b;
  return CE_OK;
}

int ce_batch_launch(ce_batch* b, void* stream) {
  if (!b || !b->exec) return ce::fail(nullptr, CE_ERR_ARG, "null batch");
  CE_CUDA_TRY(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
  return CE_OK;
}

void ce_batch_destroy(ce_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->ss.destroy();
  delete b;
}

int ce_autotune(ce_ctx* ctx, int R, void* stream) {
  if (!ctx) return ce::fail(nullptr, CE_ERR_ARG, "null context");
  if (ctx->mode < 0) return ce::fail(ctx, CE_ERR_STATE, "ce_krige_weights has not been called");
  if (!ctx->sqrt_lam) return ce::fail(ctx, CE_ERR_STATE, "the context has no embedding");
  if (R < 1 || R > 4096) return ce::fail(ctx, CE_ERR_ARG, "R must be in [1, 4096]");
  int st = ce_condsim_prepare(ctx, R);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t ybytes = sizeof(float) * (size_t)R * ctx->m * ctx->m;
  float* y = (float*)ce::dalloc(ctx, ybytes);
  if (!y) return ce::fail(ctx, CE_ERR_OOM, "autotune buffer");
  // 1. the unconditional ensemble: the L2 budget of one chunk of the FFT intermediate
  {
    const int budgets[3] = {32, 64, 96};
    cudaEvent_t a, b;
    CE_CUDA_TRY(cudaEventCreate(&a));
    CE_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    int best_mb = ctx->fft_chunk_mb;
    for (int o = 0; o < 3 && st == CE_OK; ++o) {
      ctx->fft_chunk_mb = budgets[o];
      st = ce::fft_unconditional(ctx, R, 1, 0, y, s);   // warm-up (allocates the chunk buffer)
      if (st) break;
      cudaEventRecord(a, s);
      for (int k = 0; k < 3 && st == CE_OK; ++k) st = ce::fft_unconditional(ctx, R, 1, 0, y, s);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) { best = ms; best_mb = budgets[o]; }
    }
    ctx->fft_chunk_mb = best_mb;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st == CE_OK) st = ce::ensure_fft_buffer(ctx, R);
    if (st) { ce::dfree(ctx, y); return st; }
  }
  if (ctx->prec == CE_PREC_FP32 || ctx->prec == CE_PREC_FP64) {   // nothing more to tune
    ce::dfree(ctx, y);
    return CE_OK;
  }
  // 2. the tensor-core correction: 8 or 16 producer warps
  CE_CUDA_TRY(cudaMemsetAsync(y, 0, ybytes, s));
  CE_CUDA_TRY(cudaMemsetAsync(ctx->Bm, 0, sizeof(float) * (size_t)((R + 15) / 16 * 16) * ctx->nobs_pad, s));
  cudaEvent_t a, b;
  CE_CUDA_TRY(cudaEventCreate(&a));
  CE_CUDA_TRY(cudaEventCreate(&b));
  const int options[2] = {8, 16};
  float best = 1e30f;
  int best_w = ctx->tc_producer_warps;
  for (int o = 0; o < 2 && st == CE_OK; ++o) {
    ctx->tc_producer_warps = options[o];
    st = ce::launch_correct(ctx, ctx->Bm, R, y, s);   // warm-up
    if (st) break;
    cudaEventRecord(a, s);
    for (int k = 0; k < 3 && st == CE_OK; ++k) st = ce::launch_correct(ctx, ctx->Bm, R, y, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) { best = ms; best_w = options[o]; }
  }
  ctx->tc_producer_warps = best_w;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ce::dfree(ctx, y);
  if (st) return st;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // extern "C"
