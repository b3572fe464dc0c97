// Tensor-core form of the Kriging correction, step 5 of Section 2:
// v_r = y_r + sum_j C(|g - s_j|) B[j, r] on every grid node (Eq. (condmvn)),
// with the grid x site covariance evaluated per tile and never stored.
//
// One persistent block per SM, warp-specialised:
//   warps 0-7   producers: for a tile of 128 nodes of one grid row and a chunk
//               of 64 sites, evaluate C / sigma^2 (Matern, Section 3.3) in FP32,
//               split it into bf16 hi + lo (both rounded to nearest) and store
//               both in the 128-byte-swizzled K-major layout the MMA reads;
//   warp 13     loader: one bulk async copy per chunk of the pre-split
//               weights sigma^2 B (hi and lo, same layout) and the chunk's
//               site coordinates;
//   warp 12     MMA: allocates tensor memory, and for every chunk issues
//               tcgen05.mma kind::f16 (bf16 in, FP32 accumulate, M=128,
//               N=R padded to 16, K=16) for hi*hi + hi*lo + lo*hi: the
//               low-precision product plus one refinement pass for its
//               residual; the accumulator is double-buffered in tensor memory;
//   warps 8-11  epilogue: tcgen05.ld the accumulator and add it to y in place.
// Stages of shared memory are handed over with mbarriers.  Every wait is
// bounded; on expiry the block records CE_ERR_TIMEOUT, drains its own copies
// and tensor-core work, frees its tensor memory and returns.
#include <cstdint>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
MaternF matern_grid_units(const ce_ctx* ctx);

namespace {

constexpr int TM = 128;            // nodes per tile (MMA M)
constexpr int TK = 64;             // sites per chunk: 128 bytes of bf16 per row
constexpr int NPROD = 256;         // producer threads
constexpr int EPI_WARP0 = 8;       // epilogue warps 8..11
constexpr int MMA_WARP = 12;
constexpr int LOAD_WARP = 13;
constexpr int NTHREADS = 14 * 32;
constexpr uint32_t kWaitLimit = 1u << 22;

struct TcArgs {
  float* y;
  int m, R, Npad, nchunks, tiles, tiles_per_row, stages;
  const uint8_t* bsplit;       // nchunks blocks of block_bytes
  uint32_t block_bytes;        // 1024 (sites) + 2 * Npad * 128 (B hi, B lo)
  uint32_t stage_bytes;        // 32768 (A hi, A lo) + block_bytes
  uint32_t tmem_cols;          // 2 accumulators
  uint32_t acc_stride;         // columns between the two accumulators
  uint32_t idesc;              // tcgen05 instruction descriptor
  float b, c1;                 // exponent factor (log2 units) and (a / b) for nu = 3/2
  int nu3;
  int* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on the phase with the given parity.  Returns false on expiry
// or when another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, int* status) {
  *abort_flag = 1;
  atomicExch(status, CE_ERR_TIMEOUT);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// bf16 bits of x rounded to nearest (ties away from zero), in the upper half.
__device__ __forceinline__ uint32_t bf16_round_bits(float x) { return (__float_as_uint(x) + 0x8000u) & 0xFFFF0000u; }

__device__ __forceinline__ void split_pack(float c0, float c1, uint32_t& hi, uint32_t& lo) {
  const uint32_t h0 = bf16_round_bits(c0), h1 = bf16_round_bits(c1);
  const float l0 = c0 - __uint_as_float(h0), l1 = c1 - __uint_as_float(h1);
  hi = __byte_perm(h0, h1, 0x7632);
  lo = __byte_perm(bf16_round_bits(l0), bf16_round_bits(l1), 0x7632);
}

__global__ void __launch_bounds__(NTHREADS, 1) correct_tc_kernel(const TcArgs p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_a[4], full_b[4], empty_bar[4], acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full_a[s]), NPROD);
      mbar_init(smem_u32(&full_b[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 128);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  const int my_tiles = p.tiles > (int)blockIdx.x ? (p.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const long long M = (long long)p.m * p.m;

  if (warp < EPI_WARP0) {
    // ------------------------------------------------------------ producers
    const int t = threadIdx.x;
    const int c = t & 7;                              // 16-byte chunk: sites 8c .. 8c+7
    const int row0 = 16 * warp + 4 * ((t & 31) >> 3);  // rows row0 .. row0+3 of the tile
    long long it = 0;
    bool ok = true;
    for (int tl = 0; tl < my_tiles && ok; ++tl) {
      const int tile = (int)blockIdx.x + tl * (int)gridDim.x;
      const int gi = tile / p.tiles_per_row;
      const int j0 = (tile % p.tiles_per_row) * TM;
      const float fgi = (float)gi;
      float fgj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) fgj[u] = (float)(j0 + row0 + u);
      for (int kc = 0; kc < p.nchunks; ++kc, ++it) {
        const int s = (int)(it % S);
        const uint32_t ph = (uint32_t)((it / S) & 1);
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &abort_flag)) { ok = false; break; }
        uint8_t* st = smem + (size_t)s * p.stage_bytes;
        // this chunk's sites arrive with the B copy
        if (!mbar_wait(smem_u32(&full_b[s]), ph, &abort_flag)) { ok = false; break; }
        const float4* sites = reinterpret_cast<const float4*>(st + 32768);
        float sxi[8], sxf[8], dy2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 o = sites[j * 8 + c];
          sxi[j] = o.x;
          sxf[j] = o.y;
          const float dy = (fgi - o.z) - o.w;
          dy2[j] = fmaf(dy, dy, 1e-30f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float cv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float dx = (fgj[u] - sxi[j]) - sxf[j];
            const float d2 = fmaf(dx, dx, dy2[j]);
            const float tt = p.b * (d2 * fast_rsqrt(d2));
            const float e = fast_ex2(tt);
            cv[j] = p.nu3 ? fmaf(p.c1, tt, 1.0f) * e : e;
          }
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) split_pack(cv[2 * j], cv[2 * j + 1], hi[j], lo[j]);
          const int row = row0 + u;
          const uint32_t off = (uint32_t)row * 128u + ((uint32_t)(c ^ (row & 7)) << 4);
          *reinterpret_cast<uint4*>(st + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(st + 16384 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&full_a[s]));
      }
    }
    if (!ok) raise_abort(&abort_flag, p.status);
  } else if (warp < MMA_WARP) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                 // tensor-memory lanes 32q .. 32q+31
    const int row = 32 * q + lane;
    for (int tl = 0; tl < my_tiles; ++tl) {
      const int tile = (int)blockIdx.x + tl * (int)gridDim.x;
      const int gi = tile / p.tiles_per_row;
      const int gj = (tile % p.tiles_per_row) * TM + row;
      const int buf = tl & 1;
      if (!mbar_wait(smem_u32(&acc_full[buf]), (uint32_t)((tl >> 1) & 1), &abort_flag)) {
        raise_abort(&abort_flag, p.status);
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * p.acc_stride;
      float* yg = p.y + (long long)gi * p.m + gj;
      for (int c0 = 0; c0 < p.Npad; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (gj < p.m) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int rr = c0 + k;
            if (rr < p.R) yg[(long long)rr * M] += __uint_as_float(r[k]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acc_empty[buf]));
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      bool issued = false;
      for (int tl = 0; tl < my_tiles && ok; ++tl) {
        const int buf = tl & 1;
        if (!mbar_wait(smem_u32(&acc_empty[buf]), (uint32_t)(((tl >> 1) & 1) ^ 1), &abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)buf * p.acc_stride;
        for (int kc = 0; kc < p.nchunks; ++kc, ++it) {
          const int s = (int)(it % S);
          const uint32_t ph = (uint32_t)((it / S) & 1);
          if (!mbar_wait(smem_u32(&full_a[s]), ph, &abort_flag) || !mbar_wait(smem_u32(&full_b[s]), ph, &abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + (size_t)s * p.stage_bytes);
          const uint32_t a_hi = base, a_lo = base + 16384u;
          const uint32_t b_hi = base + 32768u + 1024u, b_lo = b_hi + (uint32_t)p.Npad * 128u;
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
            const uint32_t o = 32u * kk;
            const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
            mma_bf16(d_tmem, sw128_desc(a_hi + o), sw128_desc(b_hi + o), p.idesc, acc);
            mma_bf16(d_tmem, sw128_desc(a_hi + o), sw128_desc(b_lo + o), p.idesc, 1u);
            mma_bf16(d_tmem, sw128_desc(a_lo + o), sw128_desc(b_hi + o), p.idesc, 1u);
          }
          issued = true;
          mma_commit(smem_u32(&empty_bar[s]));
        }
        if (ok) mma_commit(smem_u32(&acc_full[buf]));
      }
      if (!ok) raise_abort(&abort_flag, p.status);
      if (issued) {   // all tensor-core work of this block has finished before the memory is freed
        mma_commit(smem_u32(&drain_bar));
        if (!mbar_wait(smem_u32(&drain_bar), 0u, &abort_flag)) {
          // expiry here means the block is already aborting; one more bounded wait
          for (uint32_t k = 0; k < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0u); ++k) {
          }
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ loader
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      const long long total = (long long)my_tiles * p.nchunks;
      for (; it < total; ++it) {
        const int s = (int)(it % S);
        const uint32_t ph = (uint32_t)((it / S) & 1);
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &abort_flag)) { ok = false; break; }
        const int kc = (int)(it % p.nchunks);
        const uint32_t bar = smem_u32(&full_b[s]);
        mbar_arrive_expect_tx(bar, p.block_bytes);
        bulk_g2s(smem_u32(smem + (size_t)s * p.stage_bytes + 32768), p.bsplit + (size_t)kc * p.block_bytes, p.block_bytes, bar);
      }
      if (!ok) raise_abort(&abort_flag, p.status);
      // copies still in flight land before the block exits
      const long long first = it > S ? it - S : 0;
      for (long long k = first; k < it; ++k) {
        const int s = (int)(k % S);
        const uint32_t ph = (uint32_t)((k / S) & 1);
        for (uint32_t w = 0; w < kWaitLimit && !mbar_try(smem_u32(&full_b[s]), ph); ++w) {
        }
      }
    }
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(p.tmem_cols) : "memory");
  }
}

// Weights sigma^2 B (rows = realizations, padded to Npad) split into bf16 hi + lo
// in the swizzled K-major layout, and the chunk's site coordinates, one block of
// block_bytes per chunk of 64 sites.  Site k of a chunk is stored at slot
// (k % 8) * 8 + k / 8 so that the producers' loads do not collide in banks.
__global__ void prep_b_kernel(const float* __restrict__ B, int ldb, int R, int nobs, int Npad, int nchunks, float scale,
                              const float4* __restrict__ obs, uint8_t* __restrict__ out, uint32_t block_bytes) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_chunk = (long long)Npad * TK;
  if (e < (long long)nchunks * per_chunk) {
    const int kc = (int)(e / per_chunk);
    const int rem = (int)(e % per_chunk);
    const int r = rem / TK, k = rem % TK;
    const int q = kc * TK + k;
    const float v = (r < R && q < nobs) ? B[(long long)r * ldb + q] * scale : 0.f;
    const uint32_t hb = bf16_round_bits(v);
    const uint32_t lb = bf16_round_bits(v - __uint_as_float(hb));
    uint8_t* blk = out + (size_t)kc * block_bytes;
    const uint32_t off = 1024u + (uint32_t)r * 128u + ((uint32_t)((k >> 3) ^ (r & 7)) << 4) + (uint32_t)(k & 7) * 2u;
    *reinterpret_cast<uint16_t*>(blk + off) = (uint16_t)(hb >> 16);
    *reinterpret_cast<uint16_t*>(blk + off + (uint32_t)Npad * 128u) = (uint16_t)(lb >> 16);
    if (r == 0) reinterpret_cast<float4*>(blk)[(k & 7) * 8 + (k >> 3)] = obs[q];
  }
}

}  // namespace

int launch_correct_tc(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  if (ctx->prec != CE_PREC_BF16X3 && ctx->prec != CE_PREC_F16X3) return fail(ctx, CE_ERR_ARG, "unknown precision");
  if (ctx->prec == CE_PREC_F16X3) return fail(ctx, CE_ERR_ARG, "f16x3 correction is not built");
  const int m = ctx->m;
  const int nchunks = ctx->nobs_pad / TK;
  const MaternF mf = matern_grid_units(ctx);
  const int tiles_per_row = (m + TM - 1) / TM;
  const int tiles = m * tiles_per_row;
  int dev = 0, nsm = 0;
  CE_CUDA_TRY(cudaGetDevice(&dev));
  CE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  for (int r0 = 0; r0 < R; r0 += 256) {
    const int Rc = R - r0 < 256 ? R - r0 : 256;
    const int Npad = (Rc + 15) / 16 * 16;
    const uint32_t block_bytes = 1024u + 2u * (uint32_t)Npad * 128u;
    const size_t need = (size_t)nchunks * block_bytes;
    if (ctx->bsplit_bytes < need) {
      dfree(ctx, ctx->Bsplit);
      ctx->Bsplit = dalloc(ctx, need);
      ctx->bsplit_bytes = ctx->Bsplit ? need : 0;
      if (!ctx->Bsplit) return fail(ctx, CE_ERR_OOM, "split weights");
    }
    const long long tot = (long long)nchunks * Npad * TK;
    prep_b_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B + (size_t)r0 * ctx->nobs_pad, ctx->nobs_pad, Rc, ctx->nobs,
                                                                Npad, nchunks, mf.s2, ctx->obs,
                                                                (uint8_t*)ctx->Bsplit, block_bytes);
    TcArgs a;
    a.y = y + (size_t)r0 * m * m;
    a.m = m;
    a.R = Rc;
    a.Npad = Npad;
    a.nchunks = nchunks;
    a.tiles = tiles;
    a.tiles_per_row = tiles_per_row;
    a.bsplit = (const uint8_t*)ctx->Bsplit;
    a.block_bytes = block_bytes;
    a.stage_bytes = 32768u + block_bytes;
    const uint32_t smem_budget = 200u * 1024u;
    a.stages = (int)(smem_budget / a.stage_bytes);
    if (a.stages > 4) a.stages = 4;
    if (a.stages < 2) return fail(ctx, CE_ERR_ARG, "tensor-core stage does not fit in shared memory");
    const uint32_t ncol = Npad <= 32 ? 32u : (Npad <= 64 ? 64u : (Npad <= 128 ? 128u : 256u));
    a.acc_stride = ncol;
    a.tmem_cols = 2 * ncol;
    // kind::f16 descriptor: FP32 accumulate, bf16 A and B, both K-major, N = Npad, M = 128
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Npad >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    a.b = mf.b;
    a.nu3 = ctx->nu == 1.5 ? 1 : 0;
    a.c1 = a.nu3 ? mf.a / mf.b : 0.f;
    a.status = ctx->dev_status;
    const size_t smem = (size_t)a.stages * a.stage_bytes + 1024;
    CE_CUDA_TRY(cudaFuncSetAttribute(correct_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = tiles < nsm ? tiles : nsm;
    correct_tc_kernel<<<grid, NTHREADS, smem, s>>>(a);
    ctx->launches += 2;
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace ce
