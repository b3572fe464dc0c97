// Tensor-core form of the Kriging correction, step 5 of Section 2:
// v_r = y_r + sum_j C(|g - s_j|) B[j, r] on every grid node (Eq. (condmvn)),
// with the grid x site covariance evaluated per tile and never stored.
//
// One persistent block per SM, warp-specialised (NPW producer warps):
//   producers   for a tile of 128 nodes of one grid row and a chunk of sites
//               (64 of a 16-bit kind, 32 of tf32), evaluate 2^11 C (Matern,
//               Section 3.3) in FP32, split it into hi + lo of the operand kind
//               (f16, bf16 or tf32, each rounded to nearest) and store both in
//               the 128-byte-swizzled K-major layout the MMA reads;
//   MMA lane    allocates tensor memory and for every chunk issues tcgen05.mma
//               (kind::f16 or kind::tf32, FP32 accumulate, M = 128, N = R padded
//               to 16): A_hi B_hi into the unit's main accumulator, A_hi B_lo and
//               A_lo B_hi into the tile's cross accumulator, i.e. hi*hi + hi*lo +
//               lo*hi, the low-precision product plus one refinement pass for its
//               residual; main accumulators alternate between two buffers, one
//               unit of at most 512 sites each, and cross accumulators between two
//               buffers, one tile each;
//   4 epilogue  tcgen05.ld each finished unit and add it into a running FP32
//               sum kept in shared memory; after the tile's last unit add
//               (sum + cross) + last unit, scaled, to y by reductions in L2;
//   loader lane claims work items (tiles, possibly of several events) and
//               copies each chunk's pre-split weights sigma^2 B (hi and lo, same
//               layout) into the stage ring with one bulk async copy.
// With AMEM the same kernel computes the solve B = A^-1 E on the tensor cores:
// no producers, the A operand (A^-1 as f16 hi/lo blocks) copied from memory with
// the B operand, and each work item a K part of a tile written as its own partial.
// Producers read a chunk's site coordinates (1 KB, shared by every tile)
// straight from global memory through L1, before they wait for a stage.  A
// shared-memory ring refilled by bulk copies would need a proxy fence between
// the producers' generic reads of a slot and the next async-proxy copy into
// it; without one, fast refills overwrote slots still being read.
// Distances are formed in units of the exponent scale |b| (so that the
// exponent is -d and no extra multiply is needed) from the exact integer part
// and the scaled fraction of the coordinates.  Stages are handed over with
// mbarriers.  Every wait is bounded; on expiry the block records
// CE_ERR_TIMEOUT, drains its own copies and tensor-core work, frees its tensor
// memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
MaternF matern_grid_units(const ce_ctx* ctx);

namespace {

constexpr int TM = 128;            // nodes per tile (MMA M)
// Operand kinds: 16-bit halves (f16 or bf16 hi/lo, kind::f16) or tf32 hi/lo (kind::tf32).
// A row of a chunk is 128 bytes of operands, so a chunk holds 64 sites of a 16-bit kind
// or 32 of tf32, and each MMA takes 32 bytes of K (16 or 8 sites).
enum : int { KIND_F16 = 0, KIND_BF16 = 1, KIND_TF32 = 2 };
template <int KIND> struct Op {
  static constexpr int TK = KIND == KIND_TF32 ? 32 : 64;   // sites per chunk
  static constexpr int SPC = TK / 8;                         // sites per 16-byte piece of a row
};
constexpr uint32_t kWaitLimit = 1u << 22;
// Sites summed in one tensor-memory accumulator before the epilogue adds the partial
// sum to its running sum: the accumulator's FP32 additions lose low bits relative to
// its running magnitude, and partial sums over a few hundred Morton-ordered sites stay
// far smaller than the sum over all sites.
constexpr int kDrainSites = 512;

// One event of a launch: its fields, its operands and its sizes.  The same kernel
// serves the solve B = A^-1 E with the A operand read from memory (AMEM): then the
// rows of a tile are sites, "y" receives per K part one partial product, and the
// fields marked (AMEM) apply.
struct TcEvent {
  float* y;                    // fields of the launch's realizations, R x m x m (AMEM: partial products)
  const uint8_t* bsplit;       // nchunks blocks of bblock bytes: B hi, B lo
  const uint8_t* sites;        // nchunks blocks of the chunk's site records
  const unsigned* bmax;        // f16 operands: bits of max |sigma^2 B| (sets the power-of-two scale)
  const uint8_t* ablk;         // (AMEM) A operand: tiles x nchunks blocks of 32 KB (hi, lo)
  const unsigned* amax;        // (AMEM) bits of max |A| (the A operand's power-of-two scale)
  long long ystride;           // (AMEM) elements between realizations of y
  long long pstride;           // (AMEM) elements between the K parts' partial products
  int m, R, nchunks, tiles_per_row;
  int nitems;                  // work items: tiles (AMEM: tiles x K parts)
  int kparts, cpp;             // (AMEM) K parts per tile and chunks per part
  int drain;                   // chunks accumulated in tensor memory before the epilogue joins them
  int item0;                   // first work item (tile) of the event in the launch's queue
  float absb, c1;              // |exponent factor| (log2 units per grid unit); 2^11 a / b (0 for nu = 1/2)
};

// Events per launch; the descriptors travel in the kernel's parameter space.
constexpr int kMaxEvents = 64;
// Work items published ahead of the roles that take them.
constexpr int kItemRing = 8;

struct TcArgs {
  TcEvent ev[kMaxEvents];
  int nev, items;              // events; work items = the tiles of all events
  unsigned* queue;             // work-queue counter, zero at launch (dynamic)
  int Npad, stages;
  uint32_t bblock;             // 2 * Npad * 128
  uint32_t stage_bytes;        // 32768 (A hi, A lo) + bblock
  uint32_t run_off;            // offset of the epilogue's running sums (128 x Npad floats) after the stages
  uint32_t tmem_cols;          // allocated tensor-memory columns (a power of two >= 4 Npad)
  uint32_t idesc1;             // instruction descriptor, N = Npad
  float a11, a12, a21, a22;    // anisotropic map of the grid-unit offset (ANISO kernels)
  uint32_t epi_wait;           // bound on the epilogue's waits for an accumulator (try_wait rounds)
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

// One test of the phase with the given parity that may suspend the thread for up to
// `ns` nanoseconds; the thread resumes as soon as the phase completes.
__device__ __forceinline__ bool mbar_try_for(uint32_t bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait on the phase with the given parity: at most `limit` tests, each of
// which suspends the thread (up to 2 us) until the phase completes, so a waiting role
// neither polls nor oversleeps.  Returns false on expiry or when another role has
// already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_for(bar, parity, 2000u)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}

// Position in a ring of n barrier slots: the slot and the parity of the
// slot's current phase, advanced by one per chunk.
struct Ring {
  int slot = 0, n;
  uint32_t phase = 0;
  __device__ explicit Ring(int n_) : n(n_) {}
  __device__ __forceinline__ void next() {
    if (++slot == n) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, int* status) {
  *abort_flag = 1;
  atomicExch(status, CE_ERR_TIMEOUT);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
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

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  if constexpr (KIND == KIND_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// 8 consecutive 32-bit columns of this warp's 32 tensor-memory lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// The covariance tile is formed as 2^11 C: C - C_hi is about 2^-11 C, which for
// C below 1/4 would fall under FP16's normal range (2^-14) and lose relative
// precision; scaled, it stays normal down to C ~ 1e-4 (and C_hi down to 3e-8).
// The factor rides on the Matern polynomial's constants, so it costs no
// instruction, and both parts of the tile carry it.  The weights are scaled to
// the top of FP16's range, so their low part needs no factor.  The products with
// a low part (C_hi B_lo and C_lo B_hi) accumulate in their own columns; the
// epilogue adds the two column groups and removes the 2^11 (exact).
constexpr float kLoScale = 2048.f, kLoInv = 1.f / 2048.f;

// bf16 bits of x rounded to nearest (ties away from zero), in the upper half.
__device__ __forceinline__ uint32_t bf16_round_bits(float x) { return (__float_as_uint(x) + 0x8000u) & 0xFFFF0000u; }

// Two f32 -> packed bf16 (first argument in the low half), rounded to nearest even.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
  return d;
}

// Two f32 -> packed f16 (first argument in the low half), rounded to nearest even.
__device__ __forceinline__ uint32_t pack_f16x2(float lo_elem, float hi_elem) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
  return d;
}

// c0, c1 -> hi = round(c), lo = round(c - hi) in bf16 (F16 = false) or f16,
// each pair packed with c0 in the low half.  The producers pass c already
// multiplied by 2^11, so hi and lo carry the same factor (exact).
template <bool F16>
__device__ __forceinline__ void split_pack(float c0, float c1, uint32_t& hi, uint32_t& lo) {
  if constexpr (F16) {
    hi = pack_f16x2(c0, c1);
    __half2 h2;
    memcpy(&h2, &hi, sizeof(h2));
    const float2 hf = __half22float2(h2);
    lo = pack_f16x2(c0 - hf.x, c1 - hf.y);
  } else {
    hi = pack_bf16x2(c0, c1);
    lo = pack_bf16x2(c0 - __uint_as_float(hi << 16), c1 - __uint_as_float(hi & 0xFFFF0000u));
  }
}

// x rounded to tf32 (10 explicit mantissa bits, ties away from zero), as FP32 bits.
__device__ __forceinline__ uint32_t tf32_round_bits(float x) {
  uint32_t d;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(d) : "f"(x));
  return d;
}

// Power-of-two scale 2^k that brings the largest |sigma^2 B| to [2^13, 2^14): the
// f16 weights then use the top of the format's range; 1 when B is all zero.
__device__ __forceinline__ float f16_scale(unsigned maxbits) {
  const float mx = __uint_as_float(maxbits);
  if (!(mx > 0.f)) return 1.f;
  int e;
  frexpf(mx, &e);   // mx = f 2^e, f in [1/2, 1)
  return ldexpf(1.f, max(-120, min(120, 14 - e)));
}

template <int NPW>
struct TcRoles {
  static constexpr int NGROUP = NPW / 8;          // producer groups, one chunk each at a time
  static constexpr int GPROD = 256;               // threads per producer group
  static constexpr int RPT = TM * 8 / GPROD;      // tile rows per producer thread (4)
  static constexpr int EPI0 = NPW;                // 4 epilogue warps
  static constexpr int MMA = NPW + 4;
  static constexpr int BLOAD = NPW + 5;           // lane 0: B copies
  static constexpr int NTHREADS = (NPW + 6) * 32;
  // registers are allocated per scheduler: 16384 for the ceil(warps / 4) warps it holds
  static constexpr int MAXREG = NPW == 0 ? 128 : 16384 / (((NPW + 6 + 3) / 4) * 32) / 8 * 8;
};

template <int NPW, int KIND, bool NU3, bool ANISO, bool MULTI, bool AMEM>
__global__ void __maxnreg__(TcRoles<NPW>::MAXREG) correct_tc_kernel(const __grid_constant__ TcArgs p) {
  static_assert(!AMEM || NPW == 0, "the memory-operand form has no producers");
  using Ro = TcRoles<NPW>;
  constexpr int RPT = Ro::RPT;
  constexpr int TK = Op<KIND>::TK, SPC = Op<KIND>::SPC;
  constexpr bool F16 = KIND == KIND_F16;
  // warps that take every work item from the ring: producers, epilogue, MMA
  constexpr uint32_t kConsumers = NPW + 5;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // first 1024-byte-aligned shared address of the dynamic buffer
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  __shared__ __align__(8) uint64_t full_a[4], full_b[4], empty_bar[4], acc_full[2],
      acc_empty[2], tile_empty[2], drain_bar, item_full[kItemRing], item_empty[kItemRing];
  __shared__ int2 item_slot[kItemRing];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full_a[s]), Ro::GPROD);
      mbar_init(smem_u32(&full_b[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 128);
    }
    for (int k = 0; k < kItemRing; ++k) {
      mbar_init(smem_u32(&item_full[k]), 1);
      mbar_init(smem_u32(&item_empty[k]), kConsumers);
    }
    mbar_init(smem_u32(&tile_empty[0]), 128);
    mbar_init(smem_u32(&tile_empty[1]), 128);
    mbar_init(smem_u32(&drain_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == Ro::MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  // The k-th work item of this block, (event, tile) or event -1 at the end of the
  // queue, for a whole warp: every lane waits (bounded) for the ring slot, the lanes
  // agree on the outcome, and lane 0 releases the slot.  False on expiry or abort.
  // The k-th item of a static schedule: block b takes items b, b + gridDim.x, ...
  auto static_item = [&](uint32_t k) -> int2 {
    const int it = (int)blockIdx.x + (int)k * (int)gridDim.x;
    if (it >= p.items) return make_int2(-1, 0);
    int e = 0;
    while (e + 1 < p.nev && p.ev[e + 1].item0 <= it) ++e;
    return make_int2(e, it - p.ev[e].item0);
  };
  auto take_item = [&](uint32_t k, int2& item) -> bool {
    if constexpr (!MULTI) {
      item = static_item(k);
      return true;
    }
    const int slot = (int)(k % kItemRing);
    bool got = mbar_wait(smem_u32(&item_full[slot]), (k / kItemRing) & 1u, &abort_flag);
    got = __all_sync(0xffffffffu, got);
    if (got) item = item_slot[slot];
    __syncwarp();
    if (got && lane == 0) mbar_arrive(smem_u32(&item_empty[slot]));
    return got;
  };

  // The same for one thread (the MMA warp's lane 0, which counts for its warp).
  auto take_item_one = [&](uint32_t k, int2& item) -> bool {
    if constexpr (!MULTI) {
      item = static_item(k);
      return true;
    }
    const int slot = (int)(k % kItemRing);
    if (!mbar_wait(smem_u32(&item_full[slot]), (k / kItemRing) & 1u, &abort_flag)) return false;
    item = item_slot[slot];
    mbar_arrive(smem_u32(&item_empty[slot]));
    return true;
  };

  // The tile of a work item and its chunks [k0, k1): every chunk of the tile, or (AMEM)
  // the item's K part of them.
  auto item_range = [&](const TcEvent& ev, int y, int& tile, int& k0, int& k1) {
    if constexpr (AMEM) {
      tile = y / ev.kparts;
      k0 = (y % ev.kparts) * ev.cpp;
      k1 = min(ev.nchunks, k0 + ev.cpp);
    } else {
      tile = y;
      k0 = 0;
      k1 = ev.nchunks;
    }
  };

  if (warp < Ro::EPI0) {
    // ------------------------------------------------------------ producers
    // Groups of 8 warps take alternate chunks, so one group's barrier waits and
    // stores overlap the other group's evaluation.
    const int grp = threadIdx.x / Ro::GPROD;
    const int t = threadIdx.x % Ro::GPROD;
    const int c = t & 7;                  // 16-byte piece of a row: sites SPC c .. SPC c + SPC - 1
    const int row0 = (t >> 3) * RPT;      // tile rows row0 .. row0+RPT-1
    // The stage ring advances with every chunk of the block (both groups'), as
    // small counters: no division on the per-chunk path.
    Ring stage_ring(S);
    int gsel = 0;
    bool ok = true;
    for (uint32_t k = 0; ok; ++k) {
      int2 item;
      if (!take_item(k, item)) { ok = false; break; }
      if (item.x < 0) break;
      const TcEvent& ev = p.ev[MULTI ? item.x : 0];   // one event: fixed parameter offsets
      const float absb = ev.absb, c1 = ev.c1;
      // per-row shift of the offset (one node along x per row of the tile); anisotropic:
      // its image under the map, whose first column is (a11, a21)
      float ub[RPT], vb[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        ub[u] = ANISO ? (float)u * absb * p.a11 : (float)u * absb;
        vb[u] = ANISO ? (float)u * absb * p.a21 : 0.f;
      }
      // the event's fields in registers (a parameter-space read per use would be slow)
      const int nchunks = ev.nchunks;
      const float4* __restrict__ sites = reinterpret_cast<const float4*>(ev.sites);
      const int tpr = ev.tiles_per_row;
      const float fgi = (float)(item.y / tpr);
      const float fgj0 = (float)((item.y % tpr) * TM + row0);
      for (int kc = 0; kc < nchunks; ++kc, stage_ring.next(), gsel = gsel + 1 == Ro::NGROUP ? 0 : gsel + 1) {
        if (gsel != grp) continue;
        // isotropic: dx0 = the x offset, dy2 = dy^2; anisotropic: the two components of
        // the mapped offset (u, v) of the tile's first row
        float dx0[SPC], dy2[SPC];
        const float4* __restrict__ sp = sites + (size_t)kc * TK;
#pragma unroll
        for (int j = 0; j < SPC; ++j) {
          const float4 o = __ldg(sp + j * 8 + c);
          const float dx = fmaf(fgj0 - o.x, absb, -o.y);
          const float dy = fmaf(fgi - o.z, absb, -o.w);
          if (ANISO) {
            dx0[j] = fmaf(p.a11, dx, p.a12 * dy);
            dy2[j] = fmaf(p.a21, dx, p.a22 * dy);
          } else {
            dx0[j] = dx;
            dy2[j] = fmaf(dy, dy, 1e-30f);
          }
        }
        const int s = stage_ring.slot;
        if (!mbar_wait(smem_u32(&empty_bar[s]), stage_ring.phase ^ 1u, &abort_flag)) { ok = false; break; }
        const uint32_t st = smem_base + (uint32_t)s * p.stage_bytes;
#pragma unroll
        for (int h = 0; h < RPT; h += 2) {
          float cv[2][SPC];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < SPC; ++j) {
              const float dx = (h + u) ? dx0[j] + ub[h + u] : dx0[j];
              float d2;
              if (ANISO) {
                const float dv = (h + u) ? dy2[j] + vb[h + u] : dy2[j];
                d2 = fmaf(dx, dx, fmaf(dv, dv, 1e-30f));
              } else {
                d2 = fmaf(dx, dx, dy2[j]);
              }
              // |b| d (distances are in units of the exponent scale) and 2^-|b| d
              float dd;
              asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(dd) : "f"(d2));
              const float e = fast_ex2(-dd);
              // 2^11 C: c1 holds 2^11 a / b, so the factor costs nothing for nu = 3/2
              cv[u][j] = NU3 ? fmaf(-c1, dd, kLoScale) * e : e * kLoScale;
            }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint32_t hi[4], lo[4];
            if constexpr (KIND == KIND_TF32) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                hi[j] = tf32_round_bits(cv[u][j]);
                lo[j] = tf32_round_bits(cv[u][j] - __uint_as_float(hi[j]));
              }
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j) split_pack<F16>(cv[u][2 * j], cv[u][2 * j + 1], hi[j], lo[j]);
            }
            const int row = row0 + h + u;
            const uint32_t off = st + (uint32_t)row * 128u + ((uint32_t)(c ^ (row & 7)) << 4);
            sts128(off, hi[0], hi[1], hi[2], hi[3]);
            sts128(off + 16384u, lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&full_a[s]));
      }
    }
    if (!ok) raise_abort(&abort_flag, p.status);
  } else if (warp < Ro::MMA) {
    // ------------------------------------------------------------ epilogue
    // Tensor memory holds two main accumulators (C_hi B_hi) used by alternate units
    // of ev.drain chunks, each unit summed from zero, and two cross accumulators
    // (C_hi B_lo + C_lo B_hi, about 2^-11 of the main terms) used by alternate tiles;
    // the running sum of a tile's finished units is kept in shared memory by this
    // role (each thread its row: columns in float4 groups, rows adjacent).  No FP32
    // accumulator in tensor memory therefore runs over more than ev.drain chunks of
    // the large terms, and the next tile's cross products never wait for this
    // tile's total.  After the last unit the total is added to y by reductions
    // performed in L2 (nothing to wait for here; one thread's reductions to one
    // address apply in program order).
    const int q = warp & 3;                 // tensor-memory lanes 32q .. 32q+31
    const int row = 32 * q + lane;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    float4* run4 = reinterpret_cast<float4*>(smem_raw + (smem_base - smem_u32(smem_raw)) + p.run_off) + row;
    uint32_t unit = 0;
    bool ok = true;
    for (uint32_t k = 0; ok; ++k) {
      int2 item;
      if (!take_item(k, item)) { ok = false; break; }
      if (item.x < 0) break;
      const TcEvent& ev = p.ev[MULTI ? item.x : 0];   // one event: fixed parameter offsets
      int tile, k0, k1;
      item_range(ev, item.y, tile, k0, k1);
      const int units = (k1 - k0 + ev.drain - 1) / ev.drain;
      const int em = ev.m, eR = ev.R;
      float oscale;
      long long M;
      float* __restrict__ yg;
      bool live;
      if constexpr (AMEM) {
        // exact powers of two: the scales of the two f16 operands; one partial product per K part
        oscale = 1.0f / (f16_scale(*ev.amax) * f16_scale(*ev.bmax));
        M = ev.ystride;
        const int i = tile * TM + row;
        yg = ev.y + (long long)(item.y % ev.kparts) * ev.pstride + i;
        live = i < em;
      } else {
        // exact powers of two: the 2^11 of the covariance tile and the f16 weight scale
        oscale = kLoInv * (F16 ? 1.0f / f16_scale(*ev.bmax) : 1.0f);
        M = (long long)em * em;
        const int gi = tile / ev.tiles_per_row;
        const int gj = (tile % ev.tiles_per_row) * TM + row;
        yg = ev.y + (long long)gi * em + gj;
        live = gj < em;
      }
      for (int u = 0; u < units; ++u, ++unit) {
        const int buf = (int)(unit & 1u);
        // bounded by the launch's epi_wait (a host-set limit), the same in every lane
        bool got = mbar_wait(smem_u32(&acc_full[buf]), (unit >> 1) & 1u, &abort_flag, p.epi_wait);
        if (!__all_sync(0xffffffffu, got)) {
          raise_abort(&abort_flag, p.status);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t t_main = tmem_base + lanes + (uint32_t)buf * (uint32_t)p.Npad;
        const uint32_t t_cross = tmem_base + lanes + (2u + (k & 1u)) * (uint32_t)p.Npad;
        const bool first = u == 0, last = u + 1 == units;
        if (last) {
          // the tile's total: (running sum + cross accumulator) + last unit, scaled
          float* __restrict__ yp = yg;
          for (int c0 = 0; c0 < p.Npad; c0 += 8) {
            uint32_t r[8], rc[8];
            tmem_ld8(t_main + (uint32_t)c0, r);
            tmem_ld8(t_cross + (uint32_t)c0, rc);
            float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
            if (!first) {
              s0 = run4[(c0 >> 2) * TM];
              s1 = run4[((c0 >> 2) + 1) * TM];
            }
            tmem_wait_ld();
            const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
            if (live) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                if (c0 + j < eR) {
                  const float cs = first ? __uint_as_float(rc[j]) : sv[j] + __uint_as_float(rc[j]);
                  const float v = (cs + __uint_as_float(r[j])) * oscale;
                  if constexpr (AMEM) {
                    *yp = v;   // this K part's own partial product
                  } else {
                    atomicAdd(yp, v);
                  }
                }
                yp += M;
              }
            }
          }
          tc_fence_before();
          mbar_arrive(smem_u32(&tile_empty[k & 1u]));   // this tile's cross accumulator is read
        } else {
          // running sum (+)= this unit's main accumulator
          for (int c0 = 0; c0 < p.Npad; c0 += 8) {
            uint32_t r[8];
            tmem_ld8(t_main + (uint32_t)c0, r);
            float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
            if (!first) {
              s0 = run4[(c0 >> 2) * TM];
              s1 = run4[((c0 >> 2) + 1) * TM];
            }
            tmem_wait_ld();
            if (first) {
              s0 = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
              s1 = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
            } else {
              s0 = make_float4(s0.x + __uint_as_float(r[0]), s0.y + __uint_as_float(r[1]), s0.z + __uint_as_float(r[2]),
                               s0.w + __uint_as_float(r[3]));
              s1 = make_float4(s1.x + __uint_as_float(r[4]), s1.y + __uint_as_float(r[5]), s1.z + __uint_as_float(r[6]),
                               s1.w + __uint_as_float(r[7]));
            }
            run4[(c0 >> 2) * TM] = s0;
            run4[((c0 >> 2) + 1) * TM] = s1;
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&acc_empty[buf]));
      }
    }
  } else if (warp == Ro::MMA) {
    // ------------------------------------------------------------ MMA issue
    Ring ring(S);
    bool ok = true;
    bool issued = false;
    uint32_t unit = 0;
    // lane 0 alone walks the items (the other lanes wait at the end: lanes parked at a
    // per-item warp barrier cost the issuing lane measurable time)
    for (uint32_t k = 0; ok && lane == 0; ++k) {
      int2 item;
      if (!take_item_one(k, item)) { ok = false; break; }
      if (item.x < 0) break;
      const TcEvent& ev = p.ev[MULTI ? item.x : 0];   // one event: fixed parameter offsets
      if (lane == 0) {
        // the cross accumulator and the running sum of the previous tile have been read
        // the cross accumulator of this tile's parity: read by the epilogue two tiles ago
        if (!mbar_wait(smem_u32(&tile_empty[k & 1u]), ((k >> 1) & 1u) ^ 1u, &abort_flag)) ok = false;
        const uint32_t t_cross = tmem_base + (2u + (k & 1u)) * (uint32_t)p.Npad;
        uint32_t t_main = tmem_base;
        int kin = 0;   // chunk within the current accumulation unit
        int tile, k0, k1;
        item_range(ev, item.y, tile, k0, k1);
        const int drain = ev.drain;
        for (int kc = k0; kc < k1 && ok; ++kc, ring.next()) {
          if (kin == 0) {
            const int buf = (int)(unit & 1u);
            if (!mbar_wait(smem_u32(&acc_empty[buf]), ((unit >> 1) & 1u) ^ 1u, &abort_flag)) { ok = false; break; }
            tc_fence_after();
            t_main = tmem_base + (uint32_t)buf * (uint32_t)p.Npad;
          }
          const int s = ring.slot;
          const uint32_t ph = ring.phase;
          // (AMEM: the A operand arrives with B, on full_b)
          if (!mbar_wait(smem_u32(&full_b[s]), ph, &abort_flag) ||
              (!AMEM && !mbar_wait(smem_u32(&full_a[s]), ph, &abort_flag))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_base + (uint32_t)s * p.stage_bytes;
          // the unit's main accumulator: C_hi B_hi; the tile's cross accumulator: C_hi B_lo + C_lo B_hi
          // (all with the covariance tile's factor 2^11)
          const uint64_t da_hi = sw128_desc(base), da_lo = sw128_desc(base + 16384u);
          const uint64_t db_hi = sw128_desc(base + 32768u), db_lo = sw128_desc(base + 32768u + (uint32_t)p.Npad * 128u);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // 4 MMAs of 32 bytes of K (16 or 8 sites) per chunk
            const uint64_t o = 2u * kk;   // 32 bytes along K, in the descriptor's 16-byte units
            mma_issue<KIND>(t_main, da_hi + o, db_hi + o, p.idesc1, (kin > 0 || kk > 0) ? 1u : 0u);
            mma_issue<KIND>(t_cross, da_hi + o, db_lo + o, p.idesc1, (kc > k0 || kk > 0) ? 1u : 0u);
            mma_issue<KIND>(t_cross, da_lo + o, db_hi + o, p.idesc1, 1u);
          }
          issued = true;
          mma_commit(smem_u32(&empty_bar[s]));
          if (++kin == drain || kc + 1 == k1) {   // unit complete: hand it to the epilogue
            mma_commit(smem_u32(&acc_full[unit & 1u]));
            ++unit;
            kin = 0;
          }
        }
      }
    }
    if (lane == 0) {
      if (!ok) raise_abort(&abort_flag, p.status);
      if (issued) {   // all tensor-core work of this block has finished before the memory is freed
        mma_commit(smem_u32(&drain_bar));
        if (!mbar_wait(smem_u32(&drain_bar), 0u, &abort_flag)) {
          // expiry here means the block is already aborting; one more bounded wait
          for (uint32_t w = 0; w < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0u); ++w) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == Ro::BLOAD) {
    // ------------------------------------------------------------ work queue and B copies
    // Lane 0 takes the block's next work item and copies the item's chunks of split
    // weights into the stage ring.  Items are the tiles of the launch's events in
    // order.  Dynamic schedule (launches over several events): it claims the item from
    // the launch's queue (an atomic counter) and publishes it in the item ring for the
    // other roles, past the last one event -1; static schedule (one event): every role
    // computes the same sequence itself.
    if (lane == 0) {
      long long copies = 0;
      bool ok = true;
      Ring ring(S);
      for (uint32_t k = 0;; ++k) {
        int2 item;
        if constexpr (MULTI) {
          const int slot = (int)(k % kItemRing);
          if (k >= kItemRing &&
              !mbar_wait(smem_u32(&item_empty[slot]), ((k / kItemRing) - 1u) & 1u, &abort_flag)) {
            ok = false;
            break;
          }
          const int it = (int)atomicAdd(p.queue, 1u);
          int e = -1;
          if (it < p.items) {
            e = 0;
            while (e + 1 < p.nev && p.ev[e + 1].item0 <= it) ++e;
          }
          item = make_int2(e, e < 0 ? 0 : it - p.ev[e].item0);
          item_slot[slot] = item;
          mbar_arrive(smem_u32(&item_full[slot]));   // release: the slot is written
        } else {
          item = static_item(k);
        }
        if (item.x < 0) break;
        const TcEvent& ev = p.ev[item.x];
        int tile, k0, k1;
        item_range(ev, item.y, tile, k0, k1);
        const uint8_t* bsplit = ev.bsplit;
        for (int kc = k0; kc < k1; ++kc, ++copies, ring.next()) {
          const int s = ring.slot;
          if (!mbar_wait(smem_u32(&empty_bar[s]), ring.phase ^ 1u, &abort_flag)) { ok = false; break; }
          const uint32_t bar = smem_u32(&full_b[s]);
          const uint32_t dst = smem_base + (uint32_t)s * p.stage_bytes;
          if constexpr (AMEM) {
            // the A block of (tile, chunk) and the B block of the chunk, on one barrier
            mbar_arrive_expect_tx(bar, 32768u + p.bblock);
            bulk_g2s(dst, ev.ablk + ((size_t)tile * ev.nchunks + kc) * 32768u, 32768u, bar);
          } else {
            mbar_arrive_expect_tx(bar, p.bblock);
          }
          bulk_g2s(dst + 32768u, bsplit + (size_t)kc * p.bblock, p.bblock, bar);
        }
        if (!ok) break;
      }
      if (!ok) raise_abort(&abort_flag, p.status);
      // copies still in flight land before the block exits
      for (long long k = copies > S ? copies - S : 0; k < copies; ++k) {
        const uint32_t bar = smem_u32(&full_b[(int)(k % S)]);
        const uint32_t ph = (uint32_t)((k / S) & 1);
        for (uint32_t w = 0; w < kWaitLimit && !mbar_try(bar, ph); ++w) {
        }
      }
    }
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == Ro::MMA) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(p.tmem_cols) : "memory");
  }
}

// Weights sigma^2 B (rows = realizations, padded to Npad) split into hi + lo of the
// operand kind (f16 with the power-of-two scale of f16_scale, bf16, or tf32) in the
// swizzled K-major layout, bblock bytes per chunk of TK sites; and the chunk's site
// records (x integer part, x fraction * |b|, y integer part, y fraction * |b|), site k
// of a chunk at slot (k % SPC) * 8 + k / SPC so that the producers' loads do not
// collide in banks.
template <int KIND>
__global__ void prep_b_kernel(const float* __restrict__ B, int ldb, int R, int nobs, int Npad, int nchunks, float scale,
                              const float4* __restrict__ obs, float absb, uint8_t* __restrict__ bout, uint32_t bblock,
                              float4* __restrict__ sout, const unsigned* __restrict__ bmax) {
  constexpr int TK = Op<KIND>::TK, SPC = Op<KIND>::SPC;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_chunk = (long long)Npad * TK;
  if (e < (long long)nchunks * per_chunk) {
    const int kc = (int)(e / per_chunk);
    const int rem = (int)(e % per_chunk);
    const int r = rem / TK, k = rem % TK;
    const int q = kc * TK + k;
    float v = (r < R && q < nobs) ? B[(long long)r * ldb + q] * scale : 0.f;
    uint8_t* blk = bout + (size_t)kc * bblock;
    const uint32_t row = (uint32_t)r * 128u + ((uint32_t)((k / SPC) ^ (r & 7)) << 4);
    if constexpr (KIND == KIND_TF32) {
      const uint32_t h = tf32_round_bits(v);
      const uint32_t off = row + (uint32_t)(k % SPC) * 4u;
      *reinterpret_cast<uint32_t*>(blk + off) = h;
      *reinterpret_cast<uint32_t*>(blk + off + (uint32_t)Npad * 128u) = tf32_round_bits(v - __uint_as_float(h));
    } else {
      uint16_t hb, lb;
      if constexpr (KIND == KIND_F16) {
        v *= f16_scale(*bmax);
        const __half h = __float2half_rn(v);
        hb = __half_as_ushort(h);
        lb = __half_as_ushort(__float2half_rn(v - __half2float(h)));
      } else {
        const uint32_t h = bf16_round_bits(v);
        hb = (uint16_t)(h >> 16);
        lb = (uint16_t)(bf16_round_bits(v - __uint_as_float(h)) >> 16);
      }
      const uint32_t off = row + (uint32_t)(k % SPC) * 2u;
      *reinterpret_cast<uint16_t*>(blk + off) = hb;
      *reinterpret_cast<uint16_t*>(blk + off + (uint32_t)Npad * 128u) = lb;
    }
    if (r == 0) {
      const float4 o = obs[q];
      sout[(size_t)kc * TK + (k % SPC) * 8 + k / SPC] = make_float4(o.x, o.y * absb, o.z, o.w * absb);
    }
  }
}

// max |scale * B| over the R x nobs block, as float bits (nonnegative floats order as integers).
__global__ void absmax_kernel(const float* __restrict__ B, int ldb, int R, int nobs, float scale, unsigned* __restrict__ out) {
  unsigned mx = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)R * nobs;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / nobs), q = (int)(e % nobs);
    mx = max(mx, __float_as_uint(fabsf(B[(long long)r * ldb + q] * scale)));
  }
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

template <int NPW, int KIND, bool NU3, bool ANISO = false, bool MULTI = false, bool AMEM = false>
int launch_tc(const TcArgs& a, size_t smem, cudaStream_t s) {
  CE_CUDA_TRY(cudaFuncSetAttribute(correct_tc_kernel<NPW, KIND, NU3, ANISO, MULTI, AMEM>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nsm = 0, dev = 0;
  CE_CUDA_TRY(cudaGetDevice(&dev));
  CE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = a.items < nsm ? a.items : nsm;
  correct_tc_kernel<NPW, KIND, NU3, ANISO, MULTI, AMEM><<<grid, TcRoles<NPW>::NTHREADS, smem, s>>>(a);
  return CE_OK;
}

// The kernel instance for the operand kind, smoothness, anisotropy and producer count
// (tf32, the anisotropic covariance and launches over several events use 16 producer
// warps; several events are isotropic).
template <int KIND>
int launch_tc_kind(const TcArgs& a, size_t smem, cudaStream_t s, bool aniso, bool nu3, int npw, bool multi) {
  if (multi) return nu3 ? launch_tc<16, KIND, true, false, true>(a, smem, s) : launch_tc<16, KIND, false, false, true>(a, smem, s);
  if (aniso) return nu3 ? launch_tc<16, KIND, true, true>(a, smem, s) : launch_tc<16, KIND, false, true>(a, smem, s);
  if constexpr (KIND != KIND_TF32) {
    if (npw == 8) return nu3 ? launch_tc<8, KIND, true>(a, smem, s) : launch_tc<8, KIND, false>(a, smem, s);
  }
  return nu3 ? launch_tc<16, KIND, true>(a, smem, s) : launch_tc<16, KIND, false>(a, smem, s);
}

template <int KIND>
void launch_prep(const float* Bc, int ldb, int R, int nobs, int Npad, int nchunks, float scale, const float4* obs, float absb,
                 uint8_t* bbuf, uint32_t bblock, float4* sbuf, const unsigned* bmax, cudaStream_t s) {
  const long long tot = (long long)nchunks * Npad * Op<KIND>::TK;
  prep_b_kernel<KIND><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Bc, ldb, R, nobs, Npad, nchunks, scale, obs, absb, bbuf,
                                                                     bblock, sbuf, bmax);
}

// A^-1 (the FP32 pair hi + lo, n x n, leading dimension lda) as f16 hi and lo blocks of
// 128 rows x 64 columns in the swizzled K-major layout of the MMA's A operand, block
// (row tile t, chunk c) at (t nchunks + c) x 32 KB, scaled by the power of two
// f16_scale(*amax); rows and columns past n are zero.
__global__ void prep_a_kernel(const float* __restrict__ hi, const float* __restrict__ lo, int lda, int n, int mtiles,
                              int nchunks, const unsigned* __restrict__ amax, uint8_t* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long cols = (long long)nchunks * 64;
  if (e >= (long long)mtiles * TM * cols) return;
  const int i = (int)(e / cols), j = (int)(e % cols);
  float v = (i < n && j < n) ? hi[(long long)i * lda + j] + lo[(long long)i * lda + j] : 0.f;
  v *= f16_scale(*amax);
  const __half h = __float2half_rn(v);
  const uint16_t hb = __half_as_ushort(h), lb = __half_as_ushort(__float2half_rn(v - __half2float(h)));
  const int r = i % TM, kap = j % 64;
  uint8_t* blk = out + ((size_t)(i / TM) * nchunks + (size_t)(j / 64)) * 32768u;
  const uint32_t off = (uint32_t)r * 128u + ((uint32_t)((kap / 8) ^ (r & 7)) << 4) + (uint32_t)(kap % 8) * 2u;
  *reinterpret_cast<uint16_t*>(blk + off) = hb;
  *reinterpret_cast<uint16_t*>(blk + off + 16384u) = lb;
}

// B[r][i] = the sum of the K parts' partial products part[k][r][i] (row stride ldp), in
// the order of k, kept as an unevaluated float pair (TwoSum) and rounded once.
__global__ void solve_join_kernel(const float* __restrict__ part, long long pstride, int kparts, int R, int n, int ldp,
                                  float* __restrict__ B, int ldb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * n) return;
  const int r = (int)(e / n), i = (int)(e % n);
  const float* pp = part + (long long)r * ldp + i;
  float hi = 0.f, lo = 0.f;
  for (int k = 0; k < kparts; ++k) {
    const float v = pp[k * pstride];
    const float t = __fadd_rn(hi, v);
    const float z = __fsub_rn(t, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(v, z));
    hi = t;
  }
  B[(long long)r * ldb + i] = hi + lo;
}

}  // namespace


// Device buffer for the split weights and site records of operands of up to 128 rows
// (realizations), in whichever operand kind needs more (tf32: twice the chunks of half
// the sites).
int ensure_bsplit(ce_ctx* ctx, int R) {
  const int Rc = R < 128 ? R : 128;
  const int Npad = (Rc + 15) / 16 * 16;
  // per chunk: the split weights (2 Npad rows of 128 bytes) and 16 bytes of site record per site
  const size_t per16 = (size_t)(ctx->nobs_pad / Op<KIND_F16>::TK) * (2u * (size_t)Npad * 128u + 16u * Op<KIND_F16>::TK);
  const size_t per32 = (size_t)(ctx->nobs_pad / Op<KIND_TF32>::TK) * (2u * (size_t)Npad * 128u + 16u * Op<KIND_TF32>::TK);
  const size_t need = (per16 > per32 ? per16 : per32) + 16;
  if (ctx->bsplit_bytes >= need) return CE_OK;
  dfree(ctx, ctx->Bsplit);
  ctx->Bsplit = dalloc(ctx, need);
  ctx->bsplit_bytes = ctx->Bsplit ? need : 0;
  if (!ctx->Bsplit) return fail(ctx, CE_ERR_OOM, "split weights");
  return CE_OK;
}

namespace {

int tc_kind(const ce_ctx* ctx) {
  return ctx->prec == CE_PREC_F16X3 ? KIND_F16 : (ctx->prec == CE_PREC_BF16X3 ? KIND_BF16 : KIND_TF32);
}

int tc_sites_per_chunk(int kind) { return kind == KIND_TF32 ? Op<KIND_TF32>::TK : Op<KIND_F16>::TK; }

// Where a context's split weights, site records and f16 scale live for operands of Npad rows.
struct TcBuffers {
  uint8_t* bsplit;
  uint8_t* sites;
  unsigned* bmax;
  int nchunks;
  uint32_t bblock;
};

TcBuffers tc_buffers(ce_ctx* ctx, int Npad, int kind) {
  const int TK = tc_sites_per_chunk(kind);
  TcBuffers b;
  b.nchunks = ctx->nobs_pad / TK;   // nobs_pad is a multiple of 128
  b.bblock = 2u * (uint32_t)Npad * 128u;
  b.bsplit = (uint8_t*)ctx->Bsplit;
  b.sites = b.bsplit + (size_t)b.nchunks * b.bblock;
  b.bmax = reinterpret_cast<unsigned*>(b.sites + (size_t)b.nchunks * TK * 16u);
  return b;
}

// The descriptor of realizations [r0, r0 + Rc) of a context (item0 is set by tc_launch).
TcEvent tc_event(ce_ctx* ctx, int Rc, int Npad, float* y) {
  const TcBuffers b = tc_buffers(ctx, Npad, tc_kind(ctx));
  const MaternF mf = matern_grid_units(ctx);
  const int TK = tc_sites_per_chunk(tc_kind(ctx));
  TcEvent ev;
  ev.y = y;
  ev.bsplit = b.bsplit;
  ev.sites = b.sites;
  ev.bmax = b.bmax;
  ev.m = ctx->m;
  ev.R = Rc;
  ev.nchunks = b.nchunks;
  ev.tiles_per_row = (ctx->m + TM - 1) / TM;
  ev.nitems = ctx->m * ev.tiles_per_row;
  ev.ablk = nullptr;
  ev.amax = nullptr;
  ev.ystride = ev.pstride = 0;
  ev.kparts = 1;
  ev.cpp = b.nchunks;
  {   // units of at most kDrainSites sites, balanced over the tile's chunks
    const int per_unit = kDrainSites / TK;
    const int units = (b.nchunks + per_unit - 1) / per_unit;
    ev.drain = (b.nchunks + units - 1) / units;
  }
  ev.item0 = 0;
  ev.absb = -mf.b;
  ev.c1 = ctx->nu == 1.5 ? mf.a / mf.b * kLoScale : 0.f;
  return ev;
}

// One persistent launch over the tiles of events ev[0 .. nev) (nev <= kMaxEvents), all
// with operands of the same kind and Npad rows: the work-queue counter is cleared on
// the stream first.
int tc_launch(ce_ctx* owner, TcEvent* ev, int nev, int kind, int Npad, bool nu3, const Aniso& ad, cudaStream_t s,
              bool amem = false) {
  TcArgs a;
  int items = 0;
  for (int e = 0; e < nev; ++e) {
    ev[e].item0 = items;
    items += ev[e].nitems;
    a.ev[e] = ev[e];
  }
  a.nev = nev;
  a.items = items;
  a.queue = owner->queue;
  a.Npad = Npad;
  a.bblock = 2u * (uint32_t)Npad * 128u;
  a.stage_bytes = 32768u + a.bblock;
  // the epilogue's running sums (128 rows x Npad FP32) after the stages
  const uint32_t run_bytes = 128u * 4u * (uint32_t)Npad;
  const uint32_t budget = 224u * 1024u - 1024u - run_bytes;
  a.stages = (int)(budget / a.stage_bytes);
  if (a.stages > 4) a.stages = 4;
  if (a.stages < 2) return fail(owner, CE_ERR_ARG, "tensor-core stage does not fit in shared memory");
  // two main and two cross accumulators: 4 Npad <= 512 columns
  uint32_t ncol = 32;
  while (ncol < 4u * (uint32_t)Npad) ncol <<= 1;
  a.tmem_cols = ncol;
  // instruction descriptor: FP32 accumulate, A and B K-major, M = 128, N = Npad; operand
  // format field 0 = f16, 1 = bf16 (kind::f16), 2 = tf32 (kind::tf32)
  const uint32_t fmt = (uint32_t)kind;
  const uint32_t ibase = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TM >> 4) << 24);
  a.idesc1 = ibase | ((uint32_t)(Npad >> 3) << 17);
  a.a11 = (float)ad.a11;
  a.a12 = (float)ad.a12;
  a.a21 = (float)ad.a21;
  a.a22 = (float)ad.a22;
  a.epi_wait = owner->wait_limit;
  a.status = owner->dev_status;
  a.run_off = (uint32_t)a.stages * a.stage_bytes;
  const size_t smem = (size_t)a.run_off + run_bytes + 1024;
  const int npw = owner->tc_producer_warps == 8 ? 8 : 16;
  // several events: blocks claim tiles from the queue; one event: equal tiles, a static schedule
  const bool multi = nev > 1;
  if (multi) CE_CUDA_TRY(cudaMemsetAsync(owner->queue, 0, sizeof(unsigned), s));
  if (amem) {   // the solve: f16 operands, one event, a static schedule of equal items
    if (kind != KIND_F16 || multi) return fail(owner, CE_ERR_ARG, "memory-operand launch: one f16 event");
    const int st = launch_tc<0, KIND_F16, false, false, false, true>(a, smem, s);
    if (st) return st;
    CE_CUDA_TRY(cudaGetLastError());
    return CE_OK;
  }
  const int st = kind == KIND_F16    ? launch_tc_kind<KIND_F16>(a, smem, s, ad.on != 0, nu3, npw, multi)
                 : kind == KIND_BF16 ? launch_tc_kind<KIND_BF16>(a, smem, s, ad.on != 0, nu3, npw, multi)
                                     : launch_tc_kind<KIND_TF32>(a, smem, s, ad.on != 0, nu3, npw, multi);
  if (st) return st;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace

int correct_tc_prepare(ce_ctx* ctx, const float* B, int Rc, int Npad, cudaStream_t s) {
  if (ctx->prec != CE_PREC_BF16X3 && ctx->prec != CE_PREC_F16X3 && ctx->prec != CE_PREC_TF32X3)
    return fail(ctx, CE_ERR_ARG, "the tensor-core correction needs f16x3, bf16x3 or tf32x3");
  if (Rc < 1 || Rc > Npad || Npad > 128 || Npad % 16) return fail(ctx, CE_ERR_ARG, "tensor-core operand rows");
  const int kind = tc_kind(ctx);
  int st = ensure_bsplit(ctx, Npad);
  if (st) return st;
  const TcBuffers b = tc_buffers(ctx, Npad, tc_kind(ctx));
  const MaternF mf = matern_grid_units(ctx);
  const float absb = -mf.b;
  if (kind == KIND_F16) {
    CE_CUDA_TRY(cudaMemsetAsync(b.bmax, 0, sizeof(unsigned), s));
    absmax_kernel<<<152, 256, 0, s>>>(B, ctx->nobs_pad, Rc, ctx->nobs, mf.s2, b.bmax);
    ctx->launches += 1;
  }
  float4* sb4 = reinterpret_cast<float4*>(b.sites);
  if (kind == KIND_F16)
    launch_prep<KIND_F16>(B, ctx->nobs_pad, Rc, ctx->nobs, Npad, b.nchunks, mf.s2, ctx->obs, absb, b.bsplit, b.bblock, sb4, b.bmax, s);
  else if (kind == KIND_BF16)
    launch_prep<KIND_BF16>(B, ctx->nobs_pad, Rc, ctx->nobs, Npad, b.nchunks, mf.s2, ctx->obs, absb, b.bsplit, b.bblock, sb4, b.bmax, s);
  else
    launch_prep<KIND_TF32>(B, ctx->nobs_pad, Rc, ctx->nobs, Npad, b.nchunks, mf.s2, ctx->obs, absb, b.bsplit, b.bblock, sb4, b.bmax, s);
  ctx->launches += 1;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int correct_tc_batch(ce_ctx* owner, ce_ctx* const* ctxs, const int* Rs, float* const* ys, int count, int Npad,
                     cudaStream_t s) {
  if (count < 1) return CE_OK;
  const int kind = tc_kind(ctxs[0]);
  bool nu3 = false;
  for (int i = 0; i < count; ++i) {
    if (tc_kind(ctxs[i]) != kind) return fail(ctxs[0], CE_ERR_ARG, "batched correction: mixed operand kinds");
    if (make_aniso(ctxs[i]->aniso_ratio, ctxs[i]->aniso_angle).on)
      return fail(ctxs[0], CE_ERR_ARG, "batched correction: isotropic covariances only");
    nu3 = nu3 || ctxs[i]->nu == 1.5;
  }
  const Aniso iso = make_aniso(1.0, 0.0);
  for (int e0 = 0; e0 < count; e0 += kMaxEvents) {
    const int nev = count - e0 < kMaxEvents ? count - e0 : kMaxEvents;
    TcEvent ev[kMaxEvents];
    for (int e = 0; e < nev; ++e) ev[e] = tc_event(ctxs[e0 + e], Rs[e0 + e], Npad, ys[e0 + e]);
    const int st = tc_launch(owner, ev, nev, kind, Npad, nu3, iso, s);
    if (st) return st;
  }
  return CE_OK;
}

int launch_correct_tc(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  if (ctx->prec != CE_PREC_BF16X3 && ctx->prec != CE_PREC_F16X3 && ctx->prec != CE_PREC_TF32X3)
    return fail(ctx, CE_ERR_ARG, "unknown precision");
  const int kind = tc_kind(ctx);
  const Aniso ad = make_aniso(ctx->aniso_ratio, ctx->aniso_angle);
  for (int r0 = 0; r0 < R; r0 += 128) {
    const int Rc = R - r0 < 128 ? R - r0 : 128;
    const int Npad = (Rc + 15) / 16 * 16;
    int st = correct_tc_prepare(ctx, B + (size_t)r0 * ctx->nobs_pad, Rc, Npad, s);
    if (st) return st;
    TcEvent ev = tc_event(ctx, Rc, Npad, y + (size_t)r0 * ctx->m * ctx->m);
    st = tc_launch(ctx, &ev, 1, kind, Npad, ctx->nu == 1.5, ad, s);
    if (st) return st;
    ctx->launches += 1;
  }
  return CE_OK;
}


bool solve_on_tensor_cores(const ce_ctx* ctx) { return ctx->solve_form == CE_SOLVE_TENSOR; }

namespace {

// The f16 blocks of A^-1 and, after them, the bits of max |A^-1|: built once per
// set-up of the prediction matrix, on the caller's stream.
int ensure_ainv_tc(ce_ctx* ctx, cudaStream_t s, int* launches) {
  if (ctx->ainv_blk) return CE_OK;
  const int np_ = ctx->nobs_pad, mtiles = np_ / TM, nchunks = np_ / 64;
  const size_t blk = (size_t)mtiles * nchunks * 32768u;
  ctx->ainv_blk = (uint8_t*)dalloc(ctx, blk + 256);
  if (!ctx->ainv_blk) return fail(ctx, CE_ERR_OOM, "tensor-core operand of the solve");
  unsigned* amax = reinterpret_cast<unsigned*>(ctx->ainv_blk + blk);
  CE_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned), s));
  absmax_kernel<<<4 * 152, 256, 0, s>>>(ctx->Ainv_hi, np_, ctx->nobs, ctx->nobs, 1.0f, amax);
  const long long tot = (long long)mtiles * TM * nchunks * 64;
  prep_a_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->Ainv_hi, ctx->Ainv_lo, np_, ctx->nobs, mtiles, nchunks,
                                                               amax, ctx->ainv_blk);
  *launches += 2;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace

int launch_solve_tc(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s, int* launches) {
  int st = ensure_ainv_tc(ctx, s, launches);
  if (st) return st;
  const int n = ctx->nobs, np_ = ctx->nobs_pad, mtiles = np_ / TM, nchunks = np_ / 64;
  const unsigned* amax = reinterpret_cast<const unsigned*>(ctx->ainv_blk + (size_t)mtiles * nchunks * 32768u);
  // K parts: about three work items per SM, at least 8 chunks (one accumulation unit)
  // each, and no empty part
  int nsm = 0, dev = 0;
  CE_CUDA_TRY(cudaGetDevice(&dev));
  CE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int kparts = (3 * nsm + mtiles - 1) / mtiles;
  const int per_unit = kDrainSites / 64;
  kparts = std::max(1, std::min(kparts, nchunks / per_unit));
  const int cpp = (nchunks + kparts - 1) / kparts;
  kparts = (nchunks + cpp - 1) / cpp;
  const Aniso iso = make_aniso(1.0, 0.0);
  for (int r0 = 0; r0 < R; r0 += 128) {
    const int Rc = R - r0 < 128 ? R - r0 : 128;
    const int Npad = (Rc + 15) / 16 * 16;
    if ((st = ensure_bsplit(ctx, Npad))) return st;
    const size_t part_bytes = (size_t)kparts * Rc * np_ * sizeof(float);
    if (ctx->solve_part_bytes < part_bytes) {
      dfree(ctx, ctx->solve_part);
      ctx->solve_part = (float*)dalloc(ctx, part_bytes);
      ctx->solve_part_bytes = ctx->solve_part ? part_bytes : 0;
      if (!ctx->solve_part) return fail(ctx, CE_ERR_OOM, "partial products of the solve");
    }
    // E's rows r0 .. r0 + Rc as the B operand: f16 hi/lo with its own power-of-two scale
    const TcBuffers b = tc_buffers(ctx, Npad, KIND_F16);
    const float* Ec = E + (size_t)r0 * n;
    CE_CUDA_TRY(cudaMemsetAsync(b.bmax, 0, sizeof(unsigned), s));
    absmax_kernel<<<152, 256, 0, s>>>(Ec, n, Rc, n, 1.0f, b.bmax);
    launch_prep<KIND_F16>(Ec, n, Rc, n, Npad, b.nchunks, 1.0f, ctx->obs, 1.0f, b.bsplit, b.bblock,
                          reinterpret_cast<float4*>(b.sites), b.bmax, s);
    TcEvent ev;
    ev.y = ctx->solve_part;
    ev.bsplit = b.bsplit;
    ev.sites = b.sites;
    ev.bmax = b.bmax;
    ev.ablk = ctx->ainv_blk;
    ev.amax = amax;
    ev.ystride = np_;
    ev.pstride = (long long)Rc * np_;
    ev.m = n;
    ev.R = Rc;
    ev.nchunks = nchunks;
    ev.tiles_per_row = mtiles;
    ev.nitems = mtiles * kparts;
    ev.kparts = kparts;
    ev.cpp = cpp;
    {   // units of at most kDrainSites sites, balanced over a part's chunks
      const int units = (cpp + per_unit - 1) / per_unit;
      ev.drain = (cpp + units - 1) / units;
    }
    ev.item0 = 0;
    ev.absb = 0.f;
    ev.c1 = 0.f;
    if ((st = tc_launch(ctx, &ev, 1, KIND_F16, Npad, false, iso, s, true))) return st;
    const long long tot = (long long)Rc * n;
    solve_join_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->solve_part, ev.pstride, kparts, Rc, n, np_,
                                                                     B + (size_t)r0 * ldb, ldb);
    *launches += 4;
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

int solve_condsim(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s, int* launches) {
  if (solve_on_tensor_cores(ctx)) return launch_solve_tc(ctx, E, R, B, ldb, s, launches);
  launch_solve(ctx, E, R, B, ldb, s);
  *launches += 2;
  return CE_OK;
}

}  // namespace ce
