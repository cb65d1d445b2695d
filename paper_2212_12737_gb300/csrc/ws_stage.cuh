// TMA-staged passes over an FP32 matrix stored column-major (the Nystrom factor L_k):
// the shared producer/consumer machinery (ring of column tiles, bounded mbarrier waits,
// packed FP32 double-float arithmetic).  Used by the Woodbury apply's passes and by the
// Schur sums of Algorithm 1.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace gdml {

// ---------------------------------------------------------------------------
// TMA-staged passes.  One producer thread keeps a ring of 16 KB column tiles of
// L in flight (cp.async.bulk.tensor, zero fill past n and k; an L2 evict-first
// hint where L is streamed once: the apply's passes, and the Schur sums once the
// columns no longer fit in L2); eight consumer warps do the double-float
// arithmetic out of shared memory.  The bytes in flight per SM then no longer
// depend on how many loads each warp holds in registers.
// The L u pass and the Schur sums cut the rows into chunks of RC = 128 NT rows
// (NT = 1 or 2, so every lane is busy); CTA b takes chunks b, b + grid, ... and
// streams all k columns of each.  A tile is RC rows x 32 / NT columns; warp w
// takes tile columns w CPW .. w CPW + CPW - 1 (CPW = 4 / NT) and lane l rows
// 4 l + 128 t + e (t < NT, e < 4): one float4 per column and t, 16 products per
// lane and tile.  The L^T r pass uses 256-row x 16-column tiles over larger row
// units (see its kernel).
//
// Sums are double-float with the low part accumulated lazily: each exact
// product enters the high word through TwoSum and its rounding errors go
// straight into the low word; the pair is renormalised (Fast2Sum) once per tile
// instead of once per product, so the low word gathers at most 4 terms in
// between.  The arithmetic runs on packed FP32 pairs (add/sub/mul/fma .f32x2):
// 11 instructions per two products instead of 14 per product.
constexpr int kWsWarps = 8;                      // consumer warps
constexpr int kWsThreads = 32 * (kWsWarps + 1);  // + one producer warp
constexpr int kWsTile = 16384;                   // bytes per tile (RC x 32/NT floats)
constexpr int kWsStages = 6;
constexpr int kWsAlign = 128;  // TMA destination alignment (no swizzle)
constexpr int kWsSmemT = kWsAlign + kWsStages * kWsTile + 3 * 256 * 16 + (2 * kWsStages + 2) * 8 + 16;
constexpr int kWsSmemN = kWsAlign + kWsStages * kWsTile + kWsWarps * 256 * 8 + (2 * kWsStages + 2) * 8 + 16;
static_assert(2 * kWsSmemT <= 227 * 1024 && 2 * kWsSmemN <= 227 * 1024, "two CTAs per SM");

namespace {

__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = tc::smem_u32(bar);
  const uint32_t limit = tc::g_wait_limit;
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void ws_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// 2D tile load that marks the lines evict-first in L2 (L is streamed once per pass; the
// k x k matrices of the apply's core should stay resident)
__device__ __forceinline__ void ws_tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

// Packed FP32 arithmetic (two independent lanes per instruction, round to nearest even):
// the double-float sums below run on row pairs (x, y) and (z, w) of each float4.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(*reinterpret_cast<const uint64_t*>(&a)),
      "l"(*reinterpret_cast<const uint64_t*>(&b)));
  return *reinterpret_cast<const float2*>(&d);
}

// (sh, sl) += a (bh + bl) on both lanes, low word not renormalised; nbh = -bh.  The
// product's rounding error comes exactly from one FMA, the high word's from TwoSum.
__device__ __forceinline__ void df2_add_prod_lazy(float2& sh, float2& sl, float2 a, float2 bh, float2 nbh,
                                                  float2 bl) {
  const float2 ph = f2mul(a, bh);
  const float2 pn = f2fma(a, nbh, ph);  // ph - a bh: minus the rounding error of ph, exact
  const float2 t = f2add(sh, ph);
  const float2 v = f2sub(t, sh);
  const float2 e = f2add(f2sub(sh, f2sub(t, v)), f2sub(ph, v));
  const float2 q = f2fma(a, bl, e);  // e + a bl
  sl = f2add(sl, f2sub(q, pn));
  sh = t;
}

// the same with bl = 0 (an FP32 multiplier)
__device__ __forceinline__ void df2_add_prod_lazy(float2& sh, float2& sl, float2 a, float2 bh, float2 nbh) {
  const float2 ph = f2mul(a, bh);
  const float2 pn = f2fma(a, nbh, ph);
  const float2 t = f2add(sh, ph);
  const float2 v = f2sub(t, sh);
  const float2 e = f2add(f2sub(sh, f2sub(t, v)), f2sub(ph, v));
  sl = f2add(sl, f2sub(e, pn));
  sh = t;
}

__device__ __forceinline__ void df2_renorm(float2& sh, float2& sl) {
  const float2 t = f2add(sh, sl);
  sl = f2sub(sl, f2sub(t, sh));
  sh = t;
}

__device__ __forceinline__ float2 lo_pair(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi_pair(const float4& v) { return make_float2(v.z, v.w); }

// Bounded barrier of the 256 consumer threads (the producer warp does not take part) on an
// mbarrier with 256 arrivals per phase; false (warp-uniform) on timeout or abort.
__device__ __forceinline__ bool ws_consumer_sync(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  ws_arrive(bar);
  bool ok = ws_wait(bar, parity);
  if (!ok) {
    atomicExch(err, tc::ERR_TIMEOUT_DONE);
    *abort_flag = 1;
  }
  ok = ok && !*abort_flag;
  return __all_sync(0xffffffffu, ok);
}

// Bounded wait of a whole consumer warp on a full slot; false (warp-uniform) on timeout or abort.
__device__ __forceinline__ bool ws_consume_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  bool ok = ws_wait(bar, parity);
  if (!ok) {
    atomicExch(err, tc::ERR_TIMEOUT_FULL);
    *abort_flag = 1;
  }
  ok = ok && !*abort_flag;
  return __all_sync(0xffffffffu, ok);
}

// ring position: slot and phase parity advance together
struct WsRing {
  uint32_t slot = 0, phase = 0;
  __device__ __forceinline__ void next() {
    if (++slot == kWsStages) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

// The producer: tile (chunk, s) = rows [chunk RC, chunk RC + RC) x columns [s COLS, s COLS + COLS).
// Returns the number of tiles issued.
template <int NT, bool EVICT_FIRST>
__device__ uint32_t ws_produce(const CUtensorMap* map, uint8_t* ring, uint64_t* full, uint64_t* empty,
                               volatile int* abort_flag, int64_t nch, int ntiles, int* err) {
  constexpr int RC = 128 * NT, COLS = 32 / NT;
  uint64_t policy;
  if (EVICT_FIRST)
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  else
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(policy));
  WsRing rp;
  uint32_t issued = 0;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x)
    for (int s = 0; s < ntiles; ++s, ++issued, rp.next()) {
      if (!ws_wait(&empty[rp.slot], rp.phase ^ 1u)) {
        atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
        *abort_flag = 1;
        return issued;
      }
      if (*abort_flag) return issued;
      tc::mbar_expect_tx(&full[rp.slot], kWsTile);
      ws_tma_load(ring + rp.slot * kWsTile, map, &full[rp.slot], (int)(ch * RC), s * COLS, policy);
    }
  return issued;
}

// After an abort: wait (bounded) until the last copy issued into each slot has landed, so
// that no TMA write is in flight when the CTA exits.
__device__ void ws_drain(uint64_t* full, uint32_t issued) {
  for (uint32_t s = 0; s < kWsStages && s < issued; ++s) {
    const uint32_t last = s + ((issued - 1 - s) / kWsStages) * kWsStages;
    (void)ws_wait(&full[s], (last / kWsStages) & 1u);
  }
}

__device__ __forceinline__ void ws_init(uint64_t* full, uint64_t* empty, uint64_t* cbar, volatile int* abort_flag) {
  for (int s = 0; s < kWsStages; ++s) {
    tc::mbar_init(&full[s], 1);
    tc::mbar_init(&empty[s], kWsWarps);
  }
  if (cbar) {
    tc::mbar_init(&cbar[0], 32 * kWsWarps);
    tc::mbar_init(&cbar[1], 32 * kWsWarps);
  }
  *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

}  // namespace

}  // namespace gdml
