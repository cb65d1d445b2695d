// tcgen05 / TMA GEMM building block for sm_103a (5th-generation tensor cores).
//
//   acc[m, n] = sum_k A[m, k] * B[n, k]      A: M x K, B: N x K, both K-major
//
// Operands are TF32 (stored as fp32) or BF16, staged by TMA (128-byte swizzle)
// into a multi-stage shared-memory ring; one elected thread issues
// tcgen05.mma (kind::tf32 or kind::f16) into an FP32 accumulator in TMEM;
// four epilogue warps read the accumulator back with tcgen05.ld and hand each
// row fragment to an epilogue functor.  No cluster multicast is used.
//
// Warp roles (192 threads): warp 0 TMA producer, warp 1 TMEM owner + MMA
// issuer, warps 2..5 epilogue (warp w reads TMEM lanes 32*(w%4) ...).
// Every mbarrier wait is bounded; on timeout the CTA records an error code in
// *err, skips the remaining work, and still releases its TMEM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gdml {
namespace tc {

constexpr int BM = 128;          // rows per tile (UMMA M)
constexpr int BK_BYTES = 128;    // one 128-byte swizzle span of K per stage
constexpr int NUM_THREADS = 192;
constexpr uint32_t kSpinLimit = 1u << 26;  // bounded waits (seconds, not forever)

// Polls of every bounded wait of this translation unit: kSpinLimit unless a test lowers it
// (gdml_test_set_wait_limit; 0 makes each wait give up at once, before any copy or MMA of the
// waiting role is issued).  Each translation unit holds its own copy.
static __constant__ uint32_t g_wait_limit = kSpinLimit;
static inline cudaError_t set_wait_limit_here(uint32_t polls) {
  return cudaMemcpyToSymbol(g_wait_limit, &polls, sizeof(polls));
}

enum : int { ERR_NONE = 0, ERR_TIMEOUT_FULL = 1, ERR_TIMEOUT_EMPTY = 2, ERR_TIMEOUT_DONE = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const uint32_t limit = g_wait_limit;
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// Wait with the fixed bound kSpinLimit whatever g_wait_limit says: for a thread that waits on
// its own MMAs before the CTA releases its tensor memory and exits.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms 1024 bytes apart (SBO), version 1 (sm_100 family).
__device__ __forceinline__ uint64_t make_sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)(16 >> 4) << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
  return d;
}

// Instruction descriptor for kind::tf32 (fmt 2) or kind::f16 with BF16 (fmt 1):
// FP32 accumulate, K-major A and B, M = 128, N = n.
__host__ __device__ constexpr uint32_t make_idesc(int ab_fmt, int n) {
  return (1u << 4)                      // D format: F32
         | ((uint32_t)ab_fmt << 7)      // A format
         | ((uint32_t)ab_fmt << 10)     // B format
         | ((uint32_t)(n >> 3) << 17)   // N >> 3
         | ((uint32_t)(BM >> 4) << 24); // M >> 4
}

template <bool BF16>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int BN, int STAGES>
struct Smem {
  static constexpr int A_BYTES = BM * BK_BYTES;
  static constexpr int B_BYTES = BN * BK_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

// Generic tile kernel.  grid: (ceil(N/BN), ceil(M/BM), ksplit).  Each CTA
// accumulates K blocks [kb_begin, kb_end) of its split and calls
//   epi(row, col0, vals[32], valid_cols, split)
// for every 32-column fragment of every row of its tile.
template <bool BF16, int BN, int STAGES, typename Epi>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                int num_kb, int kb_per_split, Epi epi, int* __restrict__ err) {
  using SM = Smem<BN, STAGES>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * SM::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int kb_begin = blockIdx.z * kb_per_split;
  const int kb_end = min(num_kb, kb_begin + kb_per_split);
  const int nk = kb_end - kb_begin;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // TMEM allocation (whole warp)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(BN < 32 ? 32 : BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // MMA thread: issued at least one MMA / a wait gave up.  A thread that gave up before
  // issuing anything commits nothing, so no asynchronous arrive outlives the CTA.
  bool mma_any = false, mma_failed = false;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(err, ERR_TIMEOUT_EMPTY);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* sa = smem + s * SM::STAGE_BYTES;
      uint8_t* sb = sa + SM::A_BYTES;
      mbar_expect_tx(&full[s], SM::STAGE_BYTES);
      const int kx = (kb_begin + i) * (BF16 ? 64 : 32);
      tma_load_2d(sa, &mapA, &full[s], kx, m0);
      tma_load_2d(sb, &mapB, &full[s], kx, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(BF16 ? 1 : 2, BN);
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        atomicExch(err, ERR_TIMEOUT_FULL);
        *abort_flag = 1;
        ok = false;
        break;
      }
      if (*abort_flag) {
        ok = false;
        break;
      }
      // the mbarrier's TMA completion orders the stage for the tensor core: no tcgen05 fence
      const uint32_t sa = smem_u32(smem + s * SM::STAGE_BYTES);
      const uint32_t sb = sa + SM::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK_BYTES / 32; ++kk) {  // 32 bytes of K per instruction
        mma_issue<BF16>(tmem, make_sw128_desc(sa + kk * 32), make_sw128_desc(sb + kk * 32), idesc,
                        (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_any = true;
      mma_commit(&empty[s]);  // stage reusable once these MMAs have read it
    }
    mma_failed = !ok;
    // arrives when every MMA issued above has completed
    if (mma_any || ok) mma_commit(done);
  } else if (warp >= 2) {
    // ---------------- epilogue
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    int go = 0;
    if (lane == 0) {
      const bool ok = mbar_wait(done, 0);
      if (!ok) {
        atomicExch(err, ERR_TIMEOUT_DONE);
        *abort_flag = 1;
      }
      go = ok && !*abort_flag;
    }
    go = __shfl_sync(0xffffffffu, go, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
    fence_after_sync();
    if (go) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
        if (nk <= 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        const int valid = min(32, N - (n0 + c0));
        if (row < M && valid > 0) epi(row, n0 + c0, v, valid, (int)blockIdx.z);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    // the accumulator must be idle before it is released (already true unless a wait timed out)
    if (lane == 0 && (mma_any || !mma_failed)) (void)mbar_wait_bounded(done, 0);
    __syncwarp();
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(BN < 32 ? 32 : BN)));
  }
}

}  // namespace tc
}  // namespace gdml
