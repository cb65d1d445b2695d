// Sliced-BF16 tensor-core matvec (see oz.cuh for the scheme).  Data layout in HBM:
//   <op>.slices  BF16 [7][Rp][Kp]   K-major, zero padded (A operands Rp % 128 == 0, B operands % 64,
//                                   Kp % 128 == 0)
//   <op>.e       int  [chunk][rows] power-of-two exponent of each 256-entry chunk of a row
//   Tp           float2 [D-chunks][M][M]    double-float partials of T = Xc W^T
//   Up           float2 [2 M-chunks][M][D]  double-float partials of U = A W + beta Xc
//   rs2          float2 [M-chunks][M]       partial row sums of beta
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "kernels.cuh"
#include "oz.cuh"
#include "tc.cuh"
#include "tc_gemm.cuh"

namespace gdml {

namespace {

using bf16 = __nv_bfloat16;

// matvec GEMM: warp 0 TMA (A), warp 1 MMA, warp 2 TMA (B) and every wait, warps 3.. epilogue
// (kEpiWarps: 4 per TMEM lane quarter, 16 of the tile's 64 columns each)
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (3 + kEpiWarps);
constexpr int kAStages = 6;
constexpr int kATile = oz::BM * 128;     // 16 KB: 128 rows x one 128-byte K span
constexpr int kBTile = oz::BN * 128;     // 8 KB
constexpr int kBGroup = oz::S * kBTile;  // all slices of one B k-block
constexpr int kSmemData = 2 * kBGroup + kAStages * kATile;
constexpr int kSmemTotal = kSmemData + 1024 + 256;
constexpr uint32_t kTmemCols = 512;
constexpr int kKbPerChunk = oz::KC / oz::KB;
constexpr int kWaiterWarp = 11;           // the accumulating GEMM's extra warp: mbarrier waits
constexpr int kThreadsAcc = 32 * 12;
constexpr int kStageLd = oz::BN + 1;  // padded row of the staged output tile (float2)
// matvec GEMM: k-blocks of 64 K entries (one 128-byte swizzle span per tile).  The B group of
// a k-block (7 slices, 56 KB) is double-buffered; the A slices stream through a 6-deep ring
// (a 7-deep ring, one whole k-block of look-ahead at 226.75 KB, measured no faster).
constexpr int kBGroupM = oz::S * kBTile;                               // 56 KB
constexpr int kBStagesM = 2;
constexpr int kAStagesM = 6;
constexpr int kSmemDataM = kBStagesM * kBGroupM + kAStagesM * kATile;  // 208 KB
constexpr int kExpStage = oz::BM + oz::BN;                             // a chunk's row and column exponents
constexpr int kSmemTotalM = kSmemDataM + 1024 + 256 + 2 * kExpStage * 4;
constexpr int kKbPerChunkM = oz::KC / oz::KB;                          // 4
constexpr int kEpiCols = oz::BN * 4 / kEpiWarps;                       // 16 columns per epilogue warp
constexpr int kTilesPerHandoff = 2;  // A tiles the waiter hands to the MMA warp per named-barrier meeting
constexpr int kLevelsPerMma = 4;     // slice pairs (adjacent levels) per MMA: N = 64 x 4 = 256 at most
static_assert(oz::BM * kStageLd * 8 <= kSmemDataM, "output staging fits the operand buffers");
static_assert(kSmemTotalM <= 227 * 1024, "shared memory per CTA");
static_assert(kEpiCols % 8 == 0, "epilogue columns in groups of 8");
static_assert(oz::BM * kStageLd * 8 <= kSmemData, "output staging fits the operand buffers");
static_assert(oz::S * oz::BN <= (int)kTmemCols, "one TMEM accumulator per level");
static_assert(kSmemTotal <= 227 * 1024, "shared memory per CTA");

// ------------------------------------------------------------ double-float helpers
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // needs |a| >= |b| or a == 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (h, l) += x
__device__ __forceinline__ void df_add_f(float& h, float& l, float x) {
  float s, e;
  two_sum(h, x, s, e);
  e = __fadd_rn(e, l);
  fast_two_sum(s, e, h, l);
}
// (h, l) += (bh, bl)
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  fast_two_sum(s, e, h, l);
}
// (h, l) = (ah, al) * (bh, bl)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  fast_two_sum(p, e, h, l);
}
__device__ __forceinline__ float2 split_d(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}
// 2^k for -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// x * 2^e, exact unless the result leaves the FP32 range
__device__ __forceinline__ float scale2(float x, int e) {
  while (e > 127) {
    x *= pow2f(127);
    e -= 127;
  }
  while (e < -126) {
    x *= pow2f(-126);
    e += 126;
  }
  return x * pow2f(e);
}

// Slices of one entry (hi + lo) of a chunk whose magnitudes are all below 2^ex:
// s_i = rint(y), y <- (y - s_i) * 2^7, starting from y = x 2^(7 - ex).  All
// steps are exact; |s_1| <= 128 and |s_i| <= 64 for i > 1.  (y_h, y_l) stays normalised
// (|y_l| <= ulp(y_h) / 2), and y_h - s_i is exact and either 0 or at least ulp(y_h), so
// the exact sum (y_h - s_i) + y_l comes from Fast2Sum (its operand order holds or the
// first operand is 0).
__device__ __forceinline__ void slice_write(float2 xs, int ex, bf16* __restrict__ sl, int64_t row, int64_t k,
                                            int64_t Rp, int64_t Kp) {
  if (k >= Kp) return;
  float yh = scale2(xs.x, oz::BITS - ex), yl = scale2(xs.y, oz::BITS - ex);
  const float up = (float)(1 << oz::BITS);
#pragma unroll
  for (int i = 0; i < oz::S; ++i) {
    const float s = rintf(yh);
    sl[((int64_t)i * Rp + row) * Kp + k] = __float2bfloat16_rn(s);
    float h, l;
    fast_two_sum(__fsub_rn(yh, s), yl, h, l);
    yh = __fmul_rn(h, up);
    yl = __fmul_rn(l, up);
  }
}

// 16 columns of one TMEM lane quarter (32x32b.x16), without waiting for completion
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 8 columns of one TMEM lane quarter (32x32b.x8), without waiting for completion
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// packed FP32 pairs (two independent lanes per instruction, round to nearest even)
__device__ __forceinline__ float2 pf_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pf_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pf_sub(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(*reinterpret_cast<const uint64_t*>(&a)),
      "l"(*reinterpret_cast<const uint64_t*>(&b)));
  return *reinterpret_cast<const float2*>(&d);
}
// TwoSum on both lanes: s + e = a + b exactly
__device__ __forceinline__ void pf_two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = pf_add(a, b);
  const float2 bb = pf_sub(s, a);
  e = pf_add(pf_sub(a, pf_sub(s, bb)), pf_sub(b, bb));
}

// zeros into 16 columns of one TMEM lane quarter (32x32b.x16), then wait for the stores
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1};\n tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(z)
      : "memory");
}

// largest |x| of the CTA (256 threads), and the exponent ex with every |x| < 2^ex
__device__ __forceinline__ int chunk_exponent(float m, float* red) {
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  int ex = 0;
  if (m > 0.f) (void)frexpf(m, &ex);
  return ex;
}

// ------------------------------------------------------------ slicing kernels
// One CTA per (row, 256-entry chunk) of X (rows x K, row stride ldx).  Optionally
// also converts t[row] into a double-float pair (first chunk only).
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(const double* __restrict__ X, int64_t ldx, int64_t K,
                                                            int64_t rows, int64_t Rp, int64_t Kp,
                                                            bf16* __restrict__ sl, int* __restrict__ e,
                                                            const double* __restrict__ t, float2* __restrict__ t2) {
  __shared__ float red[8];
  const int64_t row = blockIdx.x, q = blockIdx.y;
  const int64_t k = q * oz::KC + threadIdx.x;
  const float2 xs = split_d(k < K ? X[row * ldx + k] : 0.0);
  const int ex = chunk_exponent(fabsf(xs.x), red);
  if (threadIdx.x == 0) {
    e[q * rows + row] = ex;
    if (t2 && q == 0) t2[row] = split_d(t[row]);
  }
  slice_write(xs, ex, sl, row, k, Rp, Kp);
}

// Same slicing for FP32 input rows (the FP32-stored Nystrom factor): hi = x, lo = 0.
__global__ void __launch_bounds__(256) oz_slice_rows_f32_kernel(const float* __restrict__ X, int64_t ldx, int64_t K,
                                                                int64_t rows, int64_t Rp, int64_t Kp,
                                                                bf16* __restrict__ sl, int* __restrict__ e) {
  __shared__ float red[8];
  const int64_t row = blockIdx.x, q = blockIdx.y;
  const int64_t k = q * oz::KC + threadIdx.x;
  const float x = k < K ? X[row * ldx + k] : 0.f;
  const int ex = chunk_exponent(fabsf(x), red);
  if (threadIdx.x == 0) e[q * rows + row] = ex;
  slice_write(make_float2(x, 0.f), ex, sl, row, k, Rp, Kp);
}

// an entry as a float pair (hi, lo) with hi + lo = x (FP64: rounded to 48 bits)
__device__ __forceinline__ float2 as_pair(double x) { return split_d(x); }
__device__ __forceinline__ float2 as_pair(float2 x) { return x; }

// Slicing of a COLUMN-major source: operand row r (r < rows) is row r0 + r of the n x K
// matrix whose column j starts at src + j ld, i.e. entry (r, j) = src[j ld + r0 + r].  One
// CTA per RB rows (16, or 4 when 16 would leave most SMs idle) and one 256-entry chunk:
// coalesced reads down the columns into a shared tile, a per-row exponent, then slice rows
// written along K (coalesced).
template <typename T, int RB = 16>
__global__ void __launch_bounds__(256) oz_slice_cols_kernel(const T* __restrict__ src, int64_t ld, int64_t r0,
                                                            int64_t rows, int64_t K, int64_t Rp, int64_t Kp,
                                                            bf16* __restrict__ sl, int* __restrict__ e) {
  static_assert(RB <= 16 && 256 % RB == 0, "rows per CTA");
  __shared__ float2 tile[oz::KC][RB + 1];
  __shared__ int ex_s[RB];
  const int64_t rb = (int64_t)blockIdx.x * RB, q = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {  // load: RB threads per column read RB consecutive rows
    const int r = tid % RB;
#pragma unroll 4
    for (int jj = tid / RB; jj < oz::KC; jj += 256 / RB) {
      const int64_t j = q * oz::KC + jj;
      const int64_t row = rb + r;
      float2 x = make_float2(0.f, 0.f);
      if (j < K && row < rows) x = as_pair(src[j * ld + r0 + row]);
      tile[jj][r] = x;
    }
  }
  __syncthreads();
  {  // exponent of each row: warp w takes rows 2w and 2w + 1, 16 lanes per row
    const int r = 2 * warp + (lane >> 4);
    float m = 0.f;
    if (r < RB)
      for (int jj = lane & 15; jj < oz::KC; jj += 16) m = fmaxf(m, fabsf(tile[jj][r].x));
    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((lane & 15) == 0 && r < RB) {
      int ex = 0;
      if (m > 0.f) (void)frexpf(m, &ex);
      ex_s[r] = ex;
      if (rb + r < rows) e[q * rows + rb + r] = ex;
    }
  }
  __syncthreads();
  for (int r = 0; r < RB; ++r) {
    if (rb + r >= rows) break;
    slice_write(tile[tid][r], ex_s[r], sl, rb + r, q * oz::KC + tid, Rp, Kp);
  }
}

// sum of the square-sum partials of each row, in a fixed slot order
__global__ void oz_rowsq_reduce_kernel(const double* __restrict__ sq, int slots, int64_t n, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = 0; k < slots; ++k) s += sq[(int64_t)k * n + i];
  out[i] = s;
}

// (h, l) = (ah, al) - (bh, bl)
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, -bh, s, e);
  e = __fadd_rn(e, __fsub_rn(al, bl));
  fast_two_sum(s, e, h, l);
}

// Sum of (h, l) over the 256 threads of the CTA in double-float, in a fixed order (valid in
// thread 0); red2 holds 8 pairs.
__device__ __forceinline__ void cta_df_sum(float& h, float& l, float2* red2) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
  if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = make_float2(h, l);
  __syncthreads();
  if (threadIdx.x == 0) {
    h = red2[0].x;
    l = red2[0].y;
    for (int w = 1; w < 8; ++w) df_add(h, l, red2[w].x, red2[w].y);
  }
}

// The projection W_a = J_a v_a, t_a = xc_a . w_a (the matvec's first step, Sec. 2.1) in
// double-float arithmetic, fused with the slicing of row a of W into GEMM 1's B operand
// (rows of up to kProjChunks 256-entry chunks).  GB300's FP64 pipe runs at ~1/64 of the FP32
// rate, so the FP64 form of this kernel was FP64-pipe bound; here every operation is an
// FP32 error-free transformation (TwoSum, FMA-based TwoProduct) on float pairs, ~2^-48
// relative, below the slicing's own 2^-43 per chunk.  G2, Xc2: the Jacobian factors and the
// centred descriptors as float pairs; v is split once per geometry in shared memory.  One
// CTA of 256 threads per geometry, every load of the row issued before the first chunk;
// per chunk, w as a float pair (also stored, Wf, for GEMM 2's transposed operand), its
// exponent (a CTA reduction of the high parts) and its slices.
constexpr int kProjChunks = 4;
__global__ void __launch_bounds__(256) oz_proj_slice_df_kernel(const float2* __restrict__ G2,
                                                               const float2* __restrict__ Xc2,
                                                               const double* __restrict__ v, int64_t M, int N, int D,
                                                               int nchunks, float2* __restrict__ Wf,
                                                               double* __restrict__ t, float2* __restrict__ t2,
                                                               int64_t Rp, int64_t Kp, bf16* __restrict__ sl,
                                                               int* __restrict__ e) {
  extern __shared__ float2 sv2[];  // 3N
  __shared__ float red[8];
  __shared__ float2 red2[8];
  const int64_t a = blockIdx.x;
  const int tid = threadIdx.x;
  const int B = 3 * N;
  const float2* Ga = G2 + a * D * 3;
  float2 g[kProjChunks][3], xc[kProjChunks];
#pragma unroll
  for (int q = 0; q < kProjChunks; ++q) {
    const int p = q * oz::KC + tid;
    const bool in = q < nchunks && p < D;
    const float2 z = make_float2(0.f, 0.f);
    g[q][0] = in ? Ga[3 * p] : z;
    g[q][1] = in ? Ga[3 * p + 1] : z;
    g[q][2] = in ? Ga[3 * p + 2] : z;
    xc[q] = in ? Xc2[a * D + p] : z;
  }
  for (int l = tid; l < B; l += blockDim.x) sv2[l] = split_d(v[a * B + l]);
  __syncthreads();
  float th = 0.f, tl = 0.f;
#pragma unroll
  for (int q = 0; q < kProjChunks; ++q) {
    if (q >= nchunks) break;
    const int p = q * oz::KC + tid;
    float wh = 0.f, wl = 0.f;
    if (p < D) {
      int i, j;
      pair_of(p, i, j);
#pragma unroll
      for (int c = 0; c < 3; ++c) {  // w -= g_c (v_ic - v_jc)
        const float2 vi = sv2[3 * i + c], vj = sv2[3 * j + c];
        float dh, dl, ph, pl;
        df_sub(vi.x, vi.y, vj.x, vj.y, dh, dl);
        df_mul(g[q][c].x, g[q][c].y, dh, dl, ph, pl);
        df_add(wh, wl, -ph, -pl);
      }
      Wf[a * D + p] = make_float2(wh, wl);
      float ph, pl;
      df_mul(xc[q].x, xc[q].y, wh, wl, ph, pl);
      df_add(th, tl, ph, pl);
    }
    const int ex = chunk_exponent(fabsf(wh), red);  // contains a __syncthreads
    if (tid == 0) e[q * M + a] = ex;
    slice_write(make_float2(wh, wl), ex, sl, a, p, Rp, Kp);
    __syncthreads();  // red is reused by the next chunk's reduction
  }
  cta_df_sum(th, tl, red2);
  if (tid == 0) {
    t[a] = (double)th + (double)tl;
    t2[a] = make_float2(th, tl);
  }
}

// XT (cols x rows) = X^T, X rows x cols with row stride ldx (32 x 32 tiles)
__global__ void oz_transpose_kernel(const double* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                    double* __restrict__ XT) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t r = r0 + yy, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[yy][threadIdx.x] = X[r * ldx + c];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t c = c0 + yy, r = r0 + threadIdx.x;
    if (r < rows && c < cols) XT[c * rows + r] = tile[threadIdx.x][yy];
  }
}

__global__ void oz_s2_kernel(const double* __restrict__ S, int64_t count, double c2, float2* __restrict__ S2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) S2[i] = split_d(c2 * S[i]);
}

// ------------------------------------------------------------ sliced GEMM
// Bounded wait without back-off, for the producer and MMA threads on the
// critical path (try_wait already suspends in hardware for a short while).
__device__ __forceinline__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity) {
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


// Named barrier 2 between the MMA warp and the waiter warp (64 threads), with the OR of
// the participants' flags: the MMA warp learns of a failed wait without reading shared memory.
__device__ __forceinline__ bool handoff(bool failed) {
  uint32_t any;
  asm volatile(
      "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.or.pred pout, 2, 64, pin;\n"
      " selp.u32 %0, 1, 0, pout;\n}\n"
      : "=r"(any)
      : "r"(failed ? 1u : 0u)
      : "memory");
  return any != 0;
}

// grid (ceil(N/64), ceil(M/128), ceil(chunks / G)).  CTA z accumulates the G K-chunks
// z G .. z G + G - 1, each 4 k-blocks of 64 K entries.
//  * Warp 0 loads the 7 A slice tiles of each k-block (16 KB each) into a 6-deep ring, in the
//    order 6, 5, ..., 0.
//  * Warp 2 loads the B group of each k-block (its 7 slices, 56 KB) into one of two buffers,
//    the next k-block's group while the current one is multiplied, and does every mbarrier
//    wait of the MMA side: it hands each A tile to warp 1 at named barrier 2 (a wait or any
//    shared-memory read in the MMA-issuing thread stalls the tensor pipe).
//  * Warp 1 multiplies A slice i with B slices j = 0..6-i (per K step of 16) into TMEM
//    accumulator i + j ("level").  Up to four consecutive pairs (i, j .. j + 3) go into one
//    MMA of N = 64 .. 256: 10 MMAs per K step instead of 28.  The CTA's first k-block
//    overwrites level i with its pair (i, 0), the first to reach that level in the order
//    6, 5, ..., 0 (14 MMAs per K step there, where pair (i, 0) stays alone); every later
//    chunk accumulates from its first MMA into levels the epilogue has zeroed.  Fewer, wider
//    MMAs measured faster at every step (28 -> 16 -> 10 per K step): the issuing thread's
//    progress, not a bandwidth, paces the pipeline.
//  * The epilogue warps drain a finished chunk level by level, 6 down to 0 (levels 6..4 summed
//    in FP32, 3..0 added in double-float, then scaled by 2^(eA + eB) into running
//    double-float sums held in registers), writing zeros into each level after reading it and
//    releasing it at once (tfree[L]).  A slice i of the next chunk needs levels i..6 only, so
//    its MMAs start while the drain is still on the lower levels.  After the last chunk they
//    store the group's double-float partial once.
// NLEV (1..7) keeps the levels below NLEV only (slices 0..NLEV-1, pairs i + j < NLEV): a cheaper,
// less accurate product for an inner solve; NLEV = 7 is the full product.  A compile-time count
// lets the tile loop unroll, so the MMA-issuing thread runs straight-line code (with a run-time
// count the MMA issue slowed by ~45 %).
template <int NLEV>
__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int Ap,
                   int Bp, int M, int N, int num_kb, int chunks_per_cta, const int* __restrict__ eA,
                   const int* __restrict__ eB, float2* __restrict__ out, int64_t ldo, int64_t split_stride,
                   int* __restrict__ err, const __grid_constant__ CUtensorMap mapA2,
                   const __grid_constant__ CUtensorMap mapB2, int Ap2, int Bp2, const int* __restrict__ eA2,
                   const int* __restrict__ eB2, int kb_split) {
  constexpr int nlev = NLEV;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sB = smem;                           // [2] B groups
  uint8_t* sA = smem + kBStagesM * kBGroupM;    // [kAStagesM] A tiles
  uint64_t* bfull = reinterpret_cast<uint64_t*>(smem + kSmemDataM);  // [2]
  uint64_t* bempty = bfull + kBStagesM;                               // [2]
  uint64_t* afull = bempty + kBStagesM;                               // [kAStagesM]
  uint64_t* aempty = afull + kAStagesM;                               // [kAStagesM]
  uint64_t* cdone = aempty + kAStagesM;  // the MMAs of a chunk have completed
  uint64_t* tfree = cdone + 1;           // [7] the epilogue has read level L of a chunk
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + oz::S);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* sexp = reinterpret_cast<int*>(smem + kSmemDataM + 256);  // [2][rows 128 | columns 64] exponents
  float2* stage = reinterpret_cast<float2*>(smem);  // output tile, reuses the operand buffers after the MMAs

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * oz::BN, m0 = blockIdx.y * oz::BM;
  const int q_begin = blockIdx.z * chunks_per_cta;
  const int kb_begin = q_begin * kKbPerChunkM;
  const int kb_end = min(num_kb, kb_begin + chunks_per_cta * kKbPerChunkM);
  const int nk = kb_end - kb_begin;
  const int nq = (nk + kKbPerChunkM - 1) / kKbPerChunkM;  // chunks of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < kBStagesM; ++s) {
      tc::mbar_init(&bfull[s], 1);
      tc::mbar_init(&bempty[s], 1);
    }
    for (int s = 0; s < kAStagesM; ++s) {
      tc::mbar_init(&afull[s], 1);
      tc::mbar_init(&aempty[s], 1);
    }
    tc::mbar_init(cdone, 1);
    for (int L = 0; L < oz::S; ++L) tc::mbar_init(&tfree[L], kEpiWarps);  // one arrival per epilogue warp
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // MMA thread: issued at least one MMA / learned of a failed wait.  A thread that failed
  // before issuing anything commits nothing, so no asynchronous arrive outlives the CTA.
  bool mma_any = false, mma_failed = false;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer, A slices (order 6, 5, ..., 0 within each k-block)
    int a_issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      // k-blocks from kb_split on belong to the second K segment (its own operands)
      const int gk = kb_begin + kb;
      const bool seg2 = gk >= kb_split;
      const CUtensorMap* mA = seg2 ? &mapA2 : &mapA;
      const int kx = (seg2 ? gk - kb_split : gk) * oz::KB;
      const int ap = seg2 ? Ap2 : Ap;
      bool ok = true;
      for (int pos = 0; pos < nlev; ++pos) {
        const int ai = kb * nlev + pos;
        const int s = ai % kAStagesM;
        const uint32_t ph = (uint32_t)(ai / kAStagesM) & 1u;
        if (!mbar_wait_spin(&aempty[s], ph ^ 1u)) {
          atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (*abort_flag) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(&afull[s], kATile);
        tc::tma_load_2d(sA + s * kATile, mA, &afull[s], kx, (nlev - 1 - pos) * ap + m0);
        a_issued = ai + 1;
      }
      if (!ok) break;
    }
    // no copy may outlive the CTA: after a failure nobody waits for the last tiles issued
    // (earlier ones were consumed before their slot was refilled); bounded waits
    for (int ai = max(0, a_issued - kAStagesM); ai < a_issued; ++ai)
      (void)tc::mbar_wait_bounded(&afull[ai % kAStagesM], (uint32_t)(ai / kAStagesM) & 1u);
  } else if (warp == 2) {
    // ---------------- B producer (lane 0) and waiter (whole warp).  The group of k-block kb + 1
    // goes into the buffer of k-block kb - 1 once that one's MMAs have completed (checked after
    // the second A hand-off of k-block kb, when they normally have).  Before the first k-block
    // of chunk q > 0, A slice i also waits for the epilogue's release of level i of chunk q - 1.
    // The warp arrives at named barrier 2 exactly nk * 7 times whatever happens, and a failed
    // wait travels in the barrier's OR-reduction.
    bool failed = false;
    int b_issued = 0, b_waited = 0;  // lane 0: B groups issued / whose arrival was waited for
    auto issue_b = [&](int kb) {  // lane 0; the buffer is known to be free
      b_issued = kb + 1;
      const int st2 = kb & 1;
      const int gk = kb_begin + kb;
      const bool seg2 = gk >= kb_split;
      const CUtensorMap* mB = seg2 ? &mapB2 : &mapB;
      const int kx = (seg2 ? gk - kb_split : gk) * oz::KB;
      const int bp = seg2 ? Bp2 : Bp;
      tc::mbar_expect_tx(&bfull[st2], nlev * kBTile);
      for (int j = 0; j < nlev; ++j)
        tc::tma_load_2d(sB + st2 * kBGroupM + j * kBTile, mB, &bfull[st2], kx, j * bp + n0);
    };
    {
      // the first wait comes before the first copy (a fresh buffer's previous phase counts
      // as complete), so a wait that gives up at once leaves nothing in flight
      int ok0 = 1;
      if (lane == 0 && nk > 0) {
        if (!mbar_wait_spin(&bempty[0], 1u)) {
          atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
          *abort_flag = 1;
          ok0 = 0;
        } else {
          issue_b(0);
          if (nk > 1) issue_b(1);
        }
      }
      failed = !__shfl_sync(0xffffffffu, ok0, 0);
    }
    for (int kb = 0; kb < nk; ++kb) {
      const int q = kb / kKbPerChunkM;
      const bool chunk_start = kb % kKbPerChunkM == 0 && q > 0;
      int okw = 1;
      if (lane == 0 && !failed) {
        if (!mbar_wait_spin(&bfull[kb & 1], (uint32_t)(kb >> 1) & 1u)) {
          atomicExch(err, tc::ERR_TIMEOUT_FULL);
          *abort_flag = 1;
          okw = 0;
        } else {
          b_waited = kb + 1;
          if (*abort_flag) okw = 0;
        }
      }
      failed = failed || !__shfl_sync(0xffffffffu, okw, 0);
#pragma unroll
      for (int p0 = 0; p0 < nlev; p0 += kTilesPerHandoff) {
        int oka = 1;
        if (lane == 0 && !failed) {
#pragma unroll
          for (int pos = p0; pos < min(p0 + kTilesPerHandoff, nlev); ++pos) {
            const int ai = kb * nlev + pos;
            const int s = ai % kAStagesM;
            const uint32_t ph = (uint32_t)(ai / kAStagesM) & 1u;
            if (!oka) break;
            if (chunk_start && !mbar_wait_spin(&tfree[nlev - 1 - pos], (uint32_t)(q - 1) & 1u)) {
              atomicExch(err, tc::ERR_TIMEOUT_DONE);
              *abort_flag = 1;
              oka = 0;
            } else if (!mbar_wait_spin(&afull[s], ph)) {
              atomicExch(err, tc::ERR_TIMEOUT_FULL);
              *abort_flag = 1;
              oka = 0;
            } else if (*abort_flag) {
              oka = 0;
            }
          }
        }
        failed = failed || !__shfl_sync(0xffffffffu, oka, 0);
        (void)handoff(failed);
        if (p0 + kTilesPerHandoff > min(1, nlev - 1) && p0 <= min(1, nlev - 1) && kb >= 1 && kb + 1 < nk) {
          int okb = 1;
          if (lane == 0 && !failed) {
            if (!mbar_wait_spin(&bempty[(kb - 1) & 1], (uint32_t)((kb - 1) >> 1) & 1u)) {
              atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
              *abort_flag = 1;
              okb = 0;
            } else if (*abort_flag) {
              okb = 0;
            } else {
              issue_b(kb + 1);
            }
          }
          failed = failed || !__shfl_sync(0xffffffffu, okb, 0);
        }
      }
    }
    // no copy may outlive the CTA: B groups issued but not waited for (after a failure)
    if (lane == 0)
      for (int kb = b_waited; kb < b_issued; ++kb)
        (void)tc::mbar_wait_bounded(&bfull[kb & 1], (uint32_t)(kb >> 1) & 1u);
  } else if (warp == 1) {
    // ---------------- MMA issuer (lane 0; the whole warp meets the waiter at barrier 2)
    constexpr uint32_t idesc = tc::make_idesc(1, oz::BN);
    constexpr uint32_t idesc2 = tc::make_idesc(1, 2 * oz::BN);  // 2, 3, 4 adjacent slices and levels
    constexpr uint32_t idesc3 = tc::make_idesc(1, 3 * oz::BN);
    constexpr uint32_t idesc4 = tc::make_idesc(1, 4 * oz::BN);
    const uint64_t adesc0 = tc::make_sw128_desc(tc::smem_u32(sA));
    const uint64_t bdesc0 = tc::make_sw128_desc(tc::smem_u32(sB));
    bool& failed = mma_failed;
    for (int kb = 0; kb < nk; ++kb) {
      // only the CTA's first k-block overwrites: the epilogue zeroes each level as it drains a
      // chunk, so the MMAs of every later chunk accumulate from the start
      const bool chunk_first = kb == 0;
#pragma unroll
      for (int p0 = 0; p0 < nlev; p0 += kTilesPerHandoff) {
        failed = handoff(false) || failed;
        tc::fence_after_sync();
#pragma unroll
        for (int pos = p0; pos < min(p0 + kTilesPerHandoff, nlev); ++pos) {
        const int i = nlev - 1 - pos;
        const int ai = kb * nlev + pos;
        const int s = ai % kAStagesM;
        if (lane == 0) {
          if (!failed) {
            // descriptors are linear in the start address (bits 0..13 = address / 16): a K
            // step of 32 bytes adds 2, B slice j of buffer b adds (b * group + j * tile) / 16
            const uint64_t ad = adesc0 + (uint64_t)(s * (kATile >> 4));
            const uint64_t bg = bdesc0 + (uint64_t)((kb & 1) * (kBGroupM >> 4));
            // descriptors of the four K steps: A + 2t, B + 2t
            auto mma4 = [&](uint32_t d, uint64_t bj, uint32_t id, uint32_t acc0) {
              tc::mma_issue<true>(d, ad, bj, id, acc0);
              tc::mma_issue<true>(d, ad + 2, bj + 2, id, 1u);
              tc::mma_issue<true>(d, ad + 4, bj + 4, id, 1u);
              tc::mma_issue<true>(d, ad + 6, bj + 6, id, 1u);
            };
            // Up to kLevelsPerMma consecutive pairs (i, j) .. (i, j + g - 1) go into one MMA of
            // N = 64 g: their levels i + j .. i + j + g - 1 are adjacent 64-column blocks of TMEM
            // and B slices j .. j + g - 1 adjacent 64-row tiles, so A is read once for all g.
            auto group = [&](int j, uint32_t acc0) {
              const int g = min(kLevelsPerMma, nlev - i - j);
              const uint32_t id = g == 1 ? idesc : g == 2 ? idesc2 : g == 3 ? idesc3 : idesc4;
              mma4(tmem + (uint32_t)((i + j) * oz::BN), bg + (uint64_t)(j * (kBTile >> 4)), id, acc0);
            };
            // the CTA's first k-block overwrites level i with pair (i, 0) alone; levels above
            // i were first written by an earlier slice of this k-block (the order is
            // 6, 5, ..., 0), so the pairs from j = 1 on accumulate
            const int j0 = chunk_first ? 1 : 0;
            if (chunk_first) mma4(tmem + (uint32_t)(i * oz::BN), bg, idesc, 0u);
#pragma unroll
            for (int m = 0; m * kLevelsPerMma < oz::S; ++m)
              if (i + j0 + m * kLevelsPerMma < nlev) group(j0 + m * kLevelsPerMma, 1u);
            mma_any = true;
          }
          // also after a failure (the A producer never starves), unless the failure came
          // before any MMA: then no asynchronous arrive may outlive the CTA
          if (mma_any || !failed) tc::mma_commit(&aempty[s]);
        }
        }
        __syncwarp();
      }
      if (lane == 0 && (mma_any || !failed)) {
        tc::mma_commit(&bempty[kb & 1]);
        if (kb % kKbPerChunkM == kKbPerChunkM - 1 || kb == nk - 1) tc::mma_commit(cdone);
      }
      __syncwarp();
    }
  } else if (warp >= 3) {
    // ---------------- epilogue: per chunk, level by level (6 .. 0), then scale and add
    const int quarter = warp & 3;
    const int cbase = ((warp - 3) >> 2) * kEpiCols;  // this warp's columns of the tile's 64
    const int et = threadIdx.x - 96;                 // 0 .. 32 kEpiWarps - 1
    constexpr int kEpiThreads = 32 * kEpiWarps;
    // a chunk's 128 row and 64 column exponents into shared memory, one coalesced load each,
    // a chunk ahead of its drain (the drain then reads no global memory)
    // chunks of the first K segment (a single segment may end on a half chunk: round up)
    const int nch1 = (kb_split + kKbPerChunkM - 1) / kKbPerChunkM;
    auto load_exps = [&](int q) {
      int* dst = sexp + (q & 1) * kExpStage;
      const int64_t zg = q_begin + q;
      const bool seg2 = zg >= nch1;
      const int* ea = seg2 ? eA2 : eA;
      const int* eb = seg2 ? eB2 : eB;
      const int64_t zq = seg2 ? zg - nch1 : zg;
      if (et < oz::BM)
        dst[et] = m0 + et < M ? ea[zq * M + m0 + et] : 0;
      else if (et < kExpStage)
        dst[et] = n0 + et - oz::BM < N ? eb[zq * N + n0 + et - oz::BM] : 0;
    };
    if (nq > 0) load_exps(0);
    float rh[kEpiCols], rl[kEpiCols], hh[kEpiCols], ll[kEpiCols];
#pragma unroll
    for (int t = 0; t < kEpiCols; ++t) rh[t] = rl[t] = 0.f;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cbase;
    auto release = [&](int L) {  // this warp has read level L of the chunk
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&tfree[L])) : "memory");
    };
    bool go = true;
    // every epilogue warp passes named barrier 1 exactly nq + 1 times, whatever fails: after a
    // failed wait a warp keeps looping without waiting or reading the accumulators
    for (int q = 0; q < nq; ++q) {
      // chunk q's exponents are visible, and chunk q - 1's buffer may be refilled
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (q + 1 < nq) load_exps(q + 1);
      if (!go) continue;
      int okw = 1;
      if (lane == 0) {
        okw = tc::mbar_wait(cdone, (uint32_t)q & 1u) ? 1 : 0;
        if (!okw) {
          atomicExch(err, tc::ERR_TIMEOUT_DONE);
          *abort_flag = 1;
        }
        if (*abort_flag) okw = 0;
      }
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) {
        go = false;
        continue;
      }
      tc::fence_after_sync();
      // levels 6..4 are scaled by 2^-56..2^-42 against the leading level's 2^-14, so a plain
      // FP32 sum of them errs by < 2^-48 of the leading level's range; levels 3..0 are added
      // by TwoSum with the errors gathered in the low word (renormalised once after level 0).
      // Packed FP32 pairs halve the drain's instructions: its warps share the issue slots of
      // the MMA warp while the next chunk starts
#pragma unroll
      for (int t = 0; t < kEpiCols; ++t) ll[t] = 0.f;
#pragma unroll
      for (int L = oz::S - 1; L >= 0; --L) {
        if (L >= nlev) continue;
        const float sc = pow2f(-oz::BITS * (L + 2));
        const float2 sc2 = make_float2(sc, sc);
#pragma unroll
        for (int c8 = 0; c8 < kEpiCols; c8 += 8) {
          uint32_t v[8];
          tmem_ld8_nowait(lane_base + (uint32_t)(L * oz::BN + c8), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int t = 0; t < 8; t += 2) {
            const float2 x = pf_mul(make_float2(__uint_as_float(v[t]), __uint_as_float(v[t + 1])), sc2);
            float2 h = make_float2(hh[c8 + t], hh[c8 + t + 1]);
            if (L == nlev - 1) {
              h = x;
            } else if (L >= 4) {
              h = pf_add(h, x);
            } else {
              float2 sum, e;
              pf_two_sum(h, x, sum, e);
              const float2 l = pf_add(make_float2(ll[c8 + t], ll[c8 + t + 1]), e);
              ll[c8 + t] = l.x;
              ll[c8 + t + 1] = l.y;
              h = sum;
            }
            hh[c8 + t] = h.x;
            hh[c8 + t + 1] = h.y;
          }
        }
        // level L starts from zero in the next chunk: its MMAs then all accumulate
        static_assert(kEpiCols == 16, "one 16-column zero store per level");
        tmem_zero16(lane_base + (uint32_t)(L * oz::BN));
        release(L);
      }
#pragma unroll
      for (int t = 0; t < kEpiCols; t += 2) {  // renormalise the level sum (TwoSum: any order)
        float2 sum, e;
        pf_two_sum(make_float2(hh[t], hh[t + 1]), make_float2(ll[t], ll[t + 1]), sum, e);
        hh[t] = sum.x;
        hh[t + 1] = sum.y;
        ll[t] = e.x;
        ll[t + 1] = e.y;
      }
      const int* ex = sexp + (q & 1) * kExpStage;
      const int ea = ex[quarter * 32 + lane];
#pragma unroll
      for (int t = 0; t < kEpiCols; ++t) {
        const int e2 = ea + ex[oz::BM + cbase + t];
        df_add(rh[t], rl[t], scale2(hh[t], e2), scale2(ll[t], e2));
      }
    }
    // stage the group's tile in the (now idle) operand buffers, then a coalesced write-out;
    // the epilogue warps sync among themselves (barrier 1)
    if (go) {
      float2* srow = stage + (quarter * 32 + lane) * kStageLd;
#pragma unroll
      for (int t = 0; t < kEpiCols; ++t) srow[cbase + t] = make_float2(rh[t], rl[t]);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
    if (go) {
      for (int idx = et; idx < oz::BM * oz::BN; idx += kEpiThreads) {
        const int rr = idx / oz::BN, cc = idx % oz::BN;
        const int grow = m0 + rr, gcol = n0 + cc;
        if (grow < M && gcol < N) out[blockIdx.z * split_stride + (int64_t)grow * ldo + gcol] = stage[rr * kStageLd + cc];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    // the epilogue has waited on every chunk's completion (or a wait gave up)
    if (lane == 0 && (mma_any || !mma_failed) && nq > 0) (void)tc::mbar_wait_bounded(cdone, (uint32_t)(nq - 1) & 1u);
    __syncwarp();
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

enum { ACC_ROWMAJOR = 0, ACC_COLMAJOR = 1, ACC_ROWSQ = 2 };
struct AccOut {  // what the accumulating GEMM stores (see oz_gemm_acc_kernel)
  int mode;
  int lower_only;
  int tri_b;
  double* C;
  float* C32;
  double* sq;
  int64_t ldc;
};

// Same sliced product accumulated over ALL K chunks inside the CTA, FP64 output:
//   C[m][n] = sum_chunks 2^(eA + eB) sum_levels acc_level 2^-7(level + 2)
// The MMA warp signals the end of each chunk on cdone; the 8 epilogue warps read the 7
// level accumulators of their 32 columns, add the scaled chunk value into a running
// double-float sum held in registers, and release the TMEM on tfree before the MMA
// warp starts the next chunk (whose first MMA per level overwrites).
//  o.lower_only: tiles wholly above the diagonal exit at once (symmetric products);
//  o.tri_b: row c of B is zero beyond column c (lower triangular B), so the CTA of B rows
//    [n0, n0 + 64) stops after K entry n0 + 63;
//  o.mode: ACC_ROWMAJOR  C[m][n] at C[m ldc + n];
//          ACC_COLMAJOR  C[m][n] at C[n ldc + m] (and as FP32 at C32[n ldc + m] if C32);
//          ACC_ROWSQ     sq[(2 blockIdx.x + half) ldc + m] = sum over the half tile's 32
//                        columns n of C[m][n]^2 (no C is stored).
__global__ void __launch_bounds__(kThreadsAcc, 1)
    oz_gemm_acc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int Ap,
                       int Bp, int M, int N, int num_kb_all, const int* __restrict__ eA, const int* __restrict__ eB,
                       const AccOut o, int* __restrict__ err) {
  const int n0 = blockIdx.x * oz::BN, m0 = blockIdx.y * oz::BM;
  if (o.lower_only && n0 >= m0 + oz::BM) return;
  const int num_kb = o.tri_b ? min(num_kb_all, (n0 + oz::BN + oz::KB - 1) / oz::KB) : num_kb_all;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sB = smem;
  uint8_t* sA = smem + 2 * kBGroup;
  uint64_t* bfull = reinterpret_cast<uint64_t*>(smem + kSmemData);
  uint64_t* bempty = bfull + 2;
  uint64_t* afull = bempty + 2;
  uint64_t* aempty = afull + kAStages;
  uint64_t* cdone = aempty + kAStages;
  uint64_t* tfree = cdone + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (num_kb + kKbPerChunk - 1) / kKbPerChunk;

  if (threadIdx.x == 0) {
    for (int g = 0; g < 2; ++g) {
      tc::mbar_init(&bfull[g], 1);
      tc::mbar_init(&bempty[g], 1);
    }
    for (int s = 0; s < kAStages; ++s) {
      tc::mbar_init(&afull[s], 1);
      tc::mbar_init(&aempty[s], 1);
    }
    tc::mbar_init(cdone, 1);
    tc::mbar_init(tfree, 8);  // one arrival per epilogue warp
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // MMA thread: issued at least one MMA / learned of a failed wait.  A thread that failed
  // before issuing anything commits nothing, so no asynchronous arrive outlives the CTA.
  bool mma_any = false, mma_failed = false;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer, A slices (all k-blocks)
    for (int kb = 0; kb < num_kb; ++kb) {
      bool ok = true;
      for (int i = 0; i < oz::S; ++i) {
        const int ai = kb * oz::S + i;
        const int s = ai % kAStages;
        const uint32_t ph = (uint32_t)(ai / kAStages) & 1u;
        if (!mbar_wait_spin(&aempty[s], ph ^ 1u)) {
          atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (*abort_flag) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(&afull[s], kATile);
        tc::tma_load_2d(sA + s * kATile, &mapA, &afull[s], kb * oz::KB, i * Ap + m0);
      }
      if (!ok) break;
    }
  } else if (warp == 2 && lane == 0) {
    // ---------------- TMA producer, B slice groups
    for (int kb = 0; kb < num_kb; ++kb) {
      const int g = kb & 1;
      const uint32_t gph = (uint32_t)(kb >> 1) & 1u;
      if (!mbar_wait_spin(&bempty[g], gph ^ 1u)) {
        atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      tc::mbar_expect_tx(&bfull[g], kBGroup);
      for (int j = 0; j < oz::S; ++j)
        tc::tma_load_2d(sB + (g * oz::S + j) * kBTile, &mapB, &bfull[g], kb * oz::KB, j * Bp + n0);
    }
  } else if (warp == kWaiterWarp) {
    // ---------------- waiter: every mbarrier wait on behalf of the MMA warp (see
    // oz_gemm_kernel), one handoff per A tile at named barrier 2, num_kb * 7 in all
    bool failed = false;
    for (int kb = 0; kb < num_kb; ++kb) {
      const int q = kb / kKbPerChunk;
      const bool chunk_start = (kb % kKbPerChunk) == 0;
      const int g = kb & 1;
      const uint32_t gph = (uint32_t)(kb >> 1) & 1u;
      int okw = 1;
      if (lane == 0 && !failed) {
        if (chunk_start && q > 0 && !mbar_wait_spin(tfree, (uint32_t)(q - 1) & 1u)) {  // chunk q-1 read out
          atomicExch(err, tc::ERR_TIMEOUT_DONE);
          *abort_flag = 1;
          okw = 0;
        } else if (!mbar_wait_spin(&bfull[g], gph)) {
          atomicExch(err, tc::ERR_TIMEOUT_FULL);
          *abort_flag = 1;
          okw = 0;
        }
      }
      failed = failed || !__shfl_sync(0xffffffffu, okw, 0);
      for (int i = 0; i < oz::S; ++i) {
        const int ai = kb * oz::S + i;
        const int s = ai % kAStages;
        const uint32_t ph = (uint32_t)(ai / kAStages) & 1u;
        int oka = 1;
        if (lane == 0 && !failed) {
          if (!mbar_wait_spin(&afull[s], ph)) {
            atomicExch(err, tc::ERR_TIMEOUT_FULL);
            *abort_flag = 1;
            oka = 0;
          } else if (*abort_flag) {
            oka = 0;
          }
        }
        failed = failed || !__shfl_sync(0xffffffffu, oka, 0);
        (void)handoff(failed);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (lane 0; the whole warp meets the waiter at barrier 2)
    constexpr uint32_t idesc = tc::make_idesc(1, oz::BN);
    constexpr uint32_t idesc2 = tc::make_idesc(1, 2 * oz::BN);
    constexpr uint32_t idesc3 = tc::make_idesc(1, 3 * oz::BN);
    constexpr uint32_t idesc4 = tc::make_idesc(1, 4 * oz::BN);
    const uint64_t adesc0 = tc::make_sw128_desc(tc::smem_u32(sA));
    const uint64_t bdesc0 = tc::make_sw128_desc(tc::smem_u32(sB));
    bool& failed = mma_failed;
    for (int kb = 0; kb < num_kb; ++kb) {
      const bool chunk_start = (kb % kKbPerChunk) == 0;
      const int g = kb & 1;
      for (int i = 0; i < oz::S; ++i) {
        failed = handoff(false) || failed;
        tc::fence_after_sync();
        const int ai = kb * oz::S + i;
        const int s = ai % kAStages;
        if (lane == 0) {
          if (!failed) {
            const uint64_t ad = adesc0 + (uint64_t)(s * (kATile >> 4));
            const uint64_t bd = bdesc0 + (uint64_t)(g * oz::S * (kBTile >> 4));
            // slice 0 is the first to reach every level, so in a chunk's first k-block its MMAs
            // overwrite and all later ones accumulate; up to four pairs (i, j .. j + 3), i.e.
            // adjacent levels and adjacent B slices, go into one MMA of N = 64 .. 256
            const uint32_t first = (!chunk_start || i > 0) ? 1u : 0u;
#pragma unroll
            for (int j = 0; j < oz::S; j += kLevelsPerMma) {
              if (i + j < oz::S) {
                const int gl = min(kLevelsPerMma, oz::S - i - j);
                const uint32_t id = gl == 1 ? idesc : gl == 2 ? idesc2 : gl == 3 ? idesc3 : idesc4;
                const uint32_t d = tmem + (uint32_t)((i + j) * oz::BN);
                const uint64_t bj = bd + (uint64_t)(j * (kBTile >> 4));
                tc::mma_issue<true>(d, ad, bj, id, first);
                tc::mma_issue<true>(d, ad + 2, bj + 2, id, 1u);
                tc::mma_issue<true>(d, ad + 4, bj + 4, id, 1u);
                tc::mma_issue<true>(d, ad + 6, bj + 6, id, 1u);
              }
            }
            mma_any = true;
          }
          // also after a failure (the A producer never starves), unless the failure came
          // before any MMA: then no asynchronous arrive may outlive the CTA
          if (mma_any || !failed) tc::mma_commit(&aempty[s]);
        }
        __syncwarp();
      }
      if (lane == 0 && (mma_any || !failed)) {
        tc::mma_commit(&bempty[g]);
        if ((kb % kKbPerChunk) == kKbPerChunk - 1 || kb == num_kb - 1) tc::mma_commit(cdone);
      }
      __syncwarp();
    }
  } else if (warp >= 3) {
    // ---------------- epilogue: running double-float sums of 32 columns per thread
    const int quarter = warp & 3;
    const int cbase = ((warp - 3) >> 2) * 32;
    const int row = m0 + quarter * 32 + lane;
    float rh[32], rl[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) rh[t] = rl[t] = 0.f;
    bool go = true;
    for (int q = 0; q < nchunks && go; ++q) {
      int okw = 1;
      if (lane == 0) {
        okw = tc::mbar_wait(cdone, (uint32_t)q & 1u) ? 1 : 0;
        if (!okw) {
          atomicExch(err, tc::ERR_TIMEOUT_DONE);
          *abort_flag = 1;
        }
        if (*abort_flag) okw = 0;
      }
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) {
        go = false;
        break;
      }
      tc::fence_after_sync();
      const int ea = row < M ? eA[(int64_t)q * M + row] : 0;
#pragma unroll
      for (int c8 = 0; c8 < 32; c8 += 8) {
        uint32_t v[oz::S][8];
#pragma unroll
        for (int L = 0; L < oz::S; ++L) tmem_ld8_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(L * oz::BN + cbase + c8), v[L]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float f4 = __uint_as_float(v[4][t]), f5 = __uint_as_float(v[5][t]), f6 = __uint_as_float(v[6][t]);
          float tail = __fmul_rn(f6, pow2f(-oz::BITS * 8));
          tail = __fadd_rn(tail, __fmul_rn(f5, pow2f(-oz::BITS * 7)));
          tail = __fadd_rn(tail, __fmul_rn(f4, pow2f(-oz::BITS * 6)));
          float hh = tail, ll = 0.f;
          df_add_f(hh, ll, __fmul_rn(__uint_as_float(v[3][t]), pow2f(-oz::BITS * 5)));
          df_add_f(hh, ll, __fmul_rn(__uint_as_float(v[2][t]), pow2f(-oz::BITS * 4)));
          df_add_f(hh, ll, __fmul_rn(__uint_as_float(v[1][t]), pow2f(-oz::BITS * 3)));
          df_add_f(hh, ll, __fmul_rn(__uint_as_float(v[0][t]), pow2f(-oz::BITS * 2)));
          const int col = n0 + cbase + c8 + t;
          const int ex = ea + (col < N ? eB[(int64_t)q * N + col] : 0);
          df_add(rh[c8 + t], rl[c8 + t], scale2(hh, ex), scale2(ll, ex));
        }
      }
      // this warp has read chunk q: release the accumulators
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(tfree)) : "memory");
    }
    if (go && row < M) {
      if (o.mode == ACC_ROWMAJOR) {
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int col = n0 + cbase + t;
          if (col < N) o.C[(int64_t)row * o.ldc + col] = (double)rh[t] + (double)rl[t];
        }
      } else if (o.mode == ACC_COLMAJOR) {  // lanes hold consecutive rows: coalesced per column
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int col = n0 + cbase + t;
          if (col < N) {
            const double v = (double)rh[t] + (double)rl[t];
            o.C[(int64_t)col * o.ldc + row] = v;
            if (o.C32) o.C32[(int64_t)col * o.ldc + row] = (float)v;
          }
        }
      } else {  // ACC_ROWSQ
        double sq = 0.0;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const double v = (double)rh[t] + (double)rl[t];
          if (n0 + cbase + t < N) sq = fma(v, v, sq);
        }
        o.sq[((int64_t)blockIdx.x * 2 + (cbase >> 5)) * o.ldc + row] = sq;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    // all MMAs have completed once the last chunk was signalled (or a wait gave up)
    if (lane == 0 && (mma_any || !mma_failed) && nchunks > 0)
      (void)tc::mbar_wait_bounded(cdone, (uint32_t)(nchunks - 1) & 1u);
    __syncwarp();
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// ------------------------------------------------------------ nonlinear step and back-projection
// beta_ab = c^2 S_ab (T_ab - t_b) in double-float (T from its chunk partials), sliced
// row-wise into the A operand of segment 2, with the row sums of each 256-column chunk.
// One CTA (256 threads) per row a and 1024-column block: thread u takes columns 4u .. 4u + 3
// (16- and 32-byte loads, one 8-byte store of four BF16 per slice); the 64 threads of a
// chunk share its exponent and reduce its row sum in a fixed order.
__global__ void __launch_bounds__(256) oz_beta_kernel(const float2* __restrict__ Tp, int nsplit, int64_t M,
                                                      int64_t MB, const float2* __restrict__ S2, const float2* __restrict__ t2,
                                                      int64_t Rp, int64_t Kp, bf16* __restrict__ sl,
                                                      int* __restrict__ e, float2* __restrict__ rs2) {
  __shared__ float redm[8];
  __shared__ float2 redp[8];
  const int64_t a = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t b0 = (int64_t)blockIdx.y * 1024 + 4 * threadIdx.x; b0 - 4 * threadIdx.x < Kp; b0 += 1024 * gridDim.y) {
    float bh[4] = {0.f, 0.f, 0.f, 0.f}, bl[4] = {0.f, 0.f, 0.f, 0.f};
    if ((MB & 3) == 0 && b0 + 3 < MB) {  // 16-byte aligned rows; otherwise the scalar path below
      float th[4], tl[4];
      {  // the first partial as it is (a normalised pair), the others added
        const float4* pp = reinterpret_cast<const float4*>(Tp + a * MB + b0);
        const float4 p0 = pp[0], p1 = pp[1];
        th[0] = p0.x, tl[0] = p0.y, th[1] = p0.z, tl[1] = p0.w;
        th[2] = p1.x, tl[2] = p1.y, th[3] = p1.z, tl[3] = p1.w;
      }
      for (int s = 1; s < nsplit; ++s) {
        const float4* pp = reinterpret_cast<const float4*>(Tp + ((int64_t)s * M + a) * MB + b0);
        const float4 p0 = pp[0], p1 = pp[1];
        df_add(th[0], tl[0], p0.x, p0.y);
        df_add(th[1], tl[1], p0.z, p0.w);
        df_add(th[2], tl[2], p1.x, p1.y);
        df_add(th[3], tl[3], p1.z, p1.w);
      }
      const float4* tp = reinterpret_cast<const float4*>(t2 + b0);
      const float4* sp = reinterpret_cast<const float4*>(S2 + a * MB + b0);
      const float4 t0 = tp[0], t1 = tp[1], s0 = sp[0], s1 = sp[1];
      const float tbh[4] = {t0.x, t0.z, t1.x, t1.z}, tbl[4] = {t0.y, t0.w, t1.y, t1.w};
      const float sh[4] = {s0.x, s0.z, s1.x, s1.z}, slo[4] = {s0.y, s0.w, s1.y, s1.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        df_add(th[q], tl[q], -tbh[q], -tbl[q]);
        df_mul(sh[q], slo[q], th[q], tl[q], bh[q], bl[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t b = b0 + q;
        if (b < MB) {
          float th = 0.f, tl = 0.f;
          for (int s = 0; s < nsplit; ++s) {
            const float2 p = Tp[((int64_t)s * M + a) * MB + b];
            df_add(th, tl, p.x, p.y);
          }
          const float2 tb = t2[b];
          df_add(th, tl, -tb.x, -tb.y);
          const float2 sab = S2[a * MB + b];
          df_mul(sab.x, sab.y, th, tl, bh[q], bl[q]);
        }
      }
    }
    // chunk of these columns: threads 64 c .. 64 c + 63 (warps 2c, 2c + 1)
    float mx = fmaxf(fmaxf(fabsf(bh[0]), fabsf(bh[1])), fmaxf(fabsf(bh[2]), fabsf(bh[3])));
    float rh = bh[0], rl = bl[0];
    df_add(rh, rl, bh[1], bl[1]);
    df_add(rh, rl, bh[2], bl[2]);
    df_add(rh, rl, bh[3], bl[3]);
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float oh = __shfl_xor_sync(0xffffffffu, rh, o), ol = __shfl_xor_sync(0xffffffffu, rl, o);
      df_add(rh, rl, oh, ol);
    }
    if (lane == 0) {
      redm[warp] = mx;
      redp[warp] = make_float2(rh, rl);
    }
    __syncthreads();
    const int c = warp >> 1;
    const float m = fmaxf(redm[2 * c], redm[2 * c + 1]);
    int ex = 0;
    if (m > 0.f) {
      const int bits = __float_as_int(m);
      ex = (bits >> 23) != 0 ? (bits >> 23) - 126 : 0;  // m = f 2^ex, f in [0.5, 1), for normal m
      if ((bits >> 23) == 0) (void)frexpf(m, &ex);
    }
    const int64_t q = (b0 - 4 * (threadIdx.x & 63)) / oz::KC;  // this chunk
    if ((threadIdx.x & 63) == 0 && q * oz::KC < MB) {
      float h = redp[2 * c].x, l = redp[2 * c].y;
      df_add(h, l, redp[2 * c + 1].x, redp[2 * c + 1].y);
      rs2[q * M + a] = make_float2(h, l);
      e[q * M + a] = ex;
    }
    // 7 slices of the four entries, one 8-byte store each
    if (b0 < Kp) {
      float yh[4], yl[4];
      const int sh7 = oz::BITS - ex;
      if (sh7 >= -126 && sh7 <= 127) {  // one power of two for the eight scalings
        const float f = pow2f(sh7);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          yh[u] = __fmul_rn(bh[u], f);
          yl[u] = __fmul_rn(bl[u], f);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          yh[u] = scale2(bh[u], sh7);
          yl[u] = scale2(bl[u], sh7);
        }
      }
      const float up = (float)(1 << oz::BITS);
      bf16* dst = sl + a * Kp + b0;
      const int64_t stride = Rp * Kp;
#pragma unroll
      for (int i = 0; i < oz::S; ++i) {
        float sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sv[u] = rintf(yh[u]);
          float h, l;
          fast_two_sum(__fsub_rn(yh[u], sv[u]), yl[u], h, l);  // exact: see slice_write
          yh[u] = __fmul_rn(h, up);
          yl[u] = __fmul_rn(l, up);
        }
        const __nv_bfloat162 lo2 = __floats2bfloat162_rn(sv[0], sv[1]), hi2 = __floats2bfloat162_rn(sv[2], sv[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<const uint32_t*>(&lo2);
        pk.y = *reinterpret_cast<const uint32_t*>(&hi2);
        *reinterpret_cast<uint2*>(dst + i * stride) = pk;
      }
    }
    __syncthreads();  // redm / redp reused by the next block of columns
  }
}

// (K v)_a = J_a^T (U_a - rowsum_a xc_a) (+ lambda v_a) in double-float arithmetic (the FP64
// form of this kernel was bound by GB300's FP64 pipe).  U_a and rowsum_a are summed from
// their double-float partials; xc_a and the Jacobian factors come as float pairs (Xc2, G2).
// One CTA of 256 threads per geometry: thread p issues every load of its descriptors
// (up to kBackDesc per thread in registers, the rest in a loop), forms w_p = g_p u_p with
// u_p = U_ap - rowsum_a xc_ap; then two lanes per output (atom i, coordinate c) sum halves
// of the N - 1 pair terms from shared memory (the derivative of x_p with respect to its
// first atom i > j carries the minus sign), combined by one shuffle; the FP64 result is
// hi + lo (+ lambda v in FP64).
constexpr int kBackDesc = 4;
__global__ void __launch_bounds__(256) oz_backproj_df_kernel(const float2* __restrict__ Up, int nsplit, int64_t M,
                                                             int D, const float2* __restrict__ rs2, int nrs,
                                                             const float2* __restrict__ Xc2,
                                                             const float2* __restrict__ G2,
                                                             const double* __restrict__ v, int N, double lam,
                                                             int add_lambda, double* __restrict__ out) {
  extern __shared__ float2 w3f[];  // [D][3]: the terms g_p u_p
  __shared__ float2 rs;
  const int64_t a = blockIdx.x;
  const int tid = threadIdx.x;
  const float2* Ga = G2 + a * D * 3;
  const float2* Ua = Up + a * D;
  const int64_t sstride = M * D;
  const float2 z = make_float2(0.f, 0.f);
  // the first kBackDesc descriptors of this thread: every load in one round
  float2 g[kBackDesc][3], xc[kBackDesc], u[kBackDesc];
#pragma unroll
  for (int q = 0; q < kBackDesc; ++q) {
    const int p = q * 256 + tid;
    const bool in = p < D;
    g[q][0] = in ? Ga[3 * p] : z;
    g[q][1] = in ? Ga[3 * p + 1] : z;
    g[q][2] = in ? Ga[3 * p + 2] : z;
    xc[q] = in ? Xc2[a * D + p] : z;
    u[q] = in ? Ua[p] : z;
  }
  for (int s = 1; s < nsplit; ++s) {
#pragma unroll
    for (int q = 0; q < kBackDesc; ++q) {
      const int p = q * 256 + tid;
      const float2 w = p < D ? Ua[s * sstride + p] : z;
      df_add(u[q].x, u[q].y, w.x, w.y);
    }
  }
  if (tid < 32) {
    float h = 0.f, l = 0.f;
    for (int q = tid; q < nrs; q += 32) {
      const float2 p = rs2[(int64_t)q * M + a];
      df_add(h, l, p.x, p.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      df_add(h, l, oh, ol);
    }
    if (tid == 0) rs = make_float2(h, l);
  }
  __syncthreads();
  const float2 r = rs;
  auto term = [&](int p, float2 uu, const float2 (&gg)[3], float2 xx) {
    float ph, pl, uh = uu.x, ul = uu.y;
    df_mul(r.x, r.y, xx.x, xx.y, ph, pl);
    df_add(uh, ul, -ph, -pl);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float wh, wl;
      df_mul(gg[c].x, gg[c].y, uh, ul, wh, wl);
      w3f[3 * p + c] = make_float2(wh, wl);
    }
  };
#pragma unroll
  for (int q = 0; q < kBackDesc; ++q) {
    const int p = q * 256 + tid;
    if (p < D) term(p, u[q], g[q], xc[q]);
  }
  for (int p = kBackDesc * 256 + tid; p < D; p += 256) {  // D > 1024: the rest, one at a time
    float2 uu = Ua[p];
    for (int s = 1; s < nsplit; ++s) {
      const float2 w = Ua[s * sstride + p];
      df_add(uu.x, uu.y, w.x, w.y);
    }
    const float2 gg[3] = {Ga[3 * p], Ga[3 * p + 1], Ga[3 * p + 2]};
    term(p, uu, gg, Xc2[a * D + p]);
  }
  __syncthreads();
  const int B = 3 * N;
  const int half = tid & 1;
  for (int o0 = 0; o0 < B; o0 += 128) {  // every lane pair runs the same trip count
    const int o = o0 + (tid >> 1);
    float h = 0.f, l = 0.f;
    if (o < B) {
      const int i = o / 3, qd = o - 3 * i;
      for (int j = half; j < N; j += 2) {
        if (j == i) continue;
        const float2 w = w3f[3 * pair_idx(i, j) + qd];
        if (i > j)
          df_add(h, l, -w.x, -w.y);
        else
          df_add(h, l, w.x, w.y);
      }
    }
    const float oh = __shfl_xor_sync(0xffffffffu, h, 1), ol = __shfl_xor_sync(0xffffffffu, l, 1);
    df_add(h, l, oh, ol);
    if (o < B && half == 0) {
      double s = (double)h + (double)l;
      if (add_lambda) s = fma(lam, v[a * B + o], s);
      out[a * B + o] = s;
    }
  }
}

// C = sum of the double-float partials, as FP64 (test hook)
__global__ void oz_sum_partials_kernel(const float2* __restrict__ P, int nsplit, int64_t count, double* __restrict__ C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  float h = 0.f, l = 0.f;
  for (int s = 0; s < nsplit; ++s) {
    const float2 p = P[(int64_t)s * count + i];
    df_add(h, l, p.x, p.y);
  }
  C[i] = (double)h + (double)l;
}

}  // namespace

// ------------------------------------------------------------ host side
#define OZ_TRY(x)                 \
  do {                            \
    gdml_status _s = (x);         \
    if (_s != GDML_OK) return _s; \
  } while (0)

template <typename T>
static gdml_status oz_alloc(OzMatvec& oz, T** p, size_t count, cudaStream_t st) {
  void* v = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&v, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GDML_ERR_OOM, "sliced tensor-core buffers: cudaMalloc failed");
  }
  oz.allocs.push_back(v);
  *p = static_cast<T*>(v);
  if (cudaMemsetAsync(v, 0, bytes, st) != cudaSuccess) return fail(GDML_ERR_CUDA, "sliced buffer memset");
  return GDML_OK;
}

static gdml_status make_operand(OzMatvec& oz, OzOperand& op, int64_t rows, int64_t K, int box_rows,
                                cudaStream_t st) {
  op.rows = rows;
  op.Rp = cdiv(rows, box_rows) * box_rows;
  op.K = K;
  op.Kp = cdiv(K, 2 * oz::KB) * (2 * oz::KB);  // k-blocks of 128 for the matvec GEMM
  op.nchunks = cdiv(K, oz::KC);
  bf16* s = nullptr;
  OZ_TRY(oz_alloc(oz, &s, (size_t)(oz::S * op.Rp * op.Kp), st));
  OZ_TRY(oz_alloc(oz, &op.e, (size_t)(op.nchunks * rows), st));
  op.slices = s;
  if (!make_kmajor_map(&op.map, s, true, (uint64_t)op.Kp, (uint64_t)(oz::S * op.Rp), (uint64_t)op.Kp,
                       (uint32_t)box_rows))
    return fail(GDML_ERR_CUDA, "cuTensorMapEncodeTiled failed (sliced operand)");
  return GDML_OK;
}

static void slice_rows(const double* X, int64_t ldx, OzOperand& op, cudaStream_t st, const double* t = nullptr,
                       float2* t2 = nullptr) {
  dim3 g((unsigned)op.rows, (unsigned)op.nchunks);
  { oz_slice_rows_kernel<<<g, 256, 0, st>>>(X, ldx, op.K, op.rows, op.Rp, op.Kp, (bf16*)op.slices, op.e, t, t2); count_launch(); }
}

static void transpose(const double* X, int64_t rows, int64_t cols, int64_t ldx, double* XT, cudaStream_t st) {
  dim3 g((unsigned)cdiv(cols, 32), (unsigned)cdiv(rows, 32));
  { oz_transpose_kernel<<<g, dim3(32, 8), 0, st>>>(X, rows, cols, ldx, XT); count_launch(); }
}

// K chunks per CTA of the matvec GEMM.  Time ~ whole waves of CTAs x (chunks per CTA + a fixed
// per-CTA cost of about half a chunk: start-up, drain, write-out); the G minimising it, the
// larger G (fewer groups, fewer partials for the consumer to read) on ties.  A partial last
// wave costs as much as a full one, so e.g. 560 tiles x 20 chunks prefers one group of 20
// (3.7 waves -> 4) to three groups of 7 (11.05 waves -> 12).
int oz_auto_chunks_per_cta(int64_t tiles, int64_t nchunks) {
  const int64_t sms = num_sms();
  tiles = std::max<int64_t>(tiles, 1);
  int best = 1;
  int64_t best_cost = INT64_MAX;
  for (int64_t G = 1; G <= std::max<int64_t>(nchunks, 1); ++G) {
    const int64_t groups = cdiv(nchunks, G), geff = cdiv(nchunks, groups);
    const int64_t cost = cdiv(tiles * groups, sms) * (2 * geff + 1);  // in half chunks
    if (cost <= best_cost) {
      best_cost = cost;
      best = (int)G;
    }
  }
  return best;
}

// C partials (groups of G chunks, one float2 slab per group at out + z split_stride) of
// A B^T, or with a second pair (A2, B2) of A B^T + A2 B2^T as one product over the
// concatenated K (A2 has A's rows, B2 B's); *groups_out = number of slabs written
static gdml_status oz_gemm(const OzOperand& A, const OzOperand& B, float2* out, int64_t ldo, int64_t split_stride,
                           int* err, cudaStream_t st, int G, int* groups_out = nullptr, int nlev = oz::S,
                           const OzOperand* A2 = nullptr, const OzOperand* B2 = nullptr) {
  static bool attr_set = false;
  if (!attr_set) {
    for (auto fn : {oz_gemm_kernel<1>, oz_gemm_kernel<2>, oz_gemm_kernel<3>, oz_gemm_kernel<4>, oz_gemm_kernel<5>,
                    oz_gemm_kernel<6>, oz_gemm_kernel<7>})
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotalM) != cudaSuccess)
        return fail(GDML_ERR_CUDA, "cudaFuncSetAttribute(sliced gemm)");
    attr_set = true;
  }
  if (A.Kp != B.Kp) return fail(GDML_ERR_ARG, "sliced gemm: K mismatch");
  if (A.Kp % oz::KB != 0 || (A2 && A.Kp % oz::KC != 0)) return fail(GDML_ERR_ARG, "sliced gemm: K padding");
  if (nlev < 1 || nlev > oz::S) return fail(GDML_ERR_ARG, "sliced gemm: levels outside 1..7");
  if (!A2 != !B2) return fail(GDML_ERR_ARG, "sliced gemm: the second segment needs both operands");
  const OzOperand& SA = A2 ? *A2 : A;
  const OzOperand& SB = B2 ? *B2 : B;
  if (A2 && (SA.Kp != SB.Kp || SA.Kp % oz::KB != 0 || SA.rows != A.rows || SB.rows != B.rows))
    return fail(GDML_ERR_ARG, "sliced gemm: second segment shape mismatch");
  const int kb1 = (int)(A.Kp / oz::KB);
  const int num_kb = kb1 + (A2 ? (int)(SA.Kp / oz::KB) : 0);
  const int64_t nchunks = A.nchunks + (A2 ? SA.nchunks : 0);
  G = std::max(1, std::min<int>(G, (int)nchunks));
  const int groups = (int)cdiv(nchunks, G);
  dim3 grid((unsigned)cdiv(B.rows, oz::BN), (unsigned)cdiv(A.rows, oz::BM), (unsigned)groups);
  static void (*const kern[])(const CUtensorMap, const CUtensorMap, int, int, int, int, int, int, const int*,
                              const int*, float2*, int64_t, int64_t, int*, const CUtensorMap, const CUtensorMap, int,
                              int, const int*, const int*, int) = {
      oz_gemm_kernel<1>, oz_gemm_kernel<2>, oz_gemm_kernel<3>, oz_gemm_kernel<4>,
      oz_gemm_kernel<5>, oz_gemm_kernel<6>, oz_gemm_kernel<7>};
  { kern[nlev - 1]<<<grid, kThreads, kSmemTotalM, st>>>(A.map, B.map, (int)A.Rp, (int)B.Rp, (int)A.rows, (int)B.rows, num_kb, G, A.e, B.e, out, ldo, split_stride, err, SA.map, SB.map, (int)SA.Rp, (int)SB.Rp, SA.e, SB.e, A2 ? kb1 : num_kb); count_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("sliced gemm launch: ") + cudaGetErrorString(e));
  if (groups_out) *groups_out = groups;
  return GDML_OK;
}

gdml_status oz_setup(OzMatvec& oz, int64_t M, int N, int D, const double* Xc, const double* A, int64_t ldA,
                     const double* S, double c, cudaStream_t st, int Ssym, const int* pis, const double* XcB) {
  if (Ssym < 1 || (Ssym > 1 && (!pis || !XcB))) return fail(GDML_ERR_ARG, "sliced setup: bad symmetry arguments");
  const int64_t MB = M * Ssym;
  if (MB > (int64_t)1 << 24 || D > (1 << 20)) return fail(GDML_ERR_ARG, "system too large for the sliced path");
  oz.M = M;
  oz.MB = MB;
  oz.N = N;
  oz.D = D;
  oz.S = Ssym;
  oz.pis = pis;
  oz.XcB = Ssym > 1 ? XcB : Xc;
  OZ_TRY(make_operand(oz, oz.Xc1, M, D, oz::BM, st));
  OZ_TRY(make_operand(oz, oz.W1, MB, D, oz::BN, st));
  OZ_TRY(make_operand(oz, oz.A2, M, MB, oz::BM, st));
  OZ_TRY(make_operand(oz, oz.WT2, D, MB, oz::BN, st));
  OZ_TRY(make_operand(oz, oz.B2, M, MB, oz::BM, st));
  OZ_TRY(make_operand(oz, oz.XT2, D, MB, oz::BN, st));
  OZ_TRY(oz_alloc(oz, &oz.W, (size_t)(M * D), st));
  OZ_TRY(oz_alloc(oz, &oz.Wf, (size_t)(M * D), st));
  OZ_TRY(oz_alloc(oz, &oz.Xc2, (size_t)(M * D), st));
  if (Ssym > 1) OZ_TRY(oz_alloc(oz, &oz.WB, (size_t)(MB * D), st));
  OZ_TRY(oz_alloc(oz, &oz.WT, (size_t)(MB * D), st));
  OZ_TRY(oz_alloc(oz, &oz.t, (size_t)MB, st));
  OZ_TRY(oz_alloc(oz, &oz.t2, (size_t)MB, st));
  OZ_TRY(oz_alloc(oz, &oz.S2, (size_t)(M * MB), st));
  OZ_TRY(oz_alloc(oz, &oz.Tp, (size_t)(oz.W1.nchunks * M * MB), st));
  OZ_TRY(oz_alloc(oz, &oz.Up, (size_t)(2 * oz.A2.nchunks * M * D), st));
  OZ_TRY(oz_alloc(oz, &oz.rs2, (size_t)(oz.A2.nchunks * M), st));
  OZ_TRY(oz_alloc(oz, &oz.err, 1, st));
  oz.g1 = oz_auto_chunks_per_cta(cdiv(MB, oz::BN) * cdiv(M, oz::BM), oz.W1.nchunks);
  oz.u_merged = oz.A2.Kp % oz::KC == 0;
  oz.nch2 = oz.u_merged ? 2 * oz.A2.nchunks : oz.A2.nchunks;
  oz.g2 = oz_auto_chunks_per_cta(cdiv(D, oz::BN) * cdiv(M, oz::BM), oz.nch2);
  // fixed operands: Xc (GEMM 1 A), A (GEMM 2 A, segment 1), XcB^T (GEMM 2 B, segment 2), c^2 S;
  // Xc as float pairs for the projection and the back-projection
  slice_rows(Xc, D, oz.Xc1, st);
  launch_split_df(Xc, M * D, oz.Xc2, st);
  slice_rows(A, ldA, oz.A2, st);
  transpose(oz.XcB, MB, D, D, oz.WT, st);
  slice_rows(oz.WT, MB, oz.XT2, st);
  { oz_s2_kernel<<<(unsigned)cdiv(M * MB, 256), 256, 0, st>>>(S, M * MB, c * c, oz.S2); count_launch(); }
  if (cudaGetLastError() != cudaSuccess) return fail(GDML_ERR_CUDA, "sliced setup kernels");
  oz.ready = true;
  return GDML_OK;
}

gdml_status oz_matvec(OzMatvec& oz, const double* G, const float2* G2, const double* Xc, const double* v,
                      double* out, int add_lambda, double lam, cudaStream_t st, int lev) {
  if (!oz.ready) return fail(GDML_ERR_STATE, "sliced matvec not set up");
  if (!G2) return fail(GDML_ERR_ARG, "sliced matvec: the float-pair Jacobian factors are missing");
  const int64_t M = oz.M, MB = oz.MB;
  const int D = oz.D;
  if (oz.S > 1) {  // w_b = J_b v_b, then row b S + q = P_q w_b with t = xc_(bS+q) . w_(bS+q)
    launch_proj(G, Xc, v, M, oz.N, D, oz.W, D, oz.t, st);
    launch_sym_gather(oz.W, M, D, oz.pis, oz.S, oz.XcB, oz.WB, oz.t, st);
    slice_rows(oz.WB, D, oz.W1, st, oz.t, oz.t2);
    transpose(oz.WB, MB, D, D, oz.WT, st);
    slice_rows(oz.WT, MB, oz.WT2, st);
  } else if (oz.W1.nchunks <= kProjChunks) {
    // projection and slicing of W's rows in one kernel (double-float), then W^T's rows sliced
    // straight from the float pairs of W (a column slicing: no transposed copy)
    { oz_proj_slice_df_kernel<<<(unsigned)M, oz::KC, 3 * oz.N * sizeof(float2), st>>>(G2, oz.Xc2, v, M, oz.N, D, (int)oz.W1.nchunks, oz.Wf, oz.t, oz.t2, oz.W1.Rp, oz.W1.Kp, (bf16*)oz.W1.slices, oz.W1.e); count_launch(); }
    if (cdiv(D, 16) * oz.WT2.nchunks >= 2 * num_sms()) {
      dim3 g((unsigned)cdiv(D, 16), (unsigned)oz.WT2.nchunks);
      { oz_slice_cols_kernel<float2, 16><<<g, 256, 0, st>>>(oz.Wf, D, 0, D, MB, oz.WT2.Rp, oz.WT2.Kp, (bf16*)oz.WT2.slices, oz.WT2.e); count_launch(); }
    } else {
      dim3 g((unsigned)cdiv(D, 4), (unsigned)oz.WT2.nchunks);
      { oz_slice_cols_kernel<float2, 4><<<g, 256, 0, st>>>(oz.Wf, D, 0, D, MB, oz.WT2.Rp, oz.WT2.Kp, (bf16*)oz.WT2.slices, oz.WT2.e); count_launch(); }
    }
  } else {
    launch_proj(G, Xc, v, M, oz.N, D, oz.W, D, oz.t, st);
    slice_rows(oz.W, D, oz.W1, st, oz.t, oz.t2);
    transpose(oz.W, MB, D, D, oz.WT, st);
    slice_rows(oz.WT, MB, oz.WT2, st);
  }
  int groups1 = 0, groups2 = 0;
  OZ_TRY(oz_gemm(oz.Xc1, oz.W1, oz.Tp, MB, M * MB, oz.err, st, oz.g1, &groups1, lev));
  {
    dim3 g((unsigned)M, (unsigned)cdiv(oz.B2.Kp, 1024));
    { oz_beta_kernel<<<g, 256, 0, st>>>(oz.Tp, groups1, M, MB, oz.S2, oz.t2, oz.B2.Rp, oz.B2.Kp, (bf16*)oz.B2.slices, oz.B2.e, oz.rs2); count_launch(); }
  }
  const int64_t nch = oz.A2.nchunks;
  // U = A W + beta Xc: one product over the two K segments (when the first ends on a chunk
  // boundary), else two launches whose partials follow one another
  int nsplit2 = 0;
  if (oz.u_merged) {
    OZ_TRY(oz_gemm(oz.A2, oz.WT2, oz.Up, D, M * D, oz.err, st, oz.g2, &groups2, lev, &oz.B2, &oz.XT2));
    nsplit2 = groups2;
  } else {
    OZ_TRY(oz_gemm(oz.A2, oz.WT2, oz.Up, D, M * D, oz.err, st, oz.g2, &groups2, lev));
    OZ_TRY(oz_gemm(oz.B2, oz.XT2, oz.Up + (int64_t)groups2 * M * D, D, M * D, oz.err, st, oz.g2, nullptr, lev));
    nsplit2 = 2 * groups2;
  }
  const size_t smem = 3 * (size_t)D * sizeof(float2);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(oz_backproj_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { oz_backproj_df_kernel<<<(unsigned)M, 256, smem, st>>>(oz.Up, nsplit2, M, D, oz.rs2, (int)nch, oz.Xc2, G2, v, oz.N, lam, add_lambda, out); count_launch(); }
  if (cudaGetLastError() != cudaSuccess) return fail(GDML_ERR_CUDA, "sliced matvec kernels");
  return GDML_OK;
}

gdml_status oz_check(OzMatvec& oz, cudaStream_t st) {
  if (!oz.ready) return GDML_OK;
  int h = 0;
  if (cudaMemcpyAsync(&h, oz.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "reading the sliced-gemm error word");
  if (h) {
    cudaMemsetAsync(oz.err, 0, sizeof(int), st);
    return fail(GDML_ERR_TIMEOUT, "a sliced tcgen05 pipeline wait timed out (code " + std::to_string(h) + ")");
  }
  return GDML_OK;
}

void oz_destroy(OzMatvec& oz) {
  for (void* p : oz.allocs) cudaFree(p);
  oz.allocs.clear();
  oz.ready = false;
}

// C (lower triangle) = X X^T for the k rows of X, each of K entries, sliced by `slice`
template <typename SliceFn>
static gdml_status syrk_sliced(int64_t k, int64_t K, double* C, int64_t ldc, const SliceFn& slice, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(oz_gemm_acc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal) !=
        cudaSuccess)
      return fail(GDML_ERR_CUDA, "cudaFuncSetAttribute(sliced syrk)");
    attr_set = true;
  }
  OzMatvec t;
  OzOperand a;
  // one operand serves as A and B (a second map with the B box height)
  gdml_status s = make_operand(t, a, k, K, oz::BM, st);
  CUtensorMap mapB;
  if (s == GDML_OK && !make_kmajor_map(&mapB, a.slices, true, (uint64_t)a.Kp, (uint64_t)(oz::S * a.Rp),
                                       (uint64_t)a.Kp, (uint32_t)oz::BN))
    s = fail(GDML_ERR_CUDA, "cuTensorMapEncodeTiled failed (sliced syrk)");
  if (s == GDML_OK) s = oz_alloc(t, &t.err, 1, st);
  if (s == GDML_OK) {
    slice(a);
    dim3 grid((unsigned)cdiv(k, oz::BN), (unsigned)cdiv(k, oz::BM));
    const AccOut o{ACC_ROWMAJOR, 1, 0, C, nullptr, nullptr, ldc};
    { oz_gemm_acc_kernel<<<grid, kThreadsAcc, kSmemTotal, st>>>(a.map, mapB, (int)a.Rp, (int)a.Rp, (int)k, (int)k, (int)(a.Kp / oz::KB), a.e, a.e, o, t.err); count_launch(); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = fail(GDML_ERR_CUDA, std::string("sliced syrk launch: ") + cudaGetErrorString(e));
  }
  if (s == GDML_OK) {
    int h = 0;
    if (cudaMemcpyAsync(&h, t.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = fail(GDML_ERR_CUDA, "sliced syrk: synchronise");
    else if (h)
      s = fail(GDML_ERR_TIMEOUT, "sliced syrk: a tcgen05 pipeline wait timed out");
  }
  cudaStreamSynchronize(st);
  oz_destroy(t);
  return s;
}

gdml_status oz_syrk_lower(const float* L, int64_t n, int64_t k, double* C, int64_t ldc, cudaStream_t st) {
  if (n <= 0 || k <= 0) return fail(GDML_ERR_ARG, "oz_syrk_lower: empty sizes");
  // the k columns of L (stride n) are the rows of L^T
  return syrk_sliced(k, n, C, ldc, [&](OzOperand& a) {
    dim3 g((unsigned)k, (unsigned)a.nchunks);
    { oz_slice_rows_f32_kernel<<<g, 256, 0, st>>>(L, n, n, k, a.Rp, a.Kp, (bf16*)a.slices, a.e); count_launch(); }
  }, st);
}

gdml_status oz_syrk_lower_f64(const double* X, int64_t rows, int64_t K, int64_t ldx, double* C, int64_t ldc,
                              cudaStream_t st) {
  if (rows <= 0 || K <= 0) return fail(GDML_ERR_ARG, "oz_syrk_lower_f64: empty sizes");
  return syrk_sliced(rows, K, C, ldc, [&](OzOperand& a) {
    dim3 g((unsigned)rows, (unsigned)a.nchunks);
    { oz_slice_rows_kernel<<<g, 256, 0, st>>>(X, ldx, K, rows, a.Rp, a.Kp, (bf16*)a.slices, a.e, nullptr, nullptr); count_launch(); }
  }, st);
}

gdml_status oz_gemm_tall(const double* A, int64_t n, int64_t K, const double* B, int64_t NB, int64_t ldb, bool tri_b,
                         bool rowsq, double* out, float* out32, cudaStream_t st) {
  if (n <= 0 || K <= 0 || NB <= 0 || !A || !B || !out) return fail(GDML_ERR_ARG, "oz_gemm_tall: bad arguments");
  if (NB > ((int64_t)1 << 24) || K > ((int64_t)1 << 24)) return fail(GDML_ERR_ARG, "oz_gemm_tall: sizes too large");
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(oz_gemm_acc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal) !=
        cudaSuccess)
      return fail(GDML_ERR_CUDA, "cudaFuncSetAttribute(sliced gemm)");
    attr_set = true;
  }
  // rows of A per panel: the panel's slices (7 x P x Kp BF16) are the only copy of A made
  const int64_t P = std::min<int64_t>(cdiv(n, oz::BM) * oz::BM, 65536);
  const int64_t nbt = cdiv(NB, oz::BN);
  OzMatvec t;
  OzOperand a, b;
  double* sq = nullptr;
  gdml_status s = make_operand(t, b, NB, K, oz::BN, st);
  if (s == GDML_OK) s = make_operand(t, a, P, K, oz::BM, st);
  if (s == GDML_OK && rowsq) s = oz_alloc(t, &sq, (size_t)(2 * nbt * n), st);
  if (s == GDML_OK) s = oz_alloc(t, &t.err, 1, st);
  if (s == GDML_OK) {
    slice_rows(B, ldb, b, st);
    for (int64_t p0 = 0; p0 < n && s == GDML_OK; p0 += P) {
      const int64_t rows = std::min(P, n - p0);
      a.rows = rows;  // exponents of this panel are indexed [chunk][rows]
      {
        dim3 g((unsigned)cdiv(rows, 16), (unsigned)a.nchunks);
        oz_slice_cols_kernel<double><<<g, 256, 0, st>>>(A, n, p0, rows, K, a.Rp, a.Kp, (bf16*)a.slices, a.e);
        count_launch();
      }
      AccOut o{rowsq ? ACC_ROWSQ : ACC_COLMAJOR, 0, tri_b ? 1 : 0, rowsq ? nullptr : out + p0,
               (!rowsq && out32) ? out32 + p0 : nullptr, rowsq ? sq + p0 : nullptr, n};
      dim3 grid((unsigned)nbt, (unsigned)cdiv(rows, oz::BM));
      { oz_gemm_acc_kernel<<<grid, kThreadsAcc, kSmemTotal, st>>>(a.map, b.map, (int)a.Rp, (int)b.Rp, (int)rows, (int)NB, (int)(a.Kp / oz::KB), a.e, b.e, o, t.err); count_launch(); }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) s = fail(GDML_ERR_CUDA, std::string("sliced tall gemm launch: ") + cudaGetErrorString(e));
    }
    if (s == GDML_OK && rowsq) {
      oz_rowsq_reduce_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(sq, (int)(2 * nbt), n, out);
      count_launch();
    }
  }
  if (s == GDML_OK) {
    int h = 0;
    if (cudaMemcpyAsync(&h, t.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = fail(GDML_ERR_CUDA, "sliced tall gemm: synchronise");
    else if (h)
      s = fail(GDML_ERR_TIMEOUT, "sliced tall gemm: a tcgen05 pipeline wait timed out");
  }
  cudaStreamSynchronize(st);
  oz_destroy(t);
  return s;
}

cudaError_t set_wait_limit_oz(uint32_t polls) { return tc::set_wait_limit_here(polls); }
uint32_t tc_default_wait_limit() { return tc::kSpinLimit; }

gdml_status oz_gemm_test(const double* A, const double* B, int64_t M, int64_t N, int64_t K, int G, int nlev,
                         double* C, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return fail(GDML_ERR_ARG, "oz_gemm_test: empty sizes");
  OzMatvec t;
  OzOperand a, b;
  float2* part = nullptr;
  int groups = 0;
  gdml_status s = make_operand(t, a, M, K, oz::BM, st);
  if (s == GDML_OK) s = make_operand(t, b, N, K, oz::BN, st);
  if (s == GDML_OK) s = oz_alloc(t, &part, (size_t)(a.nchunks * M * N), st);
  if (s == GDML_OK) s = oz_alloc(t, &t.err, 1, st);
  if (s == GDML_OK) {
    slice_rows(A, K, a, st);
    slice_rows(B, K, b, st);
    if (G < 1) G = oz_auto_chunks_per_cta(cdiv(N, oz::BN) * cdiv(M, oz::BM), a.nchunks);
    s = oz_gemm(a, b, part, N, M * N, t.err, st, G, &groups, nlev);
  }
  if (s == GDML_OK) {
    { oz_sum_partials_kernel<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(part, groups, M * N, C); count_launch(); }
    int h = 0;
    if (cudaMemcpyAsync(&h, t.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = fail(GDML_ERR_CUDA, "oz_gemm_test: synchronise");
    else if (h)
      s = fail(GDML_ERR_TIMEOUT, "sliced tcgen05 pipeline wait timed out");
  }
  cudaStreamSynchronize(st);
  oz_destroy(t);
  return s;
}

}  // namespace gdml
