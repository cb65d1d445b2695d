// Woodbury apply of the Nystrom preconditioner (Eq. 4):
//   z = lambda^-1 [ r - L_k C^-1 L_k^T r ],  C = lambda I + L_k^T L_k.
// C^-1 is formed once per build from the FP64 Cholesky factor of C
// (C^-1 = L_C^-T L_C^-1), so the apply is three data-parallel passes:
//   t = L_k^T r,  u = C^-1 t (+ one refinement step),  z = (r - L_k u) / lambda
// instead of two latency-bound triangular solves per CG iteration.  L_k is
// stored column-major (n x k, column j at L + j*n) in FP64, or in FP32 for the
// mixed-precision contexts; all arithmetic is FP64.  Two HBM passes over L_k.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "tc_gemm.cuh"
#include "ws_stage.cuh"

namespace gdml {

constexpr int kRowsPerChunk = 4096;
constexpr int kColsPerCta = 8;

// part[j * nchunks + chunk] = sum_{i in chunk} L[i + j n] r[i]; one warp per column.
template <typename TL>
__global__ void __launch_bounds__(256) gemv_t_partial_kernel(const TL* __restrict__ L, int64_t n, int64_t k,
                                                             const double* __restrict__ r,
                                                             double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kColsPerCta + warp;
  const int64_t i0 = (int64_t)blockIdx.y * kRowsPerChunk;
  const int64_t i1 = i0 + kRowsPerChunk < n ? i0 + kRowsPerChunk : n;
  if (j >= k) return;
  const TL* col = L + j * n;
  double s = 0.0;
  for (int64_t i = i0 + lane; i < i1; i += 32) s = fma((double)col[i], r[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[j * gridDim.y + blockIdx.y] = s;
}

// t[j] = sum over the chunk partials part[j * nchunks + c]: one warp per column,
// lanes stride over the chunks, then a fixed shuffle tree
__global__ void __launch_bounds__(256) reduce_chunks_kernel(const double* __restrict__ part, int64_t nchunks,
                                                            int64_t k, double* __restrict__ t) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 8 + warp;
  if (j >= k) return;
  const double* pj = part + j * nchunks;
  double s = 0.0;
  for (int64_t c = lane; c < nchunks; c += 32) s += pj[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) t[j] = s;
}

// u = C^-1 t: one warp per row of the dense symmetric k x k inverse
__global__ void __launch_bounds__(256) symv_kernel(const double* __restrict__ A, int64_t k,
                                                   const double* __restrict__ t, double* __restrict__ u) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= k) return;
  const double* row = A + i * k;
  double s = 0.0;
  for (int64_t j = lane; j < k; j += 32) s = fma(row[j], t[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) u[i] = s;
}

// z[i] = (r[i] - sum_j L[i + j n] x[j]) / lambda.  64 rows x 4 column
// quarters per CTA (coalesced 512-byte row segments, 4 independent chains per
// row, combined in a fixed order); x staged through shared memory.
template <typename TL>
__global__ void __launch_bounds__(256) gemv_n_update_kernel(const TL* __restrict__ L, int64_t n, int64_t k,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ r, double inv_lam,
                                                            double* __restrict__ z) {
  __shared__ double xs[2048];
  __shared__ double part[4][64];
  const int rr = threadIdx.x & 63, q = threadIdx.x >> 6;
  const int64_t i = (int64_t)blockIdx.x * 64 + rr;
  double s = 0.0;
  for (int64_t j0 = 0; j0 < k; j0 += 2048) {
    const int64_t jn = (k - j0) < 2048 ? (k - j0) : 2048;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < jn; t += blockDim.x) xs[t] = x[j0 + t];
    __syncthreads();
    if (i < n) {
      const int64_t qa = (jn * q) / 4, qb = (jn * (q + 1)) / 4;
      const TL* Lc = L + j0 * n + i;
#pragma unroll 8
      for (int64_t j = qa; j < qb; ++j) s = fma((double)Lc[j * n], xs[j], s);
    }
  }
  part[q][rr] = s;
  __syncthreads();
  if (q == 0 && i < n) z[i] = (r[i] - ((part[0][rr] + part[1][rr]) + (part[2][rr] + part[3][rr]))) * inv_lam;
}

// e = t - C u (one warp per row)
__global__ void __launch_bounds__(256) residual_kernel(const double* __restrict__ C, int64_t k,
                                                       const double* __restrict__ t, const double* __restrict__ u,
                                                       double* __restrict__ e) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= k) return;
  const double* row = C + i * k;
  double s = 0.0;
  for (int64_t j = lane; j < k; j += 32) s = fma(row[j], u[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) e[i] = t[i] - s;
}

// u += C^-1 e
__global__ void __launch_bounds__(256) symv_add_kernel(const double* __restrict__ A, int64_t k,
                                                       const double* __restrict__ e, double* __restrict__ u) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= k) return;
  const double* row = A + i * k;
  double s = 0.0;
  for (int64_t j = lane; j < k; j += 32) s = fma(row[j], e[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) u[i] += s;
}

template <typename TL>
void woodbury_apply(const TL* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                    const double* r, double* z, double* part, double* t, cudaStream_t st) {
  const int64_t nchunks = cdiv(n, kRowsPerChunk);
  dim3 g1((unsigned)cdiv(k, kColsPerCta), (unsigned)nchunks);
  double* u = t + k;
  double* e = t + 2 * k;
  const unsigned gk = (unsigned)cdiv(k, 8);
  { gemv_t_partial_kernel<TL><<<g1, 256, 0, st>>>(L, n, k, r, part); count_launch(); }
  { reduce_chunks_kernel<<<(unsigned)cdiv(k, 8), 256, 0, st>>>(part, nchunks, k, t); count_launch(); }
  // u = C^-1 t, refined once with the FP64 residual t - C u: the explicit inverse
  // alone is accurate only to ~cond(C) eps; one step restores the accuracy of a
  // backward-stable solve at the cost of two more k x k passes
  { symv_kernel<<<gk, 256, 0, st>>>(Cinv, k, t, u); count_launch(); }
  { residual_kernel<<<gk, 256, 0, st>>>(C, k, t, u, e); count_launch(); }
  { symv_add_kernel<<<gk, 256, 0, st>>>(Cinv, k, e, u); count_launch(); }
  { gemv_n_update_kernel<TL><<<(unsigned)cdiv(n, 64), 256, 0, st>>>(L, n, k, u, r, 1.0 / lam, z); count_launch(); }
}

template void woodbury_apply<double>(const double*, int64_t, int64_t, const double*, const double*, double,
                                     const double*, double*, double*, double*, cudaStream_t);
template void woodbury_apply<float>(const float*, int64_t, int64_t, const double*, const double*, double,
                                    const double*, double*, double*, double*, cudaStream_t);

// doubles of the apply's partial buffer: the L^T r chunk partials of either layout
// (4096- or 512-row chunks) or the 16 column-group partials of the DF64 L u pass
int64_t woodbury_part_size(int64_t n, int64_t k) {
  const int64_t a = cdiv(n, 128) * k, b = 16 * n;  // row chunks of >= 128 rows (staged passes)
  return a > b ? a : b;
}

}  // namespace gdml

// ---------------------------------------------------------------------------
// DF64 contexts: L_k stored in FP32 (half the bytes); every product of an FP32
// factor entry with an FP64 vector entry is formed exactly as a pair of floats
// (TwoProduct by FMA on the vector's hi part, plus the lo part) and summed in
// double-float (TwoSum), so the passes are bandwidth-bound on the FP32 lanes
// instead of bound by the FP64 pipe.
namespace gdml {

// r split once per apply into float pairs (n FP64 operations instead of n k)
__global__ void split_df_kernel(const double* __restrict__ r, int64_t n, float2* __restrict__ rs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = r[i];
  const float hi = (float)v;
  rs[i] = make_float2(hi, (float)(v - (double)hi));
}

void launch_split_df(const double* x, int64_t count, float2* out, cudaStream_t st) {
  { split_df_kernel<<<(unsigned)cdiv(count, 256), 256, 0, st>>>(x, count, out); count_launch(); }
}

// (h, l) += (bh, bl) in double-float
__device__ __forceinline__ void df_add_pair(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float v = s - h;
  float e = (h - (s - v)) + (bh - v);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

// rows [i0 + base, i0 + base + 4) of one column as a float4 (zero past n)
template <bool VEC>
__device__ __forceinline__ float4 load4(const float* __restrict__ col, int64_t base, int64_t rem) {
  if (VEC && base + 3 < rem) return __ldcs(reinterpret_cast<const float4*>(col + base));  // streamed once
  float4 v;
  v.x = base < rem ? col[base] : 0.f;
  v.y = base + 1 < rem ? col[base + 1] : 0.f;
  v.z = base + 2 < rem ? col[base + 2] : 0.f;
  v.w = base + 3 < rem ? col[base + 3] : 0.f;
  return v;
}

constexpr int kDfRows = 512;     // rows per CTA of both passes (4 float4 per lane, 2 KB per warp and column)
constexpr int kDfTCols = 64;     // columns per CTA of the L^T r pass (8 warps x 8)
constexpr int kDfNGroups = 16;   // column groups of the L u pass (one partial per group)

template <bool VEC>
__device__ __forceinline__ void load_col(const float* __restrict__ col, int lane, int64_t rem, float4 (&v)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) v[t] = load4<VEC>(col, 128 * t + 4 * lane, rem);
}

// 8 per-lane double-float partials (one per column) -> column sums: a reduce-scatter
// across the warp (xor 16, 8, 4 halve the columns a lane keeps; xor 2, 1 finish the
// one left), 9 exchanges instead of 8 x 5.  Lane l ends with column
// ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1) summed over all 32 lanes.
__device__ __forceinline__ void reduce_scatter8(float (&h)[8], float (&l)[8], int lane, float& oh, float& ol) {
  const bool up4 = lane & 16, up2 = lane & 8, up1 = lane & 4;
  float h4[4], l4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float sh = up4 ? h[q] : h[4 + q], sl = up4 ? l[q] : l[4 + q];
    float kh = up4 ? h[4 + q] : h[q], kl = up4 ? l[4 + q] : l[q];
    df_add_pair(kh, kl, __shfl_xor_sync(0xffffffffu, sh, 16), __shfl_xor_sync(0xffffffffu, sl, 16));
    h4[q] = kh;
    l4[q] = kl;
  }
  float h2[2], l2[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float sh = up2 ? h4[q] : h4[2 + q], sl = up2 ? l4[q] : l4[2 + q];
    float kh = up2 ? h4[2 + q] : h4[q], kl = up2 ? l4[2 + q] : l4[q];
    df_add_pair(kh, kl, __shfl_xor_sync(0xffffffffu, sh, 8), __shfl_xor_sync(0xffffffffu, sl, 8));
    h2[q] = kh;
    l2[q] = kl;
  }
  {
    const float sh = up1 ? h2[0] : h2[1], sl = up1 ? l2[0] : l2[1];
    oh = up1 ? h2[1] : h2[0];
    ol = up1 ? l2[1] : l2[0];
    df_add_pair(oh, ol, __shfl_xor_sync(0xffffffffu, sh, 4), __shfl_xor_sync(0xffffffffu, sl, 4));
  }
  for (int o = 2; o > 0; o >>= 1) {
    const float sh = __shfl_xor_sync(0xffffffffu, oh, o), sl = __shfl_xor_sync(0xffffffffu, ol, o);
    df_add_pair(oh, ol, sh, sl);
  }
}

__device__ __forceinline__ void dot_col(const float4 (&a)[4], const float2 (&rv)[4][4], float& h, float& l) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    df_add_prod(h, l, a[t].x, rv[t][0].x, rv[t][0].y);
    df_add_prod(h, l, a[t].y, rv[t][1].x, rv[t][1].y);
    df_add_prod(h, l, a[t].z, rv[t][2].x, rv[t][2].y);
    df_add_prod(h, l, a[t].w, rv[t][3].x, rv[t][3].y);
  }
}

// part[j * nchunks + chunk] = sum over the chunk's 512 rows of L[i + j n] r[i]; r is
// held in registers as float pairs.  Each warp streams its 8 columns (2 KB contiguous
// per column) two at a time with the next pair's loads in flight (fully unrolled, two
// register buffers), keeps one per-lane partial per column and reduces all 8 at the
// end.  VEC: n % 4 == 0 (aligned float4 loads).
template <bool VEC>
__global__ void __launch_bounds__(256, 2) gemv_t_df_kernel(const float* __restrict__ L, int64_t n, int64_t k,
                                                           const float2* __restrict__ rs, double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.y * kDfRows;
  const int64_t rem = n - i0;
  float2 rv[4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t i = 128 * t + 4 * lane + e;
      rv[t][e] = i < rem ? rs[i0 + i] : make_float2(0.f, 0.f);
    }
  const int64_t jw = (int64_t)blockIdx.x * kDfTCols + warp * 8;
  if (jw >= k) return;
  const int ncol = (int)(jw + 8 < k ? 8 : k - jw);  // warp-uniform
  const float* base = L + jw * n + i0;
  float h[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) h[c] = l[c] = 0.f;
  float4 a0[4], b0[4], a1[4], b1[4];
  // column c of this warp is loaded only when c < ncol (never past the matrix)
  load_col<VEC>(base, lane, rem, a0);
  if (1 < ncol) load_col<VEC>(base + n, lane, rem, b0);
#pragma unroll
  for (int p = 0; p < 4; p += 2) {
    const int c = 2 * p;  // columns c, c+1 in (a0, b0); c+2, c+3 go to (a1, b1)
    if (c + 2 < ncol) load_col<VEC>(base + (int64_t)(c + 2) * n, lane, rem, a1);
    if (c + 3 < ncol) load_col<VEC>(base + (int64_t)(c + 3) * n, lane, rem, b1);
    if (c < ncol) dot_col(a0, rv, h[c], l[c]);
    if (c + 1 < ncol) dot_col(b0, rv, h[c + 1], l[c + 1]);
    if (c + 4 < ncol) load_col<VEC>(base + (int64_t)(c + 4) * n, lane, rem, a0);
    if (c + 5 < ncol) load_col<VEC>(base + (int64_t)(c + 5) * n, lane, rem, b0);
    if (c + 2 < ncol) dot_col(a1, rv, h[c + 2], l[c + 2]);
    if (c + 3 < ncol) dot_col(b1, rv, h[c + 3], l[c + 3]);
  }
  float oh, ol;
  reduce_scatter8(h, l, lane, oh, ol);
  const int col = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  if ((lane & 3) == 0 && col < ncol) part[(jw + col) * gridDim.y + blockIdx.y] = (double)oh + (double)ol;
}

// zp[g * n + i] = sum over column group g of L[i + j n] u[j]: CTA (row block of 512,
// group g); warp w takes every 8th column of the group, each lane 16 rows (4 float4,
// 2 KB contiguous per warp and column), next column's loads issued first; the 8
// warps' partials are combined in a fixed order through shared memory.
template <bool VEC>
__global__ void __launch_bounds__(256, 2) gemv_n_df_kernel(const float* __restrict__ L, int64_t n, int64_t k,
                                                           const float2* __restrict__ us, float2* __restrict__ zp) {
  __shared__ float2 part[8][kDfRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * kDfRows;
  const int64_t rem = n - i0;
  const int64_t g = blockIdx.y;
  const int64_t ja = k * g / kDfNGroups, jb = k * (g + 1) / kDfNGroups;
  float h[16], l[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) h[e] = l[e] = 0.f;
  // two columns in flight ahead of the one being summed
  int64_t j = ja + warp;
  float4 a[4], b[4];
  if (j < jb) load_col<VEC>(L + j * n + i0, lane, rem, a);
  if (j + 8 < jb) load_col<VEC>(L + (j + 8) * n + i0, lane, rem, b);
#pragma unroll 1
  for (; j < jb; j += 8) {
    float4 na[4];
    const bool more = j + 16 < jb;
    if (more) load_col<VEC>(L + (j + 16) * n + i0, lane, rem, na);
    const float2 x = us[j];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      df_add_prod(h[4 * t + 0], l[4 * t + 0], a[t].x, x.x, x.y);
      df_add_prod(h[4 * t + 1], l[4 * t + 1], a[t].y, x.x, x.y);
      df_add_prod(h[4 * t + 2], l[4 * t + 2], a[t].z, x.x, x.y);
      df_add_prod(h[4 * t + 3], l[4 * t + 3], a[t].w, x.x, x.y);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      a[t] = b[t];
      if (more) b[t] = na[t];
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) part[warp][128 * t + 4 * lane + e] = make_float2(h[4 * t + e], l[4 * t + e]);
  __syncthreads();
  for (int rr = threadIdx.x; rr < kDfRows; rr += 256) {
    if (rr >= rem) break;
    float hh = part[0][rr].x, ll = part[0][rr].y;
#pragma unroll
    for (int w = 1; w < 8; ++w) df_add_pair(hh, ll, part[w][rr].x, part[w][rr].y);
    zp[g * n + i0 + rr] = make_float2(hh, ll);
  }
}

// z[i] = (r[i] - sum_g zp[g][i]) / lambda (groups in a fixed order)
__global__ void gemv_n_df_finish_kernel(const float2* __restrict__ zp, int64_t n, const double* __restrict__ r,
                                        double inv_lam, double* __restrict__ z) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float hh = zp[i].x, ll = zp[i].y;
#pragma unroll
  for (int g = 1; g < kDfNGroups; ++g) df_add_pair(hh, ll, zp[g * n + i].x, zp[g * n + i].y);
  z[i] = (r[i] - ((double)hh + (double)ll)) * inv_lam;
}


// L^T r over units of RU rows (a multiple of 256, at most 1024) x a range of CPR columns (a
// multiple of 64): part[j * nru + ru] = sum over row unit ru of L[i + j n] r[i] as a
// double-float pair (the FP64 combination is left to the chunk reduction).  Tiles are
// 256 rows x 16 columns, taken column tile by column tile, the unit's RU / 256 row tiles
// of each in turn.  Warp w sums columns 2w, 2w + 1 of each tile over all RU rows of the unit
// (lane l: rows 4 l + 128 t + 256 rt + e, two packed chains per column: even and odd rows);
// every 4 column tiles it holds 8 columns and reduces them with one reduce-scatter, so the
// cross-lane reduction is paid once per 32 RU / 256 products per lane and column.  r of the
// unit's rows sits in shared memory as packed quads (hi, -hi, lo), loaded once per unit.
__global__ void __launch_bounds__(kWsThreads, 2)
    ws_gemv_t_kernel(const __grid_constant__ CUtensorMap map, int64_t n, int64_t k, int ru_rows, int64_t nru,
                     int ncr, int cpr, const float2* __restrict__ rs, float2* __restrict__ part,
                     int* __restrict__ err) {
  constexpr int RC = 256, COLS = 16;
  extern __shared__ uint8_t ws_smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws_smem_raw) + kWsAlign - 1) &
                                             ~uintptr_t(kWsAlign - 1));
  float4* rh4 = reinterpret_cast<float4*>(ring + kWsStages * kWsTile);  // [256] quads of rows
  float4* rn4 = rh4 + 256;
  float4* rl4 = rn4 + 256;
  uint64_t* full = reinterpret_cast<uint64_t*>(rl4 + 256);
  uint64_t* empty = full + kWsStages;
  uint64_t* cbar = empty + kWsStages;  // [2]: r quads written / unit finished
  volatile int* abort_flag = reinterpret_cast<volatile int*>(cbar + 2);
  __shared__ uint32_t issued_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rtiles = ru_rows / RC;
  const int64_t units = nru * ncr;
  if (threadIdx.x == 0) {
    ws_init(full, empty, cbar, abort_flag);
    issued_s = 0;
  }
  __syncthreads();
  if (warp == kWsWarps) {
    if (lane == 0) {
      uint64_t policy;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
      WsRing rp;
      uint32_t issued = 0;
      bool go = true;
      for (int64_t u = blockIdx.x; u < units && go; u += gridDim.x) {
        const int64_t ru = u / ncr;
        const int64_t c0 = (u % ncr) * cpr;
        const int64_t c1 = c0 + cpr < k ? c0 + cpr : k;
        const int ntc = (int)((c1 - c0 + COLS - 1) / COLS);
        for (int ct = 0; ct < ntc && go; ++ct)
          for (int rt = 0; rt < rtiles; ++rt, ++issued, rp.next()) {
            if (!ws_wait(&empty[rp.slot], rp.phase ^ 1u)) {
              atomicExch(err, tc::ERR_TIMEOUT_EMPTY);
              *abort_flag = 1;
              go = false;
              break;
            }
            if (*abort_flag) {
              go = false;
              break;
            }
            tc::mbar_expect_tx(&full[rp.slot], kWsTile);
            ws_tma_load(ring + rp.slot * kWsTile, &map, &full[rp.slot], (int)(ru * ru_rows + rt * RC),
                        (int)(c0 + ct * COLS), policy);
          }
      }
      issued_s = issued;
    }
  } else {
    WsRing rp;
    uint32_t ui = 0;
    bool go = true;
    for (int64_t u = blockIdx.x; u < units && go; u += gridDim.x, ++ui) {
      const int64_t ru = u / ncr;
      const int64_t c0 = (u % ncr) * cpr;
      const int64_t c1 = c0 + cpr < k ? c0 + cpr : k;
      const int ntc = (int)((c1 - c0 + COLS - 1) / COLS);
      const int64_t i0 = ru * ru_rows;
      {  // r of the unit's rows as packed quads
        const int g = threadIdx.x;  // 256 consumer threads, 4 rows each
        if (4 * g < ru_rows) {
          float4 h = make_float4(0.f, 0.f, 0.f, 0.f), lo = h;
          const int64_t i = i0 + 4 * g;
          if (i + 3 < n) {
            const float4 p0 = *reinterpret_cast<const float4*>(rs + i);  // n % 4 == 0: 16-byte aligned
            const float4 p1 = *reinterpret_cast<const float4*>(rs + i + 2);
            h = make_float4(p0.x, p0.z, p1.x, p1.z);
            lo = make_float4(p0.y, p0.w, p1.y, p1.w);
          }
          rh4[g] = h;
          rn4[g] = make_float4(-h.x, -h.y, -h.z, -h.w);
          rl4[g] = lo;
        }
      }
      if (!ws_consumer_sync(&cbar[0], ui & 1u, abort_flag, err)) break;
      for (int g = 0; g < ntc && go; g += 4) {
        float2 h2[8], l2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) h2[c] = l2[c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (g + q < ntc && go) {
#pragma unroll 1
            for (int rt = 0; rt < rtiles; ++rt) {
              if (!ws_consume_wait(&full[rp.slot], rp.phase, abort_flag, err)) {
                go = false;
                break;
              }
              const float* tile = reinterpret_cast<const float*>(ring + rp.slot * kWsTile) + 2 * warp * RC;
              float4 a[2][2];
#pragma unroll
              for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int t = 0; t < 2; ++t) a[c][t] = *reinterpret_cast<const float4*>(tile + c * RC + 128 * t + 4 * lane);
              __syncwarp();
              if (lane == 0) ws_arrive(&empty[rp.slot]);
              rp.next();
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const int gq = rt * 64 + 32 * t + lane;
                const float4 h = rh4[gq], ng = rn4[gq], lo = rl4[gq];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                  df2_add_prod_lazy(h2[2 * q + c], l2[2 * q + c], lo_pair(a[c][t]), lo_pair(h), lo_pair(ng), lo_pair(lo));
                  df2_add_prod_lazy(h2[2 * q + c], l2[2 * q + c], hi_pair(a[c][t]), hi_pair(h), hi_pair(ng), hi_pair(lo));
                }
              }
              df2_renorm(h2[2 * q], l2[2 * q]);
              df2_renorm(h2[2 * q + 1], l2[2 * q + 1]);
            }
          }
        }
        if (!go) break;
        float h[8], l[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          h[c] = h2[c].x;
          l[c] = l2[c].x;
          df_add_pair(h[c], l[c], h2[c].y, l2[c].y);
        }
        float oh, ol;
        reduce_scatter8(h, l, lane, oh, ol);
        // reduce-scatter slot c = 2 q + b holds column c0 + (g + q) 16 + 2 w + b
        const int c = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        const int64_t col = c0 + (int64_t)(g + (c >> 1)) * COLS + 2 * warp + (c & 1);
        if ((lane & 3) == 0 && col < c1) part[col * nru + ru] = make_float2(oh, ol);
      }
      if (!go) break;
      if (!ws_consumer_sync(&cbar[1], ui & 1u, abort_flag, err)) break;  // r quads free for the next unit
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) ws_drain(full, issued_s);
}

// z[i] = (r[i] - sum_j L[i + j n] u[j]) / lambda for the chunk's rows: 4 NT double-float
// chains per lane (its rows, packed in pairs), CPW products each per tile; the 8 warps' sums
// are combined in a fixed order through shared memory at the end of the chunk.
template <int NT>
__global__ void __launch_bounds__(kWsThreads, 2)
    ws_gemv_n_kernel(const __grid_constant__ CUtensorMap map, int64_t n, int64_t k, int64_t nch,
                     const float2* __restrict__ us, const double* __restrict__ r, double inv_lam,
                     double* __restrict__ z, int* __restrict__ err) {
  constexpr int RC = 128 * NT, COLS = 32 / NT, CPW = 4 / NT;
  extern __shared__ uint8_t ws_smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws_smem_raw) + kWsAlign - 1) &
                                             ~uintptr_t(kWsAlign - 1));
  float2* cmb = reinterpret_cast<float2*>(ring + kWsStages * kWsTile);  // [warp][RC rows]
  uint64_t* full = reinterpret_cast<uint64_t*>(cmb + kWsWarps * 256);
  uint64_t* empty = full + kWsStages;
  uint64_t* cbar = empty + kWsStages;  // [2]: combine buffer written / read
  volatile int* abort_flag = reinterpret_cast<volatile int*>(cbar + 2);
  __shared__ uint32_t issued_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (int)((k + COLS - 1) / COLS);
  if (threadIdx.x == 0) {
    ws_init(full, empty, cbar, abort_flag);
    issued_s = 0;
  }
  __syncthreads();
  if (warp == kWsWarps) {
    if (lane == 0) issued_s = ws_produce<NT, true>(&map, ring, full, empty, abort_flag, nch, ntiles, err);
  } else {
    WsRing rp;
    uint32_t ci = 0;
    bool go = true;
    for (int64_t ch = blockIdx.x; ch < nch && go; ch += gridDim.x, ++ci) {
      float2 h2[NT][2], l2[NT][2];  // rows 4 l + 128 t + {0,1} and {2,3}
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int p = 0; p < 2; ++p) h2[t][p] = l2[t][p] = make_float2(0.f, 0.f);
      for (int s = 0; s < ntiles; ++s) {
        float2 x[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const int64_t j = (int64_t)s * COLS + warp * CPW + c;
          x[c] = j < k ? us[j] : make_float2(0.f, 0.f);
        }
        if (!ws_consume_wait(&full[rp.slot], rp.phase, abort_flag, err)) {
          go = false;
          break;
        }
        const float* tile = reinterpret_cast<const float*>(ring + rp.slot * kWsTile) + warp * CPW * RC;
        float4 a[CPW][NT];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
          for (int t = 0; t < NT; ++t) a[c][t] = *reinterpret_cast<const float4*>(tile + c * RC + 128 * t + 4 * lane);
        __syncwarp();
        if (lane == 0) ws_arrive(&empty[rp.slot]);
        rp.next();
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const float2 uh = make_float2(x[c].x, x[c].x), un = make_float2(-x[c].x, -x[c].x),
                       ul = make_float2(x[c].y, x[c].y);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            df2_add_prod_lazy(h2[t][0], l2[t][0], lo_pair(a[c][t]), uh, un, ul);
            df2_add_prod_lazy(h2[t][1], l2[t][1], hi_pair(a[c][t]), uh, un, ul);
          }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
          for (int p = 0; p < 2; ++p) df2_renorm(h2[t][p], l2[t][p]);
      }
      if (!go) break;
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          cmb[warp * 256 + 128 * t + 4 * lane + 2 * p] = make_float2(h2[t][p].x, l2[t][p].x);
          cmb[warp * 256 + 128 * t + 4 * lane + 2 * p + 1] = make_float2(h2[t][p].y, l2[t][p].y);
        }
      if (!ws_consumer_sync(&cbar[0], ci & 1u, abort_flag, err)) break;
      const int64_t i0 = ch * RC;
      const int rr = threadIdx.x;  // 256 consumer threads, one row each
      if (rr < RC && i0 + rr < n) {
        float hh = cmb[rr].x, ll = cmb[rr].y;
#pragma unroll
        for (int w = 1; w < kWsWarps; ++w) df_add_pair(hh, ll, cmb[w * 256 + rr].x, cmb[w * 256 + rr].y);
        z[i0 + rr] = (r[i0 + rr] - ((double)hh + (double)ll)) * inv_lam;
      }
      if (!ws_consumer_sync(&cbar[1], ci & 1u, abort_flag, err)) break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) ws_drain(full, issued_s);
}

void ws_plan(WsPlan& plan, const float* L, int64_t n, int64_t k, int rows) {
  plan = WsPlan();
  if (!L || n < 4 || k < 1 || n % 4 != 0 || n > (int64_t(1) << 30) || k > (int64_t(1) << 30)) return;
  const int sms = num_sms();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(ws_gemv_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmemT) != cudaSuccess ||
        cudaFuncSetAttribute(ws_gemv_n_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmemN) !=
            cudaSuccess ||
        cudaFuncSetAttribute(ws_gemv_n_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmemN) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    attr = true;
  }
  // resident CTAs per SM (two by design; fewer if the shared-memory carve-out says so)
  int occ = 0, occ_t = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ws_gemv_n_kernel<2>, kWsThreads, kWsSmemN) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, ws_gemv_t_kernel, kWsThreads, kWsSmemT) != cudaSuccess) {
    (void)cudaGetLastError();
    occ = occ_t = 1;
  }
  const int64_t G = (int64_t)std::max(1, std::min(occ, occ_t)) * sms;
  // L u pass (and Schur sums): 256-row chunks (measured faster) once there is one per SM
  const int rc = rows == 128 || rows == 256 ? rows : (cdiv(n, 256) >= (int64_t)sms ? 256 : 128);
  plan.rc = rc;
  plan.nch = cdiv(n, rc);
  plan.grid = (int)std::min<int64_t>(plan.nch, G);
  // L^T r pass: row units of up to 1024 rows; column ranges fill the CTAs when the row units
  // alone do not; whole waves when they do
  const int64_t kg = cdiv(k, 64);  // 64-column groups
  int64_t ru = 1024;
  if (cdiv(n, 1024) >= G) {
    const int64_t waves = cdiv(cdiv(n, 1024), G);
    ru = 256 * cdiv(n, 256 * waves * G);
    ru = std::min<int64_t>(1024, std::max<int64_t>(256, ru));
  } else {
    for (int64_t cand : {1024, 512, 256}) {
      ru = cand;
      const int64_t nr = cdiv(n, cand);
      if (nr * std::min<int64_t>(kg, std::max<int64_t>(1, G / nr)) * 4 >= 3 * G) break;
    }
  }
  plan.ru = (int)ru;
  plan.nru = cdiv(n, ru);
  plan.ncr = (int)std::min<int64_t>(kg, std::max<int64_t>(1, G / plan.nru));
  plan.cpr = (int)(64 * cdiv(kg, plan.ncr));
  plan.ncr = (int)cdiv(k, plan.cpr);
  plan.grid_t = (int)std::min<int64_t>(plan.nru * plan.ncr, G);
  plan.L = L;
  plan.n = n;
  plan.k = k;
  if (!make_f32_map(&plan.map, L, (uint64_t)n, (uint64_t)k, (uint64_t)n, (uint32_t)rc, (uint32_t)(32 * 128 / rc)) ||
      !make_f32_map(&plan.mapT, L, (uint64_t)n, (uint64_t)k, (uint64_t)n, 256u, 16u))
    return;
  plan.ok = true;
}

static bool ws_usable(const WsPlan* plan, const float* L, int64_t n, int64_t k) {
  return plan && plan->ok && plan->L == L && plan->n == n && plan->k == k;
}

// Dense k x k products of the apply's core in double-float (DF64 contexts store C^-1
// and C as float pairs): one warp per row, 16-byte loads (two entries), each term
// (a_h + a_l)(x_h + x_l) formed by TwoProduct with the cross terms folded in, sums
// in double-float, fixed shuffle tree.
//   mode 0:  y = A x,       y2 = split(y)          (u = C^-1 t)
//   mode 1:  y2 = split(t - A x)                   (e = t - C u)
//   mode 2:  y += A x,      y2 = split(y)          (u += C^-1 e)
__device__ __forceinline__ void df_term(float& h, float& l, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, e);
  e = fmaf(al, xh, e);
  df_add_pair(h, l, p, e);
}

// One CTA (256 threads) per row i: every thread loads its share of the row and of x
// at once (16-byte loads when EVEN: k even, so rows and vectors start on 16-byte
// boundaries), so the 2000 CTAs keep the L2 busy; per-thread double-float partials
// are reduced by a fixed shuffle tree and then across the 8 warps in order.
template <bool EVEN>
__global__ void __launch_bounds__(256) symv_df_kernel(const float2* __restrict__ A, int64_t k,
                                                      const float2* __restrict__ x, int mode,
                                                      const double* __restrict__ t, double* __restrict__ y,
                                                      float2* __restrict__ y2) {
  __shared__ float2 red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = blockIdx.x;
  const float2* row = A + i * k;
  float h = 0.f, l = 0.f;
  if (EVEN) {
#pragma unroll 4
    for (int64_t j = 2 * (int64_t)threadIdx.x; j < k; j += 512) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(row + j));
      const float4 xv = __ldg(reinterpret_cast<const float4*>(x + j));
      df_term(h, l, a.x, a.y, xv.x, xv.y);
      df_term(h, l, a.z, a.w, xv.z, xv.w);
    }
  } else {
#pragma unroll 4
    for (int64_t j = threadIdx.x; j < k; j += 256) {
      const float2 a = row[j], xv = x[j];
      df_term(h, l, a.x, a.y, xv.x, xv.y);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add_pair(h, l, oh, ol);
  }
  if (lane == 0) red[warp] = make_float2(h, l);
  __syncthreads();
  if (threadIdx.x != 0) return;
  h = red[0].x;
  l = red[0].y;
#pragma unroll
  for (int w = 1; w < 8; ++w) df_add_pair(h, l, red[w].x, red[w].y);
  const double s = (double)h + (double)l;
  double v;
  if (mode == 0) {
    v = s;
    y[i] = v;
  } else if (mode == 1) {
    v = t[i] - s;
  } else {
    v = y[i] + s;
    y[i] = v;
  }
  const float vh = (float)v;
  y2[i] = make_float2(vh, (float)(v - (double)vh));
}

// The same products with one warp per row and x staged once per CTA in shared memory (k
// even, k <= kSymvRowsMaxK): 8 rows per CTA, each lane streams 16-byte pieces of its row
// (eight in flight; the k x k matrices stay in L2 between applies) against x from shared
// memory, then a fixed shuffle tree.
constexpr int kSymvRowsMaxK = 4096;

// 16-byte load marked evict-last in L2: the k x k matrices of the apply's core are re-read
// every apply and should outlive the matvec's operands in L2 (the L_k tiles are evict-first)
__device__ __forceinline__ float4 ld_evict_last(const float4* p, uint64_t policy) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(policy));
  return v;
}
// Row i of the product, by one warp (xs: the vector in shared memory, k even); the result as
// symv_df_kernel's modes: 0  y = A x;  1  y2 = t - A x;  2  y += A x (y2: float pairs of y)
__device__ __forceinline__ void symv_row_df(const float2* __restrict__ A, int64_t k, const float2* xs, int mode,
                                            const double* __restrict__ t, double* __restrict__ y,
                                            float2* __restrict__ y2, int64_t i, int lane) {
  const float4* row = reinterpret_cast<const float4*>(A + i * k);  // k even: 16-byte aligned rows
  const float4* xv4 = reinterpret_cast<const float4*>(xs);
  const int64_t nq = k / 2;  // float4 pieces per row (two entries each)
  // two independent double-float chains (even and odd entries of each piece) and the next
  // eight pieces' loads issued before the current eight are summed
  float h = 0.f, l = 0.f, h1 = 0.f, l1 = 0.f;
  uint64_t policy;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
  int64_t q = lane;
  float4 av[8];
  const bool full8 = q + 224 < nq;
  if (full8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) av[u] = ld_evict_last(row + q + 32 * u, policy);
  }
  while (q + 224 < nq) {
    float4 nv[8];
    const int64_t qn = q + 256;
    const bool more = qn + 224 < nq;
    if (more) {
#pragma unroll
      for (int u = 0; u < 8; ++u) nv[u] = ld_evict_last(row + qn + 32 * u, policy);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 xq = xv4[q + 32 * u];
      df_term(h, l, av[u].x, av[u].y, xq.x, xq.y);
      df_term(h1, l1, av[u].z, av[u].w, xq.z, xq.w);
    }
    q = qn;
    if (more) {
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = nv[u];
    }
  }
  for (; q < nq; q += 32) {
    const float4 a = ld_evict_last(row + q, policy), xq = xv4[q];
    df_term(h, l, a.x, a.y, xq.x, xq.y);
    df_term(h1, l1, a.z, a.w, xq.z, xq.w);
  }
  df_add_pair(h, l, h1, l1);
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add_pair(h, l, oh, ol);
  }
  if (lane != 0) return;
  const double s = (double)h + (double)l;
  double v;
  if (mode == 0) {
    v = s;
    y[i] = v;
  } else if (mode == 1) {
    v = t[i] - s;
  } else {
    v = y[i] + s;
    y[i] = v;
  }
  const float vh = (float)v;
  y2[i] = make_float2(vh, (float)(v - (double)vh));
}

__global__ void __launch_bounds__(256) symv_df_rows_kernel(const float2* __restrict__ A, int64_t k,
                                                           const float2* __restrict__ x, int mode,
                                                           const double* __restrict__ t, double* __restrict__ y,
                                                           float2* __restrict__ y2) {
  __shared__ __align__(16) float2 xs[kSymvRowsMaxK];
  for (int64_t j = threadIdx.x; j < k; j += 256) xs[j] = x[j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i < k) symv_row_df(A, k, xs, mode, t, y, y2, i, lane);
}

static void symv_df(const float2* A, int64_t k, const float2* x, int mode, const double* t, double* y, float2* y2,
                    cudaStream_t st) {
  if ((k & 1) == 0 && k <= kSymvRowsMaxK)
    { symv_df_rows_kernel<<<(unsigned)cdiv(k, 8), 256, 0, st>>>(A, k, x, mode, t, y, y2); count_launch(); }
  else if ((k & 1) == 0)
    { symv_df_kernel<true><<<(unsigned)k, 256, 0, st>>>(A, k, x, mode, t, y, y2); count_launch(); }
  else
    { symv_df_kernel<false><<<(unsigned)k, 256, 0, st>>>(A, k, x, mode, t, y, y2); count_launch(); }
}

// t[j] = sum of the chunk partials (as reduce_chunks_kernel), also split into t2[j]; PAIRS:
// the partials are double-float pairs (float2) rather than doubles
template <bool PAIRS>
__device__ __forceinline__ void reduce_row_df(const double* __restrict__ part, int64_t nchunks,
                                              double* __restrict__ t, float2* __restrict__ t2, int64_t j, int lane) {
  double s = 0.0;
  if (PAIRS) {
    const float2* pj = reinterpret_cast<const float2*>(part) + j * nchunks;
    for (int64_t c = lane; c < nchunks; c += 32) {
      const float2 v = pj[c];
      s += (double)v.x + (double)v.y;
    }
  } else {
    const double* pj = part + j * nchunks;
    for (int64_t c = lane; c < nchunks; c += 32) s += pj[c];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    t[j] = s;
    const float sh = (float)s;
    t2[j] = make_float2(sh, (float)(s - (double)sh));
  }
}

template <bool PAIRS>
__global__ void __launch_bounds__(256) reduce_chunks_df_kernel(const double* __restrict__ part, int64_t nchunks,
                                                               int64_t k, double* __restrict__ t,
                                                               float2* __restrict__ t2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 8 + warp;
  if (j < k) reduce_row_df<PAIRS>(part, nchunks, t, t2, j, lane);
}

// ---------------------------------------------------------------- fused Woodbury core
// The k-vector steps between the two passes over L in one cooperative launch (all CTAs resident):
//   t = sum of the L^T r chunk partials (float pairs); u = C^-1 t; e = t - C u; u += C^-1 e,
// each row by one warp with the arithmetic of reduce_row_df / symv_row_df (so the results are
// those of the separate launches), separated by a grid-wide barrier.  The barrier counts
// arrivals in bar[0]; every wait is bounded (g_wait_limit polls, then err is set and the CTA
// skips the rest), and the last CTA to leave resets bar[0] and bar[1] for the next launch.
constexpr int kCoreMaxK = 16384;  // the vector staged per CTA: k float pairs of shared memory

__device__ __forceinline__ bool core_grid_barrier(unsigned* bar, unsigned target, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    ok = 0;
    const uint32_t limit = tc::g_wait_limit;
    for (uint32_t it = 0; it < limit; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) {
        ok = 1;
        break;
      }
      __nanosleep(32);
    }
    if (!ok) atomicExch(err, tc::ERR_TIMEOUT_DONE);
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) woodbury_core_fused_kernel(const double* __restrict__ part, int64_t nchunks,
                                                                  int64_t k, const float2* __restrict__ Cinv,
                                                                  const float2* __restrict__ C, double* t,
                                                                  float2* t2, double* u, float2* u2, float2* e2,
                                                                  unsigned* bar, int* err) {
  extern __shared__ __align__(16) float2 xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * 8 + warp, nw = (int64_t)gridDim.x * 8;
  bool ok = true;
  // rows go to warps the same way in every phase, so t[i] and u[i] are re-read by the warp that
  // wrote them; the staged vectors come from every CTA and are read past L1 after the barrier
  for (int64_t j = gw; j < k; j += nw) reduce_row_df<true>(part, nchunks, t, t2, j, lane);
  ok = core_grid_barrier(bar, gridDim.x, err);
  if (ok) {  // u = C^-1 t
    for (int64_t j = threadIdx.x; j < k; j += 256) xs[j] = __ldcg(t2 + j);
    __syncthreads();
    for (int64_t i = gw; i < k; i += nw) symv_row_df(Cinv, k, xs, 0, t, u, u2, i, lane);
    ok = core_grid_barrier(bar, 2 * gridDim.x, err);
  }
  if (ok) {  // e = t - C u
    for (int64_t j = threadIdx.x; j < k; j += 256) xs[j] = __ldcg(u2 + j);
    __syncthreads();
    for (int64_t i = gw; i < k; i += nw) symv_row_df(C, k, xs, 1, t, nullptr, e2, i, lane);
    ok = core_grid_barrier(bar, 3 * gridDim.x, err);
  }
  if (ok) {  // u += C^-1 e
    for (int64_t j = threadIdx.x; j < k; j += 256) xs[j] = __ldcg(e2 + j);
    __syncthreads();
    for (int64_t i = gw; i < k; i += nw) symv_row_df(Cinv, k, xs, 2, t, u, u2, i, lane);
  }
  // the last CTA out resets the counters (no CTA reads them again in this launch)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(bar + 1, 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      bar[1] = 0u;
      __threadfence();
    }
  }
}

// t = L^T r (t2: its float pairs) from the float pairs rs of r
static void df_pass_t(const float* L, int64_t n, int64_t k, const float2* rs, double* part, double* t, float2* t2,
                      const WsPlan* plan, int* err, cudaStream_t st) {
  const unsigned gk = (unsigned)cdiv(k, 8);
  if (ws_usable(plan, L, n, k)) {
    { ws_gemv_t_kernel<<<plan->grid_t, kWsThreads, kWsSmemT, st>>>(plan->mapT, n, k, plan->ru, plan->nru, plan->ncr, plan->cpr, rs, reinterpret_cast<float2*>(part), err); count_launch(); }
    { reduce_chunks_df_kernel<true><<<gk, 256, 0, st>>>(part, plan->nru, k, t, t2); count_launch(); }
    return;
  }
  const int64_t nchunks = cdiv(n, kDfRows);
  dim3 g1((unsigned)cdiv(k, kDfTCols), (unsigned)nchunks);
  if (n % 4 == 0)
    { gemv_t_df_kernel<true><<<g1, 256, 0, st>>>(L, n, k, rs, part); count_launch(); }
  else
    { gemv_t_df_kernel<false><<<g1, 256, 0, st>>>(L, n, k, rs, part); count_launch(); }
  { reduce_chunks_df_kernel<false><<<gk, 256, 0, st>>>(part, nchunks, k, t, t2); count_launch(); }
}

// z = (r - L u) / lambda from the float pairs u2 of u; part: scratch of 16 n float pairs
static void df_pass_n(const float* L, int64_t n, int64_t k, const float2* u2, const double* r, double inv_lam,
                      double* z, double* part, const WsPlan* plan, int* err, cudaStream_t st) {
  if (ws_usable(plan, L, n, k)) {
    if (plan->rc == 256)
      { ws_gemv_n_kernel<2><<<plan->grid, kWsThreads, kWsSmemN, st>>>(plan->map, n, k, plan->nch, u2, r, inv_lam, z, err); count_launch(); }
    else
      { ws_gemv_n_kernel<1><<<plan->grid, kWsThreads, kWsSmemN, st>>>(plan->map, n, k, plan->nch, u2, r, inv_lam, z, err); count_launch(); }
    return;
  }
  float2* zp = reinterpret_cast<float2*>(part);
  dim3 g2((unsigned)cdiv(n, kDfRows), (unsigned)kDfNGroups);
  if (n % 4 == 0)
    { gemv_n_df_kernel<true><<<g2, 256, 0, st>>>(L, n, k, u2, zp); count_launch(); }
  else
    { gemv_n_df_kernel<false><<<g2, 256, 0, st>>>(L, n, k, u2, zp); count_launch(); }
  { gemv_n_df_finish_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(zp, n, r, inv_lam, z); count_launch(); }
}

// A trivial cooperative kernel, to learn once whether this driver accepts cooperative launches
// inside captured graphs (the PCG loop is one)
__global__ void coop_probe_kernel(int* x) {
  if (threadIdx.x == 0 && x) *x = 1;
}

bool coop_graph_capture_ok() {
  static int state = -1;
  if (state >= 0) return state == 1;
  state = 0;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int* none = nullptr;
    const bool launched = cudaLaunchKernelEx(&cfg, coop_probe_kernel, none) == cudaSuccess;
    ok = cudaStreamEndCapture(s, &g) == cudaSuccess && launched && g;
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (ex) cudaGraphExecDestroy(ex);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(s);
  (void)cudaGetLastError();
  state = ok ? 1 : 0;
  return ok;
}

// the fused core applies to the staged L^T r pass (float-pair partials), an even k that fits
// the staged vector, and a driver that captures cooperative launches
static bool core_fusable(const WsPlan* plan, const float* L, int64_t n, int64_t k, const unsigned* bar) {
  return bar && ws_usable(plan, L, n, k) && (k & 1) == 0 && k <= kCoreMaxK && coop_graph_capture_ok();
}

static void launch_core_fused(const double* part, int64_t nchunks, int64_t k, const float2* Ci2, const float2* C2,
                              double* t, float2* t2, double* u, float2* u2, float2* e2, unsigned* bar, int* err,
                              cudaStream_t st) {
  const size_t smem = (size_t)k * sizeof(float2);
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    cudaFuncSetAttribute(woodbury_core_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = smem;
  }
  // as many CTAs as can be resident at once (at most 4 per SM): the cooperative launch needs
  // them co-resident, and more warps keep more of each phase's row loads in flight
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, woodbury_core_fused_kernel, 256, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(num_sms() * std::min(per_sm, 4)));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute a;
  a.id = cudaLaunchAttributeCooperative;
  a.val.cooperative = 1;
  cfg.attrs = &a;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, woodbury_core_fused_kernel, part, nchunks, k, Ci2, C2, t, t2, u, u2, e2, bar, err);
  count_launch();
}

void woodbury_apply_df(const float* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                       const double* r, double* z, double* part, double* t, float2* rs, const WsPlan* plan,
                       int* err, unsigned* bar, cudaStream_t st) {
  double* u = t + k;
  float2* t2 = reinterpret_cast<float2*>(t + 3 * k);
  float2* e2 = reinterpret_cast<float2*>(t + 4 * k);
  float2* u2 = reinterpret_cast<float2*>(t + 5 * k);
  const float2* Ci2 = reinterpret_cast<const float2*>(Cinv);
  const float2* C2 = reinterpret_cast<const float2*>(C);
  { split_df_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(r, n, rs); count_launch(); }
  if (core_fusable(plan, L, n, k, bar)) {
    // L^T r partials, then the reduction and the three k x k products in one launch
    { ws_gemv_t_kernel<<<plan->grid_t, kWsThreads, kWsSmemT, st>>>(plan->mapT, n, k, plan->ru, plan->nru, plan->ncr, plan->cpr, rs, reinterpret_cast<float2*>(part), err); count_launch(); }
    launch_core_fused(part, plan->nru, k, Ci2, C2, t, t2, u, u2, e2, bar, err, st);
    df_pass_n(L, n, k, u2, r, 1.0 / lam, z, part, plan, err, st);
    return;
  }
  df_pass_t(L, n, k, rs, part, t, t2, plan, err, st);
  // u = C^-1 t, refined once with the residual t - C u (see woodbury_apply)
  symv_df(Ci2, k, t2, 0, t, u, u2, st);
  symv_df(C2, k, u2, 1, t, nullptr, e2, st);
  symv_df(Ci2, k, e2, 2, t, u, u2, st);
  // the chunk partials are dead: their buffer is the scratch of the register-streamed L u pass
  df_pass_n(L, n, k, u2, r, 1.0 / lam, z, part, plan, err, st);
}

void df_passes(const float* L, int64_t n, int64_t k, const double* r, const double* u, double lam, double* t,
               double* z, double* part, float2* rs, float2* t2, float2* u2, const WsPlan* plan, int* err,
               cudaStream_t st) {
  { split_df_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(r, n, rs); count_launch(); }
  df_pass_t(L, n, k, rs, part, t, t2, plan, err, st);
  { split_df_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(u, k, u2); count_launch(); }
  df_pass_n(L, n, k, u2, r, 1.0 / lam, z, part, plan, err, st);
}

// each double becomes the float pair (hi, lo) in the same 8 bytes
__global__ void split_df_inplace_kernel(double* a, int64_t count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = a[i];
  const float hi = (float)v;
  reinterpret_cast<float2*>(a)[i] = make_float2(hi, (float)(v - (double)hi));
}

// DF64 contexts keep C^-1 and C as float pairs (in place of the doubles)
void split_df_inplace(double* a, int64_t count, cudaStream_t st) {
  { split_df_inplace_kernel<<<(unsigned)cdiv(count, 256), 256, 0, st>>>(a, count); count_launch(); }
}

__global__ void to_float_kernel(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void widen_float_kernel(const float* __restrict__ a, int64_t n, double* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

void widen_float(const float* a, int64_t n, double* b, cudaStream_t st) {
  { widen_float_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(a, n, b); count_launch(); }
}

void to_float(const double* a, int64_t n, float* b, cudaStream_t st) {
  { to_float_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(a, n, b); count_launch(); }
}

cudaError_t set_wait_limit_wb(uint32_t polls) { return tc::set_wait_limit_here(polls); }

}  // namespace gdml
