// Woodbury apply of the Nystrom preconditioner (Eq. 4):
//   z = lambda^-1 [ r - L_k C^-1 L_k^T r ],  C = lambda I + L_k^T L_k.
// C^-1 is formed once per build from the FP64 Cholesky factor of C
// (C^-1 = L_C^-T L_C^-1), so the apply is three data-parallel passes:
//   t = L_k^T r,  u = C^-1 t (+ one refinement step),  z = (r - L_k u) / lambda
// instead of two latency-bound triangular solves per CG iteration.  L_k is
// stored column-major (n x k, column j at L + j*n) in FP64, or in FP32 for the
// mixed-precision contexts; all arithmetic is FP64.  Two HBM passes over L_k.
#include "common.cuh"
#include "kernels.cuh"

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
  const int64_t a = cdiv(n, 512) * k, b = 16 * n;
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

static void symv_df(const float2* A, int64_t k, const float2* x, int mode, const double* t, double* y, float2* y2,
                    cudaStream_t st) {
  if ((k & 1) == 0)
    { symv_df_kernel<true><<<(unsigned)k, 256, 0, st>>>(A, k, x, mode, t, y, y2); count_launch(); }
  else
    { symv_df_kernel<false><<<(unsigned)k, 256, 0, st>>>(A, k, x, mode, t, y, y2); count_launch(); }
}

// t[j] = sum of the chunk partials (as reduce_chunks_kernel), also split into t2[j]
__global__ void __launch_bounds__(256) reduce_chunks_df_kernel(const double* __restrict__ part, int64_t nchunks,
                                                               int64_t k, double* __restrict__ t,
                                                               float2* __restrict__ t2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 8 + warp;
  if (j >= k) return;
  const double* pj = part + j * nchunks;
  double s = 0.0;
  for (int64_t c = lane; c < nchunks; c += 32) s += pj[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    t[j] = s;
    const float sh = (float)s;
    t2[j] = make_float2(sh, (float)(s - (double)sh));
  }
}

void woodbury_apply_df(const float* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                       const double* r, double* z, double* part, double* t, float2* rs, cudaStream_t st) {
  const int64_t nchunks = cdiv(n, kDfRows);
  dim3 g1((unsigned)cdiv(k, kDfTCols), (unsigned)nchunks);
  double* u = t + k;
  float2* t2 = reinterpret_cast<float2*>(t + 3 * k);
  float2* e2 = reinterpret_cast<float2*>(t + 4 * k);
  float2* u2 = reinterpret_cast<float2*>(t + 5 * k);
  const float2* Ci2 = reinterpret_cast<const float2*>(Cinv);
  const float2* C2 = reinterpret_cast<const float2*>(C);
  const unsigned gk = (unsigned)cdiv(k, 8);
  const bool vec = (n % 4) == 0;
  { split_df_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(r, n, rs); count_launch(); }
  if (vec)
    { gemv_t_df_kernel<true><<<g1, 256, 0, st>>>(L, n, k, rs, part); count_launch(); }
  else
    { gemv_t_df_kernel<false><<<g1, 256, 0, st>>>(L, n, k, rs, part); count_launch(); }
  { reduce_chunks_df_kernel<<<gk, 256, 0, st>>>(part, nchunks, k, t, t2); count_launch(); }
  // u = C^-1 t, refined once with the residual t - C u (see woodbury_apply)
  symv_df(Ci2, k, t2, 0, t, u, u2, st);
  symv_df(C2, k, u2, 1, t, nullptr, e2, st);
  symv_df(Ci2, k, e2, 2, t, u, u2, st);
  // the chunk partials are dead: their buffer takes the column-group partials of L u
  float2* zp = reinterpret_cast<float2*>(part);
  dim3 g2((unsigned)nchunks, (unsigned)kDfNGroups);
  if (vec)
    { gemv_n_df_kernel<true><<<g2, 256, 0, st>>>(L, n, k, u2, zp); count_launch(); }
  else
    { gemv_n_df_kernel<false><<<g2, 256, 0, st>>>(L, n, k, u2, zp); count_launch(); }
  { gemv_n_df_finish_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(zp, n, r, 1.0 / lam, z); count_launch(); }
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

void to_float(const double* a, int64_t n, float* b, cudaStream_t st) {
  { to_float_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(a, n, b); count_launch(); }
}

}  // namespace gdml
