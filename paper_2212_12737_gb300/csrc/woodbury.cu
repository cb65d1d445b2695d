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

// part[chunk * k + j] = sum_{i in chunk} L[i + j n] r[i]; one warp per column.
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
  if (lane == 0) part[blockIdx.y * k + j] = s;
}

// t[j] = sum over chunks (fixed order)
__global__ void reduce_chunks_kernel(const double* __restrict__ part, int64_t nchunks, int64_t k,
                                     double* __restrict__ t) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int64_t c = 0; c < nchunks; ++c) s += part[c * k + j];
  t[j] = s;
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
  { reduce_chunks_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(part, nchunks, k, t); count_launch(); }
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

int64_t woodbury_part_size(int64_t n, int64_t k) { return cdiv(n, kRowsPerChunk) * k; }

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

__global__ void __launch_bounds__(256) gemv_t_df_kernel(const float* __restrict__ L, int64_t n, int64_t k,
                                                        const float2* __restrict__ rs, double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kColsPerCta + warp;
  const int64_t i0 = (int64_t)blockIdx.y * kRowsPerChunk;
  const int64_t i1 = i0 + kRowsPerChunk < n ? i0 + kRowsPerChunk : n;
  if (j >= k) return;
  const float* col = L + j * n;
  float sh = 0.f, sl = 0.f;
#pragma unroll 4
  for (int64_t i = i0 + lane; i < i1; i += 32) {
    const float2 ri = rs[i];
    df_add_prod(sh, sl, col[i], ri.x, ri.y);
  }
  double s = (double)sh + (double)sl;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[blockIdx.y * k + j] = s;
}

__global__ void __launch_bounds__(256) gemv_n_df_kernel(const float* __restrict__ L, int64_t n, int64_t k,
                                                        const double* __restrict__ x, const double* __restrict__ r,
                                                        double inv_lam, double* __restrict__ z) {
  __shared__ float2 xs[2048];
  __shared__ double part[4][64];
  const int rr = threadIdx.x & 63, q = threadIdx.x >> 6;
  const int64_t i = (int64_t)blockIdx.x * 64 + rr;
  float sh = 0.f, sl = 0.f;
  for (int64_t j0 = 0; j0 < k; j0 += 2048) {
    const int64_t jn = (k - j0) < 2048 ? (k - j0) : 2048;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < jn; t += blockDim.x) {
      const double xv = x[j0 + t];
      const float hi = (float)xv;
      xs[t] = make_float2(hi, (float)(xv - (double)hi));
    }
    __syncthreads();
    if (i < n) {
      const int64_t qa = (jn * q) / 4, qb = (jn * (q + 1)) / 4;
      const float* Lc = L + j0 * n + i;
#pragma unroll 4
      for (int64_t j = qa; j < qb; ++j) df_add_prod(sh, sl, Lc[j * n], xs[j].x, xs[j].y);
    }
  }
  part[q][rr] = (double)sh + (double)sl;
  __syncthreads();
  if (q == 0 && i < n) z[i] = (r[i] - ((part[0][rr] + part[1][rr]) + (part[2][rr] + part[3][rr]))) * inv_lam;
}

void woodbury_apply_df(const float* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                       const double* r, double* z, double* part, double* t, float2* rs, cudaStream_t st) {
  const int64_t nchunks = cdiv(n, kRowsPerChunk);
  dim3 g1((unsigned)cdiv(k, kColsPerCta), (unsigned)nchunks);
  double* u = t + k;
  double* e = t + 2 * k;
  const unsigned gk = (unsigned)cdiv(k, 8);
  { split_df_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(r, n, rs); count_launch(); }
  { gemv_t_df_kernel<<<g1, 256, 0, st>>>(L, n, k, rs, part); count_launch(); }
  { reduce_chunks_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(part, nchunks, k, t); count_launch(); }
  { symv_kernel<<<gk, 256, 0, st>>>(Cinv, k, t, u); count_launch(); }
  { residual_kernel<<<gk, 256, 0, st>>>(C, k, t, u, e); count_launch(); }
  { symv_add_kernel<<<gk, 256, 0, st>>>(Cinv, k, e, u); count_launch(); }
  { gemv_n_df_kernel<<<(unsigned)cdiv(n, 64), 256, 0, st>>>(L, n, k, u, r, 1.0 / lam, z); count_launch(); }
}

__global__ void to_float_kernel(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

void to_float(const double* a, int64_t n, float* b, cudaStream_t st) {
  { to_float_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(a, n, b); count_launch(); }
}

}  // namespace gdml
