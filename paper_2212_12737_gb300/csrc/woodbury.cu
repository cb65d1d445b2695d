// Woodbury apply of the Nystrom preconditioner (Eq. 4):
//   z = lambda^-1 [ r - L_k C^-1 L_k^T r ],  C = lambda I + L_k^T L_k = L_C L_C^T.
// L_k is stored column-major (n x k, column j at L + j*n) in FP64, or in FP32
// for the mixed-precision contexts; all arithmetic is FP64 (FP32 x FP64
// products are formed in FP64).  Two HBM passes over L_k per apply.
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

// z[i] = (r[i] - sum_j L[i + j n] x[j]) / lambda  (x staged through shared memory)
template <typename TL>
__global__ void __launch_bounds__(256) gemv_n_update_kernel(const TL* __restrict__ L, int64_t n, int64_t k,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ r, double inv_lam,
                                                            double* __restrict__ z) {
  __shared__ double xs[2048];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t j0 = 0; j0 < k; j0 += 2048) {
    const int64_t jn = (k - j0) < 2048 ? (k - j0) : 2048;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < jn; t += blockDim.x) xs[t] = x[j0 + t];
    __syncthreads();
    if (i < n) {
      const TL* Lc = L + j0 * n + i;
      int64_t j = 0;
      for (; j + 1 < jn; j += 2) {
        s0 = fma((double)Lc[j * n], xs[j], s0);
        s1 = fma((double)Lc[(j + 1) * n], xs[j + 1], s1);
      }
      if (j < jn) s0 = fma((double)Lc[j * n], xs[j], s0);
    }
  }
  if (i < n) z[i] = (r[i] - (s0 + s1)) * inv_lam;
}

template <typename TL>
void woodbury_apply(const TL* L, int64_t n, int64_t k, const double* LC, double lam, const double* r,
                    double* z, double* part, double* t, TrsvState& ts, cudaStream_t st) {
  const int64_t nchunks = cdiv(n, kRowsPerChunk);
  dim3 g1((unsigned)cdiv(k, kColsPerCta), (unsigned)nchunks);
  { gemv_t_partial_kernel<TL><<<g1, 256, 0, st>>>(L, n, k, r, part); count_launch(); }
  { reduce_chunks_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(part, nchunks, k, t); count_launch(); }
  trsv_lower(LC, k, t, false, ts, st);
  trsv_lower(LC, k, t, true, ts, st);
  { gemv_n_update_kernel<TL><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(L, n, k, t, r, 1.0 / lam, z); count_launch(); }
}

template void woodbury_apply<double>(const double*, int64_t, int64_t, const double*, double, const double*,
                                     double*, double*, double*, TrsvState&, cudaStream_t);
template void woodbury_apply<float>(const float*, int64_t, int64_t, const double*, double, const double*,
                                    double*, double*, double*, TrsvState&, cudaStream_t);

int64_t woodbury_part_size(int64_t n, int64_t k) { return cdiv(n, kRowsPerChunk) * k; }

}  // namespace gdml
