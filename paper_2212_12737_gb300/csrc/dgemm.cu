// FP64 SIMT GEMM (DFMA) for the FP64 form of the matvec contractions, the
// Woodbury core C = lambda I + L_k^T L_k (Eq. 4) and the blocked Cholesky /
// triangular-solve updates.
//
//   C[m, n] = alpha * sum_k A[m, k] * Bop[k, n] + beta * C[m, n]
//   A row-major (lda); Bop[k, n] = B[n*ldb + k] (NT) or B[k*ldb + n] (NN).
//   Operands may be stored as float (products are then exact in FP64).
//   lower_only: tiles strictly above the diagonal are skipped (SYRK-style).
//   split-K: grid.z splits of kchunk each; split z writes its partial product to
//   C + z * split_stride (beta must be 0), and the consumer sums them in order.
//
// 64x64 output tile per CTA, 256 threads x (4x4) outputs, K-steps of 16
// staged through shared memory with a register prefetch of the next step.
#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

template <typename TA, typename TB, bool NT>
__global__ void __launch_bounds__(256) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                    const TA* __restrict__ A, int64_t lda,
                                                    const TB* __restrict__ B, int64_t ldb, double beta,
                                                    double* __restrict__ C, int64_t ldc, int lower_only,
                                                    int64_t kchunk, int64_t split_stride) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  if (lower_only && n0 > m0 + BM - 1) return;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  C += (int64_t)blockIdx.z * split_stride;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  // loader mapping: 256 threads load 64x16 = 1024 elements of each tile (4 each)
  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u;          // 0..1023
      int am = e >> 4, ak = e & 15;   // A tile: row am, col ak  (k fastest -> coalesced rows)
      int64_t gm = m0 + am, gk = k0 + ak;
      ra[u] = (gm < M && gk < kend) ? (double)A[gm * lda + gk] : 0.0;
      if (NT) {
        int bn = e >> 4, bk = e & 15;
        int64_t gn = n0 + bn, gk2 = k0 + bk;
        rb[u] = (gn < N && gk2 < kend) ? (double)B[gn * ldb + gk2] : 0.0;
      } else {
        int bk = e >> 6, bn = e & 63;  // n fastest -> coalesced
        int64_t gn = n0 + bn, gk2 = k0 + bk;
        rb[u] = (gn < N && gk2 < kend) ? (double)B[gk2 * ldb + gn] : 0.0;
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u;
      As[e & 15][e >> 4] = ra[u];
      if (NT) Bs[e & 15][e >> 4] = rb[u];
      else Bs[e >> 6][e & 63] = rb[u];
    }
  };
  load(kbeg);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < kend) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double* c = C + gm * ldc + gn;
      *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
    }
  }
}

template <typename TA, typename TB>
void launch_dgemm(bool nt, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t lda,
                  const TB* B, int64_t ldb, double beta, double* C, int64_t ldc, bool lower_only,
                  cudaStream_t st, int splits, int64_t split_stride) {
  if (M <= 0 || N <= 0) return;
  if (splits < 1) splits = 1;
  const int64_t kchunk = cdiv(cdiv(K, splits), 16) * 16;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), (unsigned)splits);
  if (nt)
    { dgemm_kernel<TA, TB, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only,
                                                      kchunk, split_stride); count_launch(); }
  else
    { dgemm_kernel<TA, TB, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only,
                                                       kchunk, split_stride); count_launch(); }
}

// number of K splits that brings an M x N tile grid to ~2 waves of the SMs
int dgemm_splits(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = cdiv(M, 64) * cdiv(N, 64);
  int64_t s = (2 * (int64_t)num_sms()) / (tiles > 0 ? tiles : 1);
  const int64_t kmax = cdiv(K, 64);  // keep >= 64 of K per split
  if (s > kmax) s = kmax;
  return (int)(s < 1 ? 1 : s);
}

// ---------------------------------------------------------------------------
// Double-float GEMM on the FP32 lanes: the same contraction as dgemm_kernel,
// FP64 in and out, but each operand is split into a pair of floats
// (hi = fl32(x), lo = fl32(x - hi)), each product is formed exactly with an
// FMA (TwoProduct) plus the two cross terms, and the running sums are
// (hi, lo) pairs updated with TwoSum.  About 15 FP32 operations per
// multiply-add and ~2^-46 relative error per term: FP64-class results at the
// FP32 lane rate, which on GB300 is ~60x the FP64 rate.
__device__ __forceinline__ float2 split_df(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

template <bool NT>
__global__ void __launch_bounds__(256) dfgemm_kernel(int64_t M, int64_t N, int64_t K, const double* __restrict__ A,
                                                     int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                     double* __restrict__ C, int64_t ldc, int64_t kchunk,
                                                     int64_t split_stride) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  C += (int64_t)blockIdx.z * split_stride;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int am = e >> 4, ak = e & 15;
      const int64_t gm = m0 + am, gk = k0 + ak;
      As[ak][am] = split_df((gm < M && gk < kend) ? A[gm * lda + gk] : 0.0);
      if (NT) {
        const int64_t gn = n0 + am;
        Bs[ak][am] = split_df((gn < N && gk < kend) ? B[gn * ldb + gk] : 0.0);
      } else {
        const int bk = e >> 6, bn = e & 63;
        const int64_t gn = n0 + bn, gk2 = k0 + bk;
        Bs[bk][bn] = split_df((gn < N && gk2 < kend) ? B[gk2 * ldb + gn] : 0.0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float ph = a[i].x * b[j].x;
          float pl = fmaf(a[i].x, b[j].x, -ph);  // exact low part of hi * hi
          pl = fmaf(a[i].x, b[j].y, pl);
          pl = fmaf(a[i].y, b[j].x, pl);
          const float t = sh[i][j] + ph;  // TwoSum(sh, ph)
          const float v = t - sh[i][j];
          float e = (sh[i][j] - (t - v)) + (ph - v);
          e += sl[i][j] + pl;
          const float hi = t + e;  // renormalise
          sl[i][j] = e - (hi - t);
          sh[i][j] = hi;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn < N) C[gm * ldc + gn] = (double)sh[i][j] + (double)sl[i][j];
    }
  }
}

void launch_dfgemm(bool nt, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double* C, int64_t ldc, cudaStream_t st, int splits, int64_t split_stride) {
  if (M <= 0 || N <= 0) return;
  if (splits < 1) splits = 1;
  const int64_t kchunk = cdiv(cdiv(K, splits), 16) * 16;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), (unsigned)splits);
  if (nt)
    { dfgemm_kernel<true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk, split_stride); count_launch(); }
  else
    { dfgemm_kernel<false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk, split_stride); count_launch(); }
}

// C = A A^T (lower tiles only), A: k x n row-major FP32, in double-float:
// products of two floats are exact as (hi, lo) pairs, sums by TwoSum.
__global__ void __launch_bounds__(256) dfsyrk_kernel(int64_t k, int64_t n, const float* __restrict__ A, int64_t lda,
                                                     double* __restrict__ C, int64_t ldc) {
  __shared__ float As[16][65], Bs[16][65];
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  if (n0 > m0 + 63) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int64_t k0 = 0; k0 < n; k0 += 16) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int r = e >> 4, kk = e & 15;
      const int64_t gk = k0 + kk;
      As[kk][r] = (m0 + r < k && gk < n) ? A[(m0 + r) * lda + gk] : 0.f;
      Bs[kk][r] = (n0 + r < k && gk < n) ? A[(n0 + r) * lda + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_add_prod(sh[i][j], sl[i][j], a[i], b[j], 0.f);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < k && gn < k) C[gm * ldc + gn] = (double)sh[i][j] + (double)sl[i][j];
    }
}

void launch_dfsyrk(int64_t k, int64_t n, const float* A, int64_t lda, double* C, int64_t ldc, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(k, 64), (unsigned)cdiv(k, 64));
  { dfsyrk_kernel<<<grid, 256, 0, st>>>(k, n, A, lda, C, ldc); count_launch(); }
}

template void launch_dgemm<double, double>(bool, int64_t, int64_t, int64_t, double, const double*, int64_t,
                                           const double*, int64_t, double, double*, int64_t, bool, cudaStream_t,
                                           int, int64_t);
template void launch_dgemm<float, float>(bool, int64_t, int64_t, int64_t, double, const float*, int64_t,
                                         const float*, int64_t, double, double*, int64_t, bool, cudaStream_t, int,
                                         int64_t);

}  // namespace gdml
