// Geometry-side kernels of the force-kernel matvec (Sec. 2.1), FP64.
//
//  desc_jac   x_{a,p} = 1/|R_i - R_j|,  g_{a,p} = (R_i - R_j)/|R_i - R_j|^3  (p <-> (i, j), i > j)
//  center     xc_a = x_a - mean_b x_b   (the kernel only sees differences x_a - x_b,
//             so centring is exact and keeps the low-precision contractions small)
//  dist_tab   r_ab = |x_a - x_b|, S_ab = (c^2/3) e^{-c r_ab}, A_ab = S_ab (1 + c r_ab)
//  kdiag      diag(K)_{a,(i,q)} = (c^2/3) sum_{p owns i} g_{a,p,q}^2   (K_aa = (c^2/3) J_a^T J_a)
//  proj       w_a = J_a v_a:  w_{a,p} = -g_{a,p} . (v_{a,i} - v_{a,j});  t_a = xc_a . w_a
//  beta       beta_ab = c^2 S_ab (T_ab - t_b), T = Xc W^T; rowsum_a = sum_b beta_ab
//  backproj   (K v)_a = J_a^T u'_a with u'_a = U_a - rowsum_a xc_a, plus lambda v
//  kcol       columns K[:, c] = J_a^T H_ab J_b e_l for a list of column indices c = b*3N + l
//  dist_tab_cross, center_like   the same tables for query geometries against the training
//             set, and query descriptors centred on the training centre (force prediction)
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

__global__ void desc_jac_kernel(const double* __restrict__ R, int64_t M, int N, int D,
                                double* __restrict__ X, double* __restrict__ G) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M * D) return;
  int64_t a = t / D;
  int p = (int)(t - a * D);
  int i, j;
  pair_of(p, i, j);
  const double* Ra = R + a * N * 3;
  double dx = Ra[3 * i] - Ra[3 * j], dy = Ra[3 * i + 1] - Ra[3 * j + 1], dz = Ra[3 * i + 2] - Ra[3 * j + 2];
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  double inv_r = 1.0 / r;
  double inv_r3 = inv_r / r2;
  X[t] = inv_r;
  G[3 * t] = dx * inv_r3;
  G[3 * t + 1] = dy * inv_r3;
  G[3 * t + 2] = dz * inv_r3;
}

// column means of X in a fixed order, then Xc = X - mean
__global__ void center_kernel(const double* __restrict__ X, int64_t M, int D, double* __restrict__ Xc) {
  __shared__ double part[8][33];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int row0 = threadIdx.x >> 5;  // 0..7
  double s = 0.0;
  if (col < D)
    for (int64_t a = row0; a < M; a += 8) s += X[a * D + col];
  part[row0][threadIdx.x & 31] = s;
  __syncthreads();
  double mean = 0.0;
  for (int r = 0; r < 8; ++r) mean += part[r][threadIdx.x & 31];
  mean /= (double)M;
  if (col < D)
    for (int64_t a = row0; a < M; a += 8) Xc[a * D + col] = X[a * D + col] - mean;
}

// r_ab straight from differences (no Gram-matrix cancellation); S and A tables.
// 32x32 output tile per CTA, 256 threads, 4 outputs per thread.
__global__ void dist_tab_kernel(const double* __restrict__ X, int64_t M, int D, double c,
                                double* __restrict__ S, double* __restrict__ A, int64_t ldA) {
  __shared__ double xa[32][33], xb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7
  const int64_t a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  double acc[4] = {0, 0, 0, 0};
  for (int p0 = 0; p0 < D; p0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      int64_t ra = a0 + rr, rb = b0 + rr;
      int p = p0 + tx;
      xa[rr][tx] = (ra < M && p < D) ? X[ra * D + p] : 0.0;
      xb[rr][tx] = (rb < M && p < D) ? X[rb * D + p] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 32; ++q) {
      double vb = xb[tx][q];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        double d = xa[ty + 8 * u][q] - vb;
        acc[u] = fma(d, d, acc[u]);
      }
    }
    __syncthreads();
  }
  const double c2_3 = c * c / 3.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t a = a0 + ty + 8 * u, b = b0 + tx;
    if (a < M && b < M) {
      double r = (a == b) ? 0.0 : sqrt(acc[u]);
      double s = c2_3 * exp(-c * r);
      S[a * M + b] = s;
      A[a * ldA + b] = s * (1.0 + c * r);
    }
  }
}

// S_qb, A_qb from r_qb = |x_q - x_b| for query rows x_q against training rows x_b, tiled as
// dist_tab_kernel (32 x 32 outputs per CTA); S has row stride M, A row stride ldA.
__global__ void dist_tab_cross_kernel(const double* __restrict__ Xq, int64_t Q, const double* __restrict__ X,
                                      int64_t M, int D, double c, double* __restrict__ S, double* __restrict__ A,
                                      int64_t ldA) {
  __shared__ double xa[32][33], xb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7
  const int64_t a0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
  double acc[4] = {0, 0, 0, 0};
  for (int p0 = 0; p0 < D; p0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t ra = a0 + rr, rb = b0 + rr;
      const int p = p0 + tx;
      xa[rr][tx] = (ra < Q && p < D) ? Xq[ra * D + p] : 0.0;
      xb[rr][tx] = (rb < M && p < D) ? X[rb * D + p] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 32; ++q) {
      const double vb = xb[tx][q];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double d = xa[ty + 8 * u][q] - vb;
        acc[u] = fma(d, d, acc[u]);
      }
    }
    __syncthreads();
  }
  const double c2_3 = c * c / 3.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t a = a0 + ty + 8 * u, b = b0 + tx;
    if (a < Q && b < M) {
      const double r = sqrt(acc[u]);
      const double s = c2_3 * exp(-c * r);
      S[a * M + b] = s;
      A[a * ldA + b] = s * (1.0 + c * r);
    }
  }
}

// Xqc = Xq - mu, mu = X_0 - Xc_0: query descriptors centred on the training set's centre,
// so that (xq - mu) . w_b - xc_b . w_b = (x_q - x_b) . w_b
__global__ void center_like_kernel(const double* __restrict__ Xq, int64_t Q, int D, const double* __restrict__ X,
                                   const double* __restrict__ Xc, double* __restrict__ Xqc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Q * D) return;
  const int p = (int)(t % D);
  Xqc[t] = Xq[t] - (X[p] - Xc[p]);
}

__global__ void kdiag_kernel(const double* __restrict__ G, int64_t M, int N, int D, double c2_3,
                             double* __restrict__ diag) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int B = 3 * N;
  if (t >= M * B) return;
  int64_t a = t / B;
  int l = (int)(t - a * B), i = l / 3, q = l - 3 * (l / 3);
  const double* Ga = G + a * D * 3;
  double s = 0.0;
  // branch-free so that the loads of successive j are independent and in flight together
#pragma unroll 4
  for (int j = 0; j < N; ++j) {
    const bool skip = j == i;
    const double gl = Ga[3 * (skip ? 0 : pair_idx(i, j)) + q];  // always a valid address
    const double g = skip ? 0.0 : gl;
    s = fma(g, g, s);
  }
  diag[t] = c2_3 * s;
}

// W_a = J_a v_a and t_a = xc_a . w_a; one CTA per geometry, one descriptor p per thread (a
// second round when D exceeds the block): the G loads are issued before v_a is staged, the
// pair (i, j) of p decoded in FP32, and t_a reduced in a fixed order (shuffle tree, then warps).
__global__ void __launch_bounds__(1024) proj_cta_kernel(const double* __restrict__ G, const double* __restrict__ Xc,
                                                        const double* __restrict__ v, int64_t M, int N, int D,
                                                        double* __restrict__ W, int64_t ldW, double* __restrict__ t) {
  extern __shared__ double sv[];  // 3N
  __shared__ double red[32];
  const int64_t a = blockIdx.x;
  const int B = 3 * N;
  const double* Ga = G + a * D * 3;
  int p = threadIdx.x;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, xc = 0.0;
  if (p < D) {
    g0 = Ga[3 * p];
    g1 = Ga[3 * p + 1];
    g2 = Ga[3 * p + 2];
    xc = Xc[a * D + p];
  }
  for (int l = threadIdx.x; l < B; l += blockDim.x) sv[l] = v[a * B + l];
  __syncthreads();
  double part = 0.0;
  for (; p < D; p += blockDim.x) {
    if (p >= (int)blockDim.x) {  // later rounds (D > blockDim)
      g0 = Ga[3 * p];
      g1 = Ga[3 * p + 1];
      g2 = Ga[3 * p + 2];
      xc = Xc[a * D + p];
    }
    int i, j;
    pair_of(p, i, j);
    const double w = -(g0 * (sv[3 * i] - sv[3 * j]) + g1 * (sv[3 * i + 1] - sv[3 * j + 1]) +
                       g2 * (sv[3 * i + 2] - sv[3 * j + 2]));
    W[a * ldW + p] = w;
    part = fma(xc, w, part);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    t[a] = s;
  }
}

// beta_ab = c^2 S_ab (T_ab - t_b) into Pb[a*ldP + b]; rowsum_a = sum_b beta_ab
template <int THREADS>
__global__ void beta_kernel(const double* __restrict__ T, const double* __restrict__ S,
                            const double* __restrict__ t, int64_t M, double c2,
                            double* __restrict__ Pb, int64_t ldP, double* __restrict__ rowsum) {
  __shared__ double red[THREADS / 32];
  const int64_t a = blockIdx.x;
  double part = 0.0;
  for (int64_t b = threadIdx.x; b < M; b += THREADS) {
    double beta = c2 * S[a * M + b] * (T[a * M + b] - t[b]);
    Pb[a * ldP + b] = beta;
    part += beta;
  }
  double s = block_sum<THREADS>(part, red);
  if (threadIdx.x == 0) rowsum[a] = s;
}

// (K v)_a = J_a^T (U_a - rowsum_a xc_a) (+ lambda v_a). One CTA per geometry.
template <typename TU>
__global__ void backproj_kernel(const TU* __restrict__ U, int64_t ldU, int splits, int64_t split_stride,
                                const double* __restrict__ rowsum,
                                const double* __restrict__ Xc, const double* __restrict__ G,
                                const double* __restrict__ v, int N, int D, double lam, int add_lambda,
                                double* __restrict__ out) {
  extern __shared__ double sh_u[];  // D
  const int64_t a = blockIdx.x;
  const double rs = rowsum[a];
  for (int p = threadIdx.x; p < D; p += blockDim.x) {
    double u = 0.0;
    for (int s = 0; s < splits; ++s) u += (double)U[s * split_stride + a * ldU + p];
    sh_u[p] = u - rs * Xc[a * D + p];
  }
  __syncthreads();
  const int B = 3 * N;
  const double* Ga = G + a * D * 3;
  for (int l = threadIdx.x; l < B; l += blockDim.x) {
    int i = l / 3, q = l - 3 * i;
    double s = 0.0;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {  // branch-free: independent loads of successive j
      const bool skip = j == i;
      const int p = skip ? 0 : pair_idx(i, j);
      const double gj = Ga[3 * p + q] * sh_u[p];
      s += skip ? 0.0 : ((i > j) ? -gj : gj);  // dx_p/dR_i = -g_p if i is the first atom of p, else +g_p
    }
    if (add_lambda) s = fma(lam, v[a * B + l], s);
    out[a * B + l] = s;
  }
}

// Columns of K: out[c*n + a*3N + l'] = (J_a^T H_ab J_b e_l)_{l'} for cols[c] = b*3N + l.
// grid (M, ceil(ncols/colsPerCta)); CTA handles target geometry a for several columns.
__global__ void kcol_kernel(const int64_t* __restrict__ cols, int64_t ncols, int colsPerCta,
                            const double* __restrict__ X, const double* __restrict__ G,
                            const double* __restrict__ S, const double* __restrict__ A, int64_t ldA,
                            int64_t M, int N, int D, double c2, double* __restrict__ out, int64_t ldo,
                            const int* __restrict__ stop_flag) {
  if (stop_flag && *stop_flag) return;
  extern __shared__ double sh[];
  double* delta = sh;       // D
  double* u = sh + D;       // D
  double* wsp = sh + 2 * D; // N (w on the pairs (i, j), indexed by partner j)
  __shared__ double s_dot;
  const int64_t a = blockIdx.x;
  const int B = 3 * N;
  const double* Xa = X + a * D;
  const double* Ga = G + a * D * 3;
  int64_t c_begin = (int64_t)blockIdx.y * colsPerCta;
  int64_t c_end = c_begin + colsPerCta < ncols ? c_begin + colsPerCta : ncols;
  int64_t last_b = -1;
  for (int64_t c = c_begin; c < c_end; ++c) {
    const int64_t col = cols[c];
    const int64_t b = col / B;
    const int l = (int)(col - b * B), i = l / 3, q = l - 3 * i;
    const double* Xb = X + b * D;
    const double* Gb = G + b * D * 3;
    __syncthreads();
    if (b != last_b) {
      for (int p = threadIdx.x; p < D; p += blockDim.x) delta[p] = Xa[p] - Xb[p];
      last_b = b;
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double w = 0.0;
      if (j != i) {
        int p = pair_idx(i, j);
        w = (i > j) ? -Gb[3 * p + q] : Gb[3 * p + q];  // (J_b e_l)_p
      }
      wsp[j] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int j = 0; j < N; ++j)
        if (j != i) s = fma(delta[pair_idx(i, j)], wsp[j], s);
      s_dot = s;
    }
    __syncthreads();
    const double Sab = S[a * M + b], Aab = A[a * ldA + b];
    const double coef = -c2 * Sab * s_dot;
    for (int p = threadIdx.x; p < D; p += blockDim.x) u[p] = coef * delta[p];
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      if (j != i) u[pair_idx(i, j)] += Aab * wsp[j];
    __syncthreads();
    for (int l2 = threadIdx.x; l2 < B; l2 += blockDim.x) {
      int i2 = l2 / 3, q2 = l2 - 3 * i2;
      double s = 0.0;
#pragma unroll 4
      for (int j = 0; j < N; ++j) {
        const bool skip = j == i2;
        const int p = skip ? 0 : pair_idx(i2, j);
        const double gj = Ga[3 * p + q2] * u[p];
        s += skip ? 0.0 : ((i2 > j) ? -gj : gj);
      }
      out[c * ldo + a * B + l2] = s;
    }
  }
}

// Same columns, one warp per geometry a (W warps per CTA, grid (ceil(M/W), ncols)).
// All operands of a geometry (x_a, its Jacobian factors g_a) and of the column's
// geometry b (x_b, w = J_b e_l) are first staged in shared memory with independent,
// coalesced loads; the warp then forms s = delta_(i,.) . w (shuffle reduction),
// u = coef delta + A_ab w on the pairs of atom i, and the 3N outputs J_a^T u from
// shared memory only.  Shared memory: D + N doubles per CTA plus 5 D per warp.
__global__ void __launch_bounds__(256) kcol_warp_kernel(const int64_t* __restrict__ cols,
                                                        const double* __restrict__ X, const double* __restrict__ G,
                                                        const double* __restrict__ S, const double* __restrict__ A,
                                                        int64_t ldA, int64_t M, int N, int D, double c2,
                                                        double* __restrict__ out, int64_t ldo,
                                                        const int* __restrict__ stop_flag) {
  if (stop_flag && *stop_flag) return;
  extern __shared__ double shw[];
  const int W = blockDim.x >> 5;
  double* wsp = shw;            // N: (J_b e_l) on the pairs (i, j), indexed by partner j
  double* sxb = shw + N;        // D: x_b
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* sxa = shw + N + D + (size_t)warp * 5 * D;  // D: x_a
  double* u = sxa + D;                                 // D
  double* sga = u + D;                                 // 3 D: g_a
  const int64_t c = blockIdx.y;
  const int64_t col = cols[c];
  const int B = 3 * N;
  const int64_t b = col / B;
  const int l = (int)(col - b * B), i = l / 3, q = l - 3 * i;
  const double* Xb = X + b * D;
  const double* Gb = G + b * D * 3;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double w = 0.0;
    if (j != i) {
      const int p = pair_idx(i, j);
      w = (i > j) ? -Gb[3 * p + q] : Gb[3 * p + q];
    }
    wsp[j] = w;
  }
  for (int p = threadIdx.x; p < D; p += blockDim.x) sxb[p] = Xb[p];
  const int64_t a = (int64_t)blockIdx.x * W + warp;
  const bool live = a < M;
  if (live) {  // eight independent loads in flight per lane, then the shared-memory stores
    const double* Xa = X + a * D;
    const double* Ga = G + a * D * 3;
    for (int e0 = lane; e0 < 4 * D; e0 += 32 * 8) {
      double tmp[8];
#pragma unroll
      for (int u8 = 0; u8 < 8; ++u8) {
        const int e = e0 + 32 * u8;
        tmp[u8] = e < D ? Xa[e] : (e < 4 * D ? Ga[e - D] : 0.0);
      }
#pragma unroll
      for (int u8 = 0; u8 < 8; ++u8) {
        const int e = e0 + 32 * u8;
        if (e < D)
          sxa[e] = tmp[u8];
        else if (e < 4 * D)
          sga[e - D] = tmp[u8];
      }
    }
  }
  __syncthreads();
  if (!live) return;
  double sd = 0.0;
  for (int j = lane; j < N; j += 32)
    if (j != i) {
      const int p = pair_idx(i, j);
      sd = fma(sxa[p] - sxb[p], wsp[j], sd);
    }
  for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
  const double Aab = A[a * ldA + b];
  const double coef = -c2 * S[a * M + b] * sd;
  for (int p = lane; p < D; p += 32) u[p] = coef * (sxa[p] - sxb[p]);
  __syncwarp();
  for (int j = lane; j < N; j += 32)
    if (j != i) u[pair_idx(i, j)] += Aab * wsp[j];
  __syncwarp();
  for (int l2 = lane; l2 < B; l2 += 32) {
    const int i2 = l2 / 3, q2 = l2 - 3 * i2;
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
      const bool skip = j == i2;
      const int p = skip ? 0 : pair_idx(i2, j);
      const double gj = sga[3 * p + q2] * u[p];
      s += skip ? 0.0 : ((i2 > j) ? -gj : gj);
    }
    out[c * ldo + a * B + l2] = s;
  }
}

// ---- double-float helpers for the kernel column (pairs (hi, lo) of FP32 on the FP32 lanes)
__device__ __forceinline__ float2 dfk_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ float2 dfk_add(float2 a, float2 b) {  // a + b
  const float s = __fadd_rn(a.x, b.x);
  const float v = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 dfk_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dfk_mul(float2 a, float2 b) {  // a b
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// Kernel columns in double-float on the FP32 lanes (DF64/OZAKI contexts): the algebra of
// kcol_warp_kernel with x and g read as float pairs (split once per context) and c^2 S_ab,
// A_ab split on the fly.  GB300's FP64 pipe is a small fraction of its FP32 lanes and the
// FP64 form of this kernel was bound by it; the column is accurate to ~1e-14 of its terms,
// the class of the double-float Schur sums it meets in Algorithm 1.  S and A are symmetric:
// column b is read as row b.  One warp per geometry a, W warps per CTA.
__global__ void __launch_bounds__(256) kcol_df_kernel(const int64_t* __restrict__ cols,
                                                      const float2* __restrict__ X2, const float2* __restrict__ G2,
                                                      const double* __restrict__ S, const double* __restrict__ A,
                                                      int64_t ldA, int64_t M, int N, int D, double c2,
                                                      double* __restrict__ out, int64_t ldo,
                                                      const int* __restrict__ stop_flag) {
  if (stop_flag && *stop_flag) return;
  extern __shared__ float2 shf[];
  const int W = blockDim.x >> 5;
  float2* wsp = shf;        // N: +-g_b on the pairs (i, j), indexed by partner j
  float2* sxb = shf + N;    // D: x_b
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sxa = shf + N + D + (size_t)warp * 5 * D;  // D: x_a - x_b
  float2* u = sxa + D;                                 // D
  float2* sga = u + D;                                 // 3 D: g_a
  const int64_t c = blockIdx.y;
  const int64_t col = cols[c];
  const int B = 3 * N;
  const int64_t a = (int64_t)blockIdx.x * W + warp;
  const bool live = a < M;
  float2 sab = make_float2(0.f, 0.f), aab = sab;
  // geometry a's operands do not depend on the pivot: their loads go first
  if (live) {  // eight independent loads in flight per lane, then the shared-memory stores
    const float2* Xa = X2 + a * D;
    const float2* Ga = G2 + a * D * 3;
    for (int e0 = lane; e0 < 4 * D; e0 += 32 * 8) {
      float2 tmp[8];
#pragma unroll
      for (int u8 = 0; u8 < 8; ++u8) {
        const int e = e0 + 32 * u8;
        tmp[u8] = e < D ? Xa[e] : (e < 4 * D ? Ga[e - D] : make_float2(0.f, 0.f));
      }
#pragma unroll
      for (int u8 = 0; u8 < 8; ++u8) {
        const int e = e0 + 32 * u8;
        if (e < D)
          sxa[e] = tmp[u8];
        else if (e < 4 * D)
          sga[e - D] = tmp[u8];
      }
    }
  }
  const int64_t b = col / B;
  const int l = (int)(col - b * B), i = l / 3, q = l - 3 * i;
  const float2* Xb = X2 + b * D;
  const float2* Gb = G2 + b * D * 3;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float2 w = make_float2(0.f, 0.f);
    if (j != i) {
      const float2 g = Gb[3 * pair_idx(i, j) + q];
      w = (i > j) ? dfk_neg(g) : g;
    }
    wsp[j] = w;
  }
  for (int p = threadIdx.x; p < D; p += blockDim.x) sxb[p] = Xb[p];
  if (live && lane == 0) {
    sab = dfk_mul(dfk_split(c2), dfk_split(S[b * M + a]));
    aab = dfk_split(A[b * ldA + a]);
  }
  __syncthreads();
  if (!live) return;
  sab = make_float2(__shfl_sync(0xffffffffu, sab.x, 0), __shfl_sync(0xffffffffu, sab.y, 0));
  aab = make_float2(__shfl_sync(0xffffffffu, aab.x, 0), __shfl_sync(0xffffffffu, aab.y, 0));
  for (int p = lane; p < D; p += 32) sxa[p] = dfk_add(sxa[p], dfk_neg(sxb[p]));  // x_a - x_b
  __syncwarp();
  float2 sd = make_float2(0.f, 0.f);
  for (int j = lane; j < N; j += 32)
    if (j != i) sd = dfk_add(sd, dfk_mul(sxa[pair_idx(i, j)], wsp[j]));
  for (int o = 16; o > 0; o >>= 1)
    sd = dfk_add(sd, make_float2(__shfl_xor_sync(0xffffffffu, sd.x, o), __shfl_xor_sync(0xffffffffu, sd.y, o)));
  const float2 coef = dfk_neg(dfk_mul(sab, sd));
  for (int p = lane; p < D; p += 32) u[p] = dfk_mul(coef, sxa[p]);
  __syncwarp();
  for (int j = lane; j < N; j += 32)
    if (j != i) {
      const int p = pair_idx(i, j);
      u[p] = dfk_add(u[p], dfk_mul(aab, wsp[j]));
    }
  __syncwarp();
  for (int l2 = lane; l2 < B; l2 += 32) {
    const int i2 = l2 / 3, q2 = l2 - 3 * i2;
    float2 s2 = make_float2(0.f, 0.f);
    for (int j = 0; j < N; ++j) {
      if (j == i2) continue;
      const int p = pair_idx(i2, j);
      const float2 gj = dfk_mul(sga[3 * p + q2], u[p]);
      s2 = dfk_add(s2, (i2 > j) ? dfk_neg(gj) : gj);
    }
    out[c * ldo + a * B + l2] = (double)s2.x + (double)s2.y;
  }
}

// Many kernel columns at once (the Nystrom factor's K_nk, Eq. 5): the same double-float
// arithmetic as kcol_df_kernel, with geometry a's x_a and g_a staged ONCE per CTA and reused by
// a block of CB columns (W warps, one column at a time each), instead of once per (a, column).
// grid (M, ceil(ncols / CB)).  Shared memory: 4 D float pairs for geometry a, plus per warp
// N (w) + 2 D (x_a - x_b, u) float pairs.
constexpr int kColBlock = 64;
__global__ void __launch_bounds__(256) kcol_bulk_df_kernel(const int64_t* __restrict__ cols, int64_t ncols,
                                                           const float2* __restrict__ X2,
                                                           const float2* __restrict__ G2,
                                                           const double* __restrict__ S,
                                                           const double* __restrict__ A, int64_t ldA, int64_t M,
                                                           int N, int D, double c2, double* __restrict__ out,
                                                           int64_t ldo) {
  extern __shared__ float2 shb[];
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sxa = shb;                                   // D: x_a
  float2* sga = sxa + D;                               // 3 D: g_a
  float2* wsp = sga + 3 * D + (size_t)warp * (N + 2 * D);  // N: +-g_b on the pairs (i, j), by partner j
  float2* dab = wsp + N;                               // D: x_a - x_b
  float2* u = dab + D;                                 // D
  const int64_t a = blockIdx.x;
  const int B = 3 * N;
  {
    const float2* Xa = X2 + a * D;
    const float2* Ga = G2 + a * D * 3;
    for (int e = threadIdx.x; e < 4 * D; e += blockDim.x) {
      if (e < D)
        sxa[e] = Xa[e];
      else
        sga[e - D] = Ga[e - D];
    }
  }
  __syncthreads();
  const int64_t c_end = min(ncols, (int64_t)(blockIdx.y + 1) * kColBlock);
  for (int64_t c = (int64_t)blockIdx.y * kColBlock + warp; c < c_end; c += W) {
    const int64_t col = cols[c];
    const int64_t b = col / B;
    const int l = (int)(col - b * B), i = l / 3, q = l - 3 * i;
    const float2* Xb = X2 + b * D;
    const float2* Gb = G2 + b * D * 3;
    for (int j = lane; j < N; j += 32) {
      float2 w = make_float2(0.f, 0.f);
      if (j != i) {
        const float2 g = Gb[3 * pair_idx(i, j) + q];
        w = (i > j) ? dfk_neg(g) : g;
      }
      wsp[j] = w;
    }
    for (int p = lane; p < D; p += 32) dab[p] = dfk_add(sxa[p], dfk_neg(Xb[p]));  // x_a - x_b
    __syncwarp();
    const float2 sab = dfk_mul(dfk_split(c2), dfk_split(S[b * M + a]));
    const float2 aab = dfk_split(A[b * ldA + a]);
    float2 sd = make_float2(0.f, 0.f);
    for (int j = lane; j < N; j += 32)
      if (j != i) sd = dfk_add(sd, dfk_mul(dab[pair_idx(i, j)], wsp[j]));
    for (int o = 16; o > 0; o >>= 1)
      sd = dfk_add(sd, make_float2(__shfl_xor_sync(0xffffffffu, sd.x, o), __shfl_xor_sync(0xffffffffu, sd.y, o)));
    const float2 coef = dfk_neg(dfk_mul(sab, sd));
    for (int p = lane; p < D; p += 32) u[p] = dfk_mul(coef, dab[p]);
    __syncwarp();
    for (int j = lane; j < N; j += 32)
      if (j != i) {
        const int p = pair_idx(i, j);
        u[p] = dfk_add(u[p], dfk_mul(aab, wsp[j]));
      }
    __syncwarp();
    for (int l2 = lane; l2 < B; l2 += 32) {
      const int i2 = l2 / 3, q2 = l2 - 3 * i2;
      float2 s2 = make_float2(0.f, 0.f);
      for (int j = 0; j < N; ++j) {
        if (j == i2) continue;
        const int p = pair_idx(i2, j);
        const float2 gj = dfk_mul(sga[3 * p + q2], u[p]);
        s2 = dfk_add(s2, (i2 > j) ? dfk_neg(gj) : gj);
      }
      out[c * ldo + a * B + l2] = (double)s2.x + (double)s2.y;
    }
    __syncwarp();  // wsp, dab and u are rewritten for the warp's next column
  }
}

bool launch_kcol_bulk_df(const int64_t* cols, int64_t ncols, const float2* X2, const float2* G2, const double* S,
                         const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                         cudaStream_t st) {
  const size_t fixed = 4 * (size_t)D * sizeof(float2), per_warp = ((size_t)N + 2 * (size_t)D) * sizeof(float2);
  const size_t budget = 200 * 1024;
  if (fixed + per_warp > budget || ncols < 1 || M > 2147483647 || cdiv(ncols, kColBlock) > 65535) return false;
  const int W = (int)std::min<size_t>(8, (budget - fixed) / per_warp);
  const size_t smem = fixed + W * per_warp;
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    if (cudaFuncSetAttribute(kcol_bulk_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return false;
    attr = smem;
  }
  dim3 g((unsigned)M, (unsigned)cdiv(ncols, kColBlock));
  { kcol_bulk_df_kernel<<<g, 32 * W, smem, st>>>(cols, ncols, X2, G2, S, A, ldA, M, N, D, c * c, out, ldo); count_launch(); }
  return true;
}

bool launch_kcol_df(const int64_t* cols, int64_t ncols, const float2* X2, const float2* G2, const double* S,
                    const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                    const int* stop_flag, cudaStream_t st) {
  const size_t per_warp = 5 * (size_t)D * sizeof(float2), fixed = ((size_t)N + D) * sizeof(float2);
  int W = (int)std::min<size_t>(8, (200 * 1024 - std::min<size_t>(fixed, 200 * 1024)) / per_warp);
  if (W < 1 || ncols > 65535) return false;
  const int sms = num_sms();
  const int64_t want = std::max<int64_t>(1, M * ncols / (2 * (int64_t)sms));
  if (want < W) W = (int)want;
  const size_t wsmem = fixed + W * per_warp;
  static size_t attr = 0;
  if (wsmem > 48 * 1024 && wsmem > attr) {
    cudaFuncSetAttribute(kcol_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
    attr = wsmem;
  }
  dim3 g((unsigned)cdiv(M, W), (unsigned)ncols);
  { kcol_df_kernel<<<g, 32 * W, wsmem, st>>>(cols, X2, G2, S, A, ldA, M, N, D, c * c, out, ldo, stop_flag); count_launch(); }
  return true;
}

// ---------------------------------------------------------------- launchers
void launch_desc_jac(const double* R, int64_t M, int N, int D, double* X, double* G, cudaStream_t st) {
  int64_t tot = M * D;
  { desc_jac_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(R, M, N, D, X, G); count_launch(); }
}
void launch_center(const double* X, int64_t M, int D, double* Xc, cudaStream_t st) {
  { center_kernel<<<(unsigned)cdiv(D, 32), 256, 0, st>>>(X, M, D, Xc); count_launch(); }
}
void launch_dist_tab(const double* X, int64_t M, int D, double c, double* S, double* A, int64_t ldA,
                     cudaStream_t st) {
  dim3 grid((unsigned)cdiv(M, 32), (unsigned)cdiv(M, 32));
  { dist_tab_kernel<<<grid, 256, 0, st>>>(X, M, D, c, S, A, ldA); count_launch(); }
}
void launch_kdiag(const double* G, int64_t M, int N, int D, double c, double* diag, cudaStream_t st) {
  int64_t tot = M * 3 * N;
  { kdiag_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(G, M, N, D, c * c / 3.0, diag); count_launch(); }
}
void launch_proj(const double* G, const double* Xc, const double* v, int64_t M, int N, int D, double* W,
                 int64_t ldW, double* t, cudaStream_t st) {
  const unsigned threads = (unsigned)std::min<int64_t>(1024, 32 * cdiv(D, 32));
  { proj_cta_kernel<<<(unsigned)M, threads, 3 * N * sizeof(double), st>>>(G, Xc, v, M, N, D, W, ldW, t); count_launch(); }
}
void launch_beta(const double* T, const double* S, const double* t, int64_t M, double c, double* Pb,
                 int64_t ldP, double* rowsum, cudaStream_t st) {
  { beta_kernel<256><<<(unsigned)M, 256, 0, st>>>(T, S, t, M, c * c, Pb, ldP, rowsum); count_launch(); }
}
void launch_beta_rows(const double* T, const double* S, const double* t, int64_t rows, int64_t M, double c,
                      double* Pb, int64_t ldP, double* rowsum, cudaStream_t st) {
  { beta_kernel<256><<<(unsigned)rows, 256, 0, st>>>(T, S, t, M, c * c, Pb, ldP, rowsum); count_launch(); }
}
void launch_dist_tab_cross(const double* Xq, int64_t Q, const double* X, int64_t M, int D, double c, double* S,
                           double* A, int64_t ldA, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(M, 32), (unsigned)cdiv(Q, 32));
  { dist_tab_cross_kernel<<<grid, 256, 0, st>>>(Xq, Q, X, M, D, c, S, A, ldA); count_launch(); }
}
void launch_center_like(const double* Xq, int64_t Q, int D, const double* X, const double* Xc, double* Xqc,
                        cudaStream_t st) {
  { center_like_kernel<<<(unsigned)cdiv(Q * D, 256), 256, 0, st>>>(Xq, Q, D, X, Xc, Xqc); count_launch(); }
}
template <typename TU>
void launch_backproj(const TU* U, int64_t ldU, int splits, int64_t split_stride, const double* rowsum,
                     const double* Xc, const double* G, const double* v, int64_t M, int N, int D, double lam,
                     int add_lambda, double* out, cudaStream_t st) {
  const size_t smem = D * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(backproj_kernel<TU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { backproj_kernel<TU><<<(unsigned)M, 128, smem, st>>>(U, ldU, splits, split_stride, rowsum, Xc, G, v, N, D,
                                                       lam, add_lambda, out); count_launch(); }
}
template void launch_backproj<double>(const double*, int64_t, int, int64_t, const double*, const double*,
                                      const double*, const double*, int64_t, int, int, double, int, double*,
                                      cudaStream_t);
template void launch_backproj<float>(const float*, int64_t, int, int64_t, const double*, const double*,
                                     const double*, const double*, int64_t, int, int, double, int, double*,
                                     cudaStream_t);

void launch_kcol(const int64_t* cols, int64_t ncols, const double* X, const double* G, const double* S,
                 const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                 const int* stop_flag, cudaStream_t st) {
  // warps per CTA so that the staged operands fit in 200 KB of shared memory
  const size_t per_warp = 5 * (size_t)D * sizeof(double), fixed = ((size_t)N + D) * sizeof(double);
  int W = (int)std::min<size_t>(8, (200 * 1024 - std::min<size_t>(fixed, 200 * 1024)) / per_warp);
  {  // few columns (one per Algorithm 1 step): fewer warps per CTA so the grid covers every SM twice
    const int sms = num_sms();
    const int64_t want = std::max<int64_t>(1, M * ncols / (2 * (int64_t)sms));
    if (want < W) W = (int)want;
  }
  if (W >= 1 && ncols <= 65535) {
    const size_t wsmem = fixed + W * per_warp;
    static size_t attr = 0;
    if (wsmem > 48 * 1024 && wsmem > attr) {
      cudaFuncSetAttribute(kcol_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
      attr = wsmem;
    }
    dim3 g((unsigned)cdiv(M, W), (unsigned)ncols);
    { kcol_warp_kernel<<<g, 32 * W, wsmem, st>>>(cols, X, G, S, A, ldA, M, N, D, c * c, out, ldo, stop_flag); count_launch(); }
    return;
  }
  const int per = 8;
  dim3 grid((unsigned)M, (unsigned)cdiv(ncols, per));
  size_t smem = (2 * (size_t)D + N) * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kcol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { kcol_kernel<<<grid, 128, smem, st>>>(cols, ncols, per, X, G, S, A, ldA, M, N, D, c * c, out, ldo, stop_flag); count_launch(); }
}

// *flag = 1 if any of the count values is not finite (NaN or infinite)
__global__ void check_finite_kernel(const double* __restrict__ a, int64_t count, int* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) {
      *flag = 1;
      return;
    }
}

void launch_check_finite(const double* a, int64_t count, int* flag, cudaStream_t st) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(count, 256), 4 * num_sms()));
  { check_finite_kernel<<<grid, 256, 0, st>>>(a, count, flag); count_launch(); }
}

// ---------------------------------------------------------------- permutational symmetries
// A symmetry group of S atom permutations acts on the descriptor by pis (S x D: pi_q(p) = the
// pair index of (sigma_q(i), sigma_q(j)) for p = (i, j)) and pinv (its inverse per q).  The
// symmetric force kernel is K_ab = sum_q J_a^T H(x_a, P_q x_b) P_q J_b with (P_q x)_p = x_pi_q(p);
// its training side holds row b S + q = P_q applied to geometry b.

// out[b S + q][p] = in[b][pi_q(p)] for the M rows of `in`; with xcB, also
// t[b S + q] = xcB[b S + q] . out[b S + q].  One CTA (256 threads) per output row.
__global__ void __launch_bounds__(256) sym_gather_kernel(const double* __restrict__ in, int D,
                                                         const int* __restrict__ pis, int S,
                                                         const double* __restrict__ xcB, double* __restrict__ out,
                                                         double* __restrict__ t) {
  __shared__ double red[8];
  const int64_t row = blockIdx.x;
  const int64_t b = row / S;
  const int q = (int)(row - b * S);
  const int* pi = pis + (int64_t)q * D;
  double part = 0.0;
  for (int p = threadIdx.x; p < D; p += blockDim.x) {
    const double v = in[b * D + pi[p]];
    out[row * D + p] = v;
    if (xcB) part = fma(xcB[row * D + p], v, part);
  }
  if (xcB) {
    part = block_sum<256>(part, red);
    if (threadIdx.x == 0) t[row] = part;
  }
}

void launch_sym_gather(const double* in, int64_t M, int D, const int* pis, int S, const double* xcB, double* out,
                       double* t, cudaStream_t st) {
  { sym_gather_kernel<<<(unsigned)(M * S), 256, 0, st>>>(in, D, pis, S, xcB, out, t); count_launch(); }
}

// the value of u = J_a e_l on descriptor entry pp (zero unless pp pairs atom i with another):
// u_(i,j) = -g_(i,j),c for i > j and +g_(i,j),c for i < j
__device__ __forceinline__ double jac_col_at(const double* __restrict__ g, int pp, int i, int cc) {
  int I, J;
  pair_of(pp, I, J);  // I > J
  if (I == i) return -g[3 * pp + cc];
  if (J == i) return g[3 * pp + cc];
  return 0.0;
}

// diag(K) with symmetries: for column l = 3 i + cc of geometry a, with u = J_a e_l,
//   diag_{a,l} = sum_q u^T H(x_a, P_q x_a) P_q u = sum_q A_q (u . P_q u) - c^2 S_q (u . d_q)(P_q u . d_q),
// d_q = x_a - P_q x_a, (P_q u)_p = u_pi(p), so (P_q u) . d = sum_p' u_p' d_pinv(p').
// One CTA (256 threads) per geometry: d_q and its norm by a CTA reduction, then thread l sums
// over the N - 1 pairs of atom i.
__global__ void __launch_bounds__(256) kdiag_sym_kernel(const double* __restrict__ X, const double* __restrict__ G,
                                                        int N, int D, const int* __restrict__ pis,
                                                        const int* __restrict__ pinv, int S, double c,
                                                        double* __restrict__ diag) {
  extern __shared__ double sdq[];  // D
  __shared__ double red[8];
  __shared__ double s_r;
  const int64_t a = blockIdx.x;
  const double* Xa = X + a * D;
  const double* Ga = G + a * D * 3;
  const int B = 3 * N;
  double acc[2] = {0.0, 0.0};  // B <= 384: l = threadIdx.x, threadIdx.x + 256
  for (int q = 0; q < S; ++q) {
    const int* pi = pis + (int64_t)q * D;
    const int* pv = pinv + (int64_t)q * D;
    double part = 0.0;
    for (int p = threadIdx.x; p < D; p += blockDim.x) {
      const double d = Xa[p] - Xa[pi[p]];
      sdq[p] = d;
      part = fma(d, d, part);
    }
    part = block_sum<256>(part, red);  // synchronises: sdq is complete
    if (threadIdx.x == 0) s_r = sqrt(part);
    __syncthreads();
    const double r = s_r;
    const double Sv = (c * c / 3.0) * exp(-c * r), Av = Sv * (1.0 + c * r);
    for (int k = 0; k < 2; ++k) {
      const int l = threadIdx.x + 256 * k;
      if (l >= B) break;
      const int i = l / 3, cc = l - 3 * i;
      double ud = 0.0, vd = 0.0, uv = 0.0;
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const int pp = pair_idx(i, j);
        const double u = (i > j) ? -Ga[3 * pp + cc] : Ga[3 * pp + cc];
        ud = fma(u, sdq[pp], ud);
        vd = fma(u, sdq[pv[pp]], vd);
        uv = fma(u, jac_col_at(Ga, pi[pp], i, cc), uv);
      }
      acc[k] += Av * uv - c * c * Sv * ud * vd;
    }
    __syncthreads();  // sdq is rewritten for the next symmetry
  }
  for (int k = 0; k < 2; ++k) {
    const int l = threadIdx.x + 256 * k;
    if (l < B) diag[a * B + l] = acc[k];
  }
}

void launch_kdiag_sym(const double* X, const double* G, int64_t M, int N, int D, const int* pis, const int* pinv,
                      int S, double c, double* diag, cudaStream_t st) {
  const size_t smem = (size_t)D * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kdiag_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { kdiag_sym_kernel<<<(unsigned)M, 256, smem, st>>>(X, G, N, D, pis, pinv, S, c, diag); count_launch(); }
}

// Kernel columns with symmetries: column (b, l = 3 i + cc), u = J_b e_l, for every geometry a
//   K[a, col] = J_a^T sum_q [A_q w_q - c^2 S_q (d_q . w_q) d_q],
// w_q = P_q u ((w_q)_pinv(p') = u_p'), d_q = x_a - P_q x_b, S_q and A_q from the context's
// tables at (a, b S + q).  One warp per (geometry a, column), W warps per CTA; FP64.
__global__ void __launch_bounds__(256) kcol_sym_kernel(const int64_t* __restrict__ cols,
                                                       const double* __restrict__ X, const double* __restrict__ G,
                                                       const double* __restrict__ Stab,
                                                       const double* __restrict__ Atab, int64_t ldA, int64_t M,
                                                       int64_t MB, int N, int D, const int* __restrict__ pis,
                                                       const int* __restrict__ pinv, int S, double c2,
                                                       double* __restrict__ out, int64_t ldo,
                                                       const int* __restrict__ stop_flag) {
  if (stop_flag && *stop_flag) return;
  extern __shared__ double shs[];
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* ub = shs + (size_t)warp * (N + 6 * (size_t)D);  // N: u on the pairs (i, j), by partner j
  double* xa = ub + N;                                    // D
  double* ga = xa + D;                                    // 3 D
  double* dq = ga + 3 * D;                                // D
  double* uacc = dq + D;                                  // D
  const int64_t c = blockIdx.y;
  const int64_t col = cols[c];
  const int B = 3 * N;
  const int64_t b = col / B;
  const int l = (int)(col - b * B), i = l / 3, cc = l - 3 * i;
  const int64_t a = (int64_t)blockIdx.x * W + warp;
  if (a >= M) return;  // warp-level work only below
  const double* Xa = X + a * D;
  const double* Ga = G + a * D * 3;
  const double* Xb = X + b * D;
  const double* Gb = G + b * D * 3;
  for (int j = lane; j < N; j += 32) {
    double u = 0.0;
    if (j != i) {
      const int pp = pair_idx(i, j);
      u = (i > j) ? -Gb[3 * pp + cc] : Gb[3 * pp + cc];
    }
    ub[j] = u;
  }
  for (int p = lane; p < D; p += 32) {
    xa[p] = Xa[p];
    uacc[p] = 0.0;
  }
  for (int e = lane; e < 3 * D; e += 32) ga[e] = Ga[e];
  __syncwarp();
  for (int q = 0; q < S; ++q) {
    const int* pi = pis + (int64_t)q * D;
    const int* pv = pinv + (int64_t)q * D;
    for (int p = lane; p < D; p += 32) dq[p] = xa[p] - Xb[pi[p]];
    __syncwarp();
    double sd = 0.0;
    for (int j = lane; j < N; j += 32)
      if (j != i) sd = fma(ub[j], dq[pv[pair_idx(i, j)]], sd);
    for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
    const double Sq = Stab[a * MB + b * S + q], Aq = Atab[a * ldA + b * S + q];
    const double coef = -c2 * Sq * sd;
    for (int p = lane; p < D; p += 32) uacc[p] = fma(coef, dq[p], uacc[p]);
    __syncwarp();
    for (int j = lane; j < N; j += 32)
      if (j != i) {
        const int p = pv[pair_idx(i, j)];
        uacc[p] = fma(Aq, ub[j], uacc[p]);
      }
    __syncwarp();
  }
  for (int l2 = lane; l2 < B; l2 += 32) {
    const int i2 = l2 / 3, q2 = l2 - 3 * i2;
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
      if (j == i2) continue;
      const int p = pair_idx(i2, j);
      const double gj = ga[3 * p + q2] * uacc[p];
      s += (i2 > j) ? -gj : gj;
    }
    out[c * ldo + a * B + l2] = s;
  }
}

bool launch_kcol_sym(const int64_t* cols, int64_t ncols, const double* X, const double* G, const double* Stab,
                     const double* Atab, int64_t ldA, int64_t M, int64_t MB, int N, int D, const int* pis,
                     const int* pinv, int S, double c, double* out, int64_t ldo, const int* stop_flag,
                     cudaStream_t st) {
  const size_t per_warp = ((size_t)N + 6 * (size_t)D) * sizeof(double);
  const int W = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
  if (W < 1 || ncols < 1 || ncols > 65535) return false;
  const size_t smem = W * per_warp;
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    if (cudaFuncSetAttribute(kcol_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return false;
    attr = smem;
  }
  dim3 g((unsigned)cdiv(M, W), (unsigned)ncols);
  { kcol_sym_kernel<<<g, 32 * W, smem, st>>>(cols, X, G, Stab, Atab, ldA, M, MB, N, D, pis, pinv, S, c * c, out, ldo, stop_flag); count_launch(); }
  return true;
}

}  // namespace gdml
