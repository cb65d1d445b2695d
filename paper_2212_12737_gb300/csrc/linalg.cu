// Dense FP64 linear algebra for the Nystrom / Woodbury preconditioner (Eqs. 4-5):
//  - blocked right-looking Cholesky of a k x k SPD matrix (K_kk and C = lambda I + L^T L)
//  - forward substitution with many right-hand sides (L_k = K_nk L_kk^-T)
//  - forward / backward substitution for one vector (Woodbury apply)
// A non-positive or non-finite pivot is reported through a device status word
// (index of the failing column + 1), never by trapping.
#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

constexpr int NB = 64;  // panel width

// Unblocked Cholesky of the nb x nb diagonal block at (j0, j0), in place (lower).
__global__ void potrf_diag_kernel(double* __restrict__ A, int64_t lda, int64_t j0, int nb,
                                  int* __restrict__ status) {
  __shared__ double L[NB][NB + 1];
  __shared__ int bad;
  if (*status) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    L[r][c] = A[(j0 + r) * lda + j0 + c];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tid == 0) {
      double d = L[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = c + 1;
      } else {
        L[c][c] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double inv = 1.0 / L[c][c];
    for (int r = c + 1 + tid; r < nb; r += blockDim.x) L[r][c] *= inv;
    __syncthreads();
    // trailing update of the lower part of the block
    for (int e = tid; e < (nb - c - 1) * (nb - c - 1); e += blockDim.x) {
      int r = c + 1 + e / (nb - c - 1), cc = c + 1 + e % (nb - c - 1);
      if (cc <= r) L[r][cc] = fma(-L[r][c], L[cc][c], L[r][cc]);
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) *status = (int)(j0 + bad);
    return;
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    A[(j0 + r) * lda + j0 + c] = (c <= r) ? L[r][c] : 0.0;
  }
}

// Rows r in [r0, rend): solve x L_jj^T = A[r, j0:j0+nb]  (one thread per row).
__global__ void trsm_right_kernel(double* __restrict__ A, int64_t lda, int64_t j0, int nb, int64_t r0,
                                  int64_t rend, const int* __restrict__ status) {
  __shared__ double L[NB][NB + 1];
  if (*status) return;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    L[r][c] = A[(j0 + r) * lda + j0 + c];
  }
  __syncthreads();
  int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rend) return;
  double x[NB];
  double* row = A + r * lda + j0;
  for (int c = 0; c < nb; ++c) {
    double s = row[c];
    for (int cp = 0; cp < c; ++cp) s = fma(-x[cp], L[c][cp], s);
    x[c] = s / L[c][c];
  }
  for (int c = 0; c < nb; ++c) row[c] = x[c];
}

// Left forward substitution on a block of rows of B (k x nrhs, row-major, ld):
// B[j0:j0+nb, col] <- L_jj^-1 B[j0:j0+nb, col]; one thread per column.
__global__ void trsm_left_diag_kernel(const double* __restrict__ Lkk, int64_t ldl, int64_t j0, int nb,
                                      double* __restrict__ Bm, int64_t ldb, int64_t nrhs) {
  __shared__ double L[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    L[r][c] = Lkk[(j0 + r) * ldl + j0 + c];
  }
  __syncthreads();
  int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  double x[NB];
  for (int r = 0; r < nb; ++r) {
    double s = Bm[(j0 + r) * ldb + col];
    for (int c = 0; c < r; ++c) s = fma(-L[r][c], x[c], s);
    x[r] = s / L[r][r];
    Bm[(j0 + r) * ldb + col] = x[r];
  }
}

// Single-vector triangular solves with a lower-triangular k x k factor L
// (row-major).  Column-oriented substitution across one CTA.
__global__ void trsv_lower_kernel(const double* __restrict__ L, int64_t k, double* __restrict__ x) {
  extern __shared__ double xs[];
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) xs[i] = x[i];
  __syncthreads();
  for (int64_t c = 0; c < k; ++c) {
    const double xc = xs[c] / L[c * k + c];
    __syncthreads();
    if (threadIdx.x == 0) xs[c] = xc;
    for (int64_t r = c + 1 + threadIdx.x; r < k; r += blockDim.x) xs[r] = fma(-L[r * k + c], xc, xs[r]);
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) x[i] = xs[i];
}

// x <- L^-T x  (L lower, row-major): backward substitution over rows of L.
__global__ void trsv_lower_t_kernel(const double* __restrict__ L, int64_t k, double* __restrict__ x) {
  extern __shared__ double xs[];
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) xs[i] = x[i];
  __syncthreads();
  for (int64_t c = k - 1; c >= 0; --c) {
    const double xc = xs[c] / L[c * k + c];
    __syncthreads();
    if (threadIdx.x == 0) xs[c] = xc;
    // x_r -= L[c][r] * x_c for r < c (row c of L holds column c of L^T)
    for (int64_t r = threadIdx.x; r < c; r += blockDim.x) xs[r] = fma(-L[c * k + r], xc, xs[r]);
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) x[i] = xs[i];
}

__global__ void add_diag_kernel(double* A, int64_t lda, int64_t k, double eps) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < k) A[i * lda + i] += eps;
}

// ---------------------------------------------------------------- host drivers
// In-place lower Cholesky of the k x k row-major matrix A.  status (device int)
// receives 0 on success or (failing column + 1).
void cholesky_inplace(double* A, int64_t k, int* status, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < k; j0 += NB) {
    int nb = (int)((k - j0) < NB ? (k - j0) : NB);
    { potrf_diag_kernel<<<1, 256, 0, st>>>(A, k, j0, nb, status); count_launch(); }
    int64_t r0 = j0 + nb;
    if (r0 < k) {
      { trsm_right_kernel<<<(unsigned)cdiv(k - r0, 128), 128, 0, st>>>(A, k, j0, nb, r0, k, status); count_launch(); }
      // A22 -= L21 L21^T (lower tiles only)
      launch_dgemm<double, double>(true, k - r0, k - r0, nb, -1.0, A + r0 * k + j0, k, A + r0 * k + j0, k,
                                   1.0, A + r0 * k + r0, k, true, st);
    }
  }
}

// B (k x nrhs row-major) <- Lkk^-1 B  (blocked forward substitution)
void trsm_left_lower(const double* Lkk, int64_t k, double* Bm, int64_t nrhs, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < k; j0 += NB) {
    int nb = (int)((k - j0) < NB ? (k - j0) : NB);
    { trsm_left_diag_kernel<<<(unsigned)cdiv(nrhs, 128), 128, 0, st>>>(Lkk, k, j0, nb, Bm, nrhs, nrhs); count_launch(); }
    int64_t r0 = j0 + nb;
    if (r0 < k)  // B[r0:, :] -= L[r0:, j0:j0+nb] * B[j0:j0+nb, :]
      launch_dgemm<double, double>(false, k - r0, nrhs, nb, -1.0, Lkk + r0 * k + j0, k, Bm + j0 * nrhs, nrhs,
                                   1.0, Bm + r0 * nrhs, nrhs, false, st);
  }
}

void trsv_lower_single_cta(const double* L, int64_t k, double* x, bool transpose, cudaStream_t st) {
  size_t smem = (size_t)k * sizeof(double);
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(trsv_lower_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(trsv_lower_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (transpose)
    { trsv_lower_t_kernel<<<1, 1024, smem, st>>>(L, k, x); count_launch(); }
  else
    { trsv_lower_kernel<<<1, 1024, smem, st>>>(L, k, x); count_launch(); }
}

// Multi-CTA blocked substitution with decoupled look-back.
// Solves L y = b (forward) or L^T y = b (backward) in place on x, L lower k x k
// row-major.  Block rows of TB = 64; a CTA takes a ticket (launch order) and
// solves block t (forward) or block nb-1-t (backward).  It folds in the
// contributions of the already-solved blocks as their flags appear
// (flags[j] == 1; ticket and flags are zeroed before every launch), then
// solves its 64 x 64 diagonal block and publishes its y.  A CTA only waits on CTAs that took earlier tickets and are already
// running, so the dependency chain always makes progress; every wait is still
// bounded, and a timeout sets *err and leaves the block unsolved.
constexpr int TB = 64;
constexpr uint32_t kLookbackSpin = 1u << 24;

__global__ void __launch_bounds__(256) trsv_lookback_kernel(const double* __restrict__ L, int64_t k,
                                                            double* __restrict__ x, int* __restrict__ sync,
                                                            int backward, int* __restrict__ err) {
  unsigned* ticket = reinterpret_cast<unsigned*>(sync);
  int* flags = sync + 1;
  const int epoch = 1;
  __shared__ double yprev[TB];
  __shared__ double part[4][TB + 1];
  __shared__ double ys[TB];
  __shared__ double Ld[TB][TB + 1];
  __shared__ unsigned s_t;
  __shared__ int s_ok;
  const int nb = (int)((k + TB - 1) / TB);
  if (threadIdx.x == 0) {
    s_t = atomicAdd(ticket, 1u);
    s_ok = 1;
  }
  __syncthreads();
  const int t = (int)s_t;
  const int blk = backward ? nb - 1 - t : t;
  const int64_t r0 = (int64_t)blk * TB;
  const int rows = (int)((k - r0) < TB ? (k - r0) : TB);
  const int r = threadIdx.x & (TB - 1), q = threadIdx.x >> 6;  // 4 threads per row, 16 columns each
  double acc = 0.0;
  // contributions of earlier blocks, in solve order
  for (int jj = 0; jj < t; ++jj) {
    const int jb = backward ? nb - 1 - jj : jj;
    const int64_t c0 = (int64_t)jb * TB;
    const int cols = (int)((k - c0) < TB ? (k - c0) : TB);
    if (threadIdx.x == 0) {
      uint32_t it = 0;
      while (((volatile int*)flags)[jb] != epoch && it < kLookbackSpin) {
        ++it;
        if (it > 32) __nanosleep(128);
      }
      if (it >= kLookbackSpin) {
        s_ok = 0;
        atomicExch(err, 1);
      }
      __threadfence();
    }
    __syncthreads();
    if (!s_ok) return;
    if (threadIdx.x < cols) yprev[threadIdx.x] = ((volatile double*)x)[c0 + threadIdx.x];
    __syncthreads();
    if (r < rows) {
      for (int c = q * 16; c < q * 16 + 16 && c < cols; ++c) {
        // forward: L[r0+r][c0+c]; backward (L^T): L[c0+c][r0+r]
        const double l = backward ? L[(c0 + c) * k + r0 + r] : L[(r0 + r) * k + c0 + c];
        acc = fma(l, yprev[c], acc);
      }
    }
    __syncthreads();
  }
  part[q][r] = acc;
  if (threadIdx.x < rows) yprev[threadIdx.x] = x[r0 + threadIdx.x];  // right-hand side of this block
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int rr = e / TB, cc = e % TB;
    double v = 0.0;
    if (rr < rows && cc < rows) v = backward ? L[(r0 + cc) * k + r0 + rr] : L[(r0 + rr) * k + r0 + cc];
    Ld[rr][cc] = v;  // Ld = diagonal block of the (possibly transposed) triangular factor
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i0 = 0; i0 < rows; ++i0) {
      const int i = backward ? rows - 1 - i0 : i0;
      double s = 0.0;
      for (int c = lane; c < rows; c += 32) {
        const bool dep = backward ? (c > i) : (c < i);
        if (dep) s = fma(Ld[i][c], ys[c], s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const double b = yprev[i] - (part[0][i] + part[1][i] + part[2][i] + part[3][i]);
        ys[i] = (b - s) / Ld[i][i];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x < rows) x[r0 + threadIdx.x] = ys[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(&flags[blk], epoch);
}

void trsv_lower(const double* L, int64_t k, double* x, bool transpose, TrsvState& ts, cudaStream_t st) {
  const int nb = (int)((k + TB - 1) / TB);
  cudaMemsetAsync(ts.sync, 0, (nb + 1) * sizeof(int), st);
  { trsv_lookback_kernel<<<nb, 256, 0, st>>>(L, k, x, ts.sync, transpose ? 1 : 0, ts.err); count_launch(); }
}

int64_t trsv_sync_len(int64_t k) { return (k + TB - 1) / TB + 1; }

void add_diag(double* A, int64_t lda, int64_t k, double eps, cudaStream_t st) {
  { add_diag_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(A, lda, k, eps); count_launch(); }
}

}  // namespace gdml
