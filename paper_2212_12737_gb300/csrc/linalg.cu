// Dense FP64 linear algebra for the Nystrom / Woodbury preconditioner (Eqs. 4-5):
//  - blocked right-looking Cholesky of a k x k SPD matrix (K_kk and C = lambda I + L^T L)
//  - forward substitution with many right-hand sides (L_k = K_nk L_kk^-T)
//  - the explicit inverse C^-1 = L_C^-T L_C^-1 used by the Woodbury apply
// A non-positive or non-finite pivot is reported through a device status word
// (index of the failing column + 1), never by trapping.
#include <algorithm>

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

// B (k x nrhs row-major) <- Lkk^-1 B  (blocked forward substitution).  lower_rhs: B is lower
// triangular (the identity, for Lkk^-1 itself), so row block j0 and everything it updates
// have no nonzeros past column j0 + nb and only those columns are touched (a third of the
// flops).
void trsm_left_lower(const double* Lkk, int64_t k, double* Bm, int64_t nrhs, cudaStream_t st, bool lower_rhs) {
  for (int64_t j0 = 0; j0 < k; j0 += NB) {
    int nb = (int)((k - j0) < NB ? (k - j0) : NB);
    const int64_t ncols = lower_rhs ? std::min<int64_t>(nrhs, j0 + nb) : nrhs;
    { trsm_left_diag_kernel<<<(unsigned)cdiv(ncols, 128), 128, 0, st>>>(Lkk, k, j0, nb, Bm, nrhs, ncols); count_launch(); }
    int64_t r0 = j0 + nb;
    if (r0 < k)  // B[r0:, :ncols] -= L[r0:, j0:j0+nb] * B[j0:j0+nb, :ncols]
      launch_dgemm<double, double>(false, k - r0, ncols, nb, -1.0, Lkk + r0 * k + j0, k, Bm + j0 * nrhs, nrhs,
                                   1.0, Bm + r0 * nrhs, nrhs, false, st);
  }
}

__global__ void transpose_square_kernel(const double* __restrict__ A, int64_t k, double* __restrict__ At) {
  __shared__ double tile[32][33];
  const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t r = by + yy, c = bx + threadIdx.x;
    tile[yy][threadIdx.x] = (r < k && c < k) ? A[r * k + c] : 0.0;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t r = bx + yy, c = by + threadIdx.x;
    if (r < k && c < k) At[r * k + c] = tile[threadIdx.x][yy];
  }
}

__global__ void set_identity_kernel(double* A, int64_t k) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < k * k) A[e] = (e / k == e % k) ? 1.0 : 0.0;
}

void transpose_square(const double* A, int64_t k, double* At, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(k, 32), (unsigned)cdiv(k, 32));
  { transpose_square_kernel<<<grid, dim3(32, 8), 0, st>>>(A, k, At); count_launch(); }
}

// A[c][r] = A[r][c] for r > c (copy the lower triangle onto the upper one)
__global__ void mirror_lower_kernel(double* A, int64_t k) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int64_t r = e / k, c = e % k;
  if (r > c) A[c * k + r] = A[e];
}

void mirror_lower(double* A, int64_t k, cudaStream_t st) {
  { mirror_lower_kernel<<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(A, k); count_launch(); }
}

void set_identity(double* A, int64_t k, cudaStream_t st) {
  { set_identity_kernel<<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(A, k); count_launch(); }
}

void add_diag(double* A, int64_t lda, int64_t k, double eps, cudaStream_t st) {
  { add_diag_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(A, lda, k, eps); count_launch(); }
}

}  // namespace gdml
