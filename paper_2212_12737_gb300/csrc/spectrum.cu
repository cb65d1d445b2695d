// Spectrum diagnostics and the SVD preconditioner (Sec. 2.2, Sec. 4.1 / Fig. 3, App. A.1).
//
// * SVD preconditioner: K is PSD, so its SVD is its eigendecomposition K = U Sigma U^T; the
//   rank-k preconditioner keeps the k dominant eigenpairs, P = U_k Sigma_k U_k^T + lam I, which
//   is the Woodbury form of Eq. 4 with the n x k factor L_k = U_k Sigma_k^(1/2).  The paper uses
//   it only as the optimal reference on small n (its cost is O(n^3) here, O(k n^2) at best).
//   The dense eigendecomposition is cuSOLVER's syevd (a library routine, like a library GEMM),
//   loaded on first use so that the library does not depend on it otherwise.
// * Lanczos matrix of PCG: CG's step lengths gamma_j and ratios beta_j = rho_(j+1) / rho_j give
//   the tridiagonal T_m of the Lanczos process on P^-1 K_lam (T[0,0] = 1/gamma_0,
//   T[j,j] = 1/gamma_j + beta_(j-1)/gamma_(j-1), T[j,j+1] = sqrt(beta_j)/gamma_j).  Its
//   eigenvalues (Ritz values) lie inside the spectrum of P^-1 K_lam and converge to its extreme
//   eigenvalues, so a solve yields an estimate of cond(P^-1 K_lam) at any n.  They are found
//   by bisection on Sturm sequence counts (Barth, Martin and Wilkinson, Numer. Math. 9, 1967).
#include <cusolverDn.h>
#include <dlfcn.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace gdml {

namespace {

__global__ void svd_factor_kernel(const double* __restrict__ U, const double* __restrict__ w, int64_t n, int64_t k,
                                  double* __restrict__ L) {
  const int64_t total = n * k;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / n, i = idx - j * n;
    const int64_t src = n - 1 - j;
    L[idx] = U[src * n + i] * sqrt(fmax(w[src], 0.0));
  }
}

// cuSOLVER entry points, resolved once from the shared library
struct SolverApi {
  bool ok = false;
  std::string why;
  cusolverStatus_t (*create)(cusolverDnHandle_t*) = nullptr;
  cusolverStatus_t (*destroy)(cusolverDnHandle_t) = nullptr;
  cusolverStatus_t (*set_stream)(cusolverDnHandle_t, cudaStream_t) = nullptr;
  cusolverStatus_t (*syevd_size)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, const double*, int,
                                 const double*, int*) = nullptr;
  cusolverStatus_t (*syevd)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, double*, int, double*,
                            double*, int, int*) = nullptr;
};

SolverApi load_solver() {
  SolverApi a;
  void* h = nullptr;
  for (const char* name : {"libcusolver.so.12", "libcusolver.so.11", "libcusolver.so"})
    if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) {
    a.why = "cannot load libcusolver";
    return a;
  }
  a.create = reinterpret_cast<decltype(a.create)>(dlsym(h, "cusolverDnCreate"));
  a.destroy = reinterpret_cast<decltype(a.destroy)>(dlsym(h, "cusolverDnDestroy"));
  a.set_stream = reinterpret_cast<decltype(a.set_stream)>(dlsym(h, "cusolverDnSetStream"));
  a.syevd_size = reinterpret_cast<decltype(a.syevd_size)>(dlsym(h, "cusolverDnDsyevd_bufferSize"));
  a.syevd = reinterpret_cast<decltype(a.syevd)>(dlsym(h, "cusolverDnDsyevd"));
  a.ok = a.create && a.destroy && a.set_stream && a.syevd_size && a.syevd;
  if (!a.ok) a.why = "libcusolver lacks the syevd entry points";
  return a;
}

const SolverApi& solver_api() {
  static std::once_flag once;
  static SolverApi api;
  std::call_once(once, [] { api = load_solver(); });
  return api;
}

}  // namespace

void launch_svd_factor(const double* U, const double* w, int64_t n, int64_t k, double* L, cudaStream_t st) {
  const int64_t total = n * k;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 16 * num_sms());
  { svd_factor_kernel<<<std::max(blocks, 1), 256, 0, st>>>(U, w, n, k, L); count_launch(); }
}

std::string eigh_dense(double* A, int64_t n, double* w, cudaStream_t st) {
  if (n < 1 || n > INT_MAX) return "matrix order out of range";
  const SolverApi& api = solver_api();
  if (!api.ok) return api.why;
  cusolverDnHandle_t h = nullptr;
  if (api.create(&h) != CUSOLVER_STATUS_SUCCESS) return "cusolverDnCreate failed";
  std::string err;
  int lwork = 0;
  double* work = nullptr;
  int* info = nullptr;
  if (api.set_stream(h, st) != CUSOLVER_STATUS_SUCCESS) err = "cusolverDnSetStream failed";
  if (err.empty() && api.syevd_size(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n, A, (int)n, w,
                                    &lwork) != CUSOLVER_STATUS_SUCCESS)
    err = "syevd workspace query failed";
  if (err.empty() && (cudaMalloc(&work, (size_t)std::max(lwork, 1) * sizeof(double)) != cudaSuccess ||
                      cudaMalloc(&info, sizeof(int)) != cudaSuccess))
    err = "out of device memory for the syevd workspace";
  if (err.empty() && api.syevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n, A, (int)n, w, work, lwork,
                               info) != CUSOLVER_STATUS_SUCCESS)
    err = "syevd failed";
  int hinfo = 0;
  if (err.empty() && (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess))
    err = "syevd: reading its status failed";
  if (err.empty() && hinfo != 0) err = "syevd did not converge (info " + std::to_string(hinfo) + ")";
  cudaStreamSynchronize(st);
  if (work) cudaFree(work);
  if (info) cudaFree(info);
  api.destroy(h);
  return err;
}

void lanczos_ritz(const double* gamma, const double* beta, int64_t m, int64_t count, double* top, double* tmin,
                  double* tmax) {
  std::vector<double> d(m), e2(m > 1 ? m - 1 : 0);
  for (int64_t j = 0; j < m; ++j) {
    d[j] = 1.0 / gamma[j] + (j > 0 ? beta[j - 1] / gamma[j - 1] : 0.0);
    if (j + 1 < m) e2[j] = beta[j] / (gamma[j] * gamma[j]);  // (sqrt(beta_j) / gamma_j)^2
  }
  double lo = INFINITY, hi = -INFINITY, emax = 1.0;
  for (int64_t j = 0; j < m; ++j) {
    const double r = (j > 0 ? std::sqrt(e2[j - 1]) : 0.0) + (j + 1 < m ? std::sqrt(e2[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
    if (j + 1 < m) emax = std::max(emax, e2[j]);
  }
  const double pivmin = DBL_MIN * emax;
  // number of eigenvalues of T below x (the signs of the Sturm sequence's pivots)
  auto below = [&](double x) {
    int64_t cnt = 0;
    double q = d[0] - x;
    for (int64_t j = 0;; ++j) {
      if (std::fabs(q) < pivmin) q = -pivmin;
      if (q < 0.0) ++cnt;
      if (j + 1 == m) break;
      q = d[j + 1] - x - e2[j] / q;
    }
    return cnt;
  };
  // the j-th smallest eigenvalue (0-based) by bisection of the Gershgorin interval
  auto kth = [&](int64_t j) {
    double a = lo, z = hi;
    for (int it = 0; it < 256; ++it) {
      const double mid = 0.5 * (a + z);
      if (mid <= a || mid >= z || z - a <= 4.0 * DBL_EPSILON * std::max(std::fabs(a), std::fabs(z))) break;
      if (below(mid) > j)
        z = mid;
      else
        a = mid;
    }
    return 0.5 * (a + z);
  };
  if (tmin) *tmin = kth(0);
  if (tmax) *tmax = kth(m - 1);
  for (int64_t i = 0; i < count; ++i) top[i] = i < m ? kth(m - 1 - i) : NAN;
}

}  // namespace gdml

namespace gdml {

namespace {

// tau_i = sum_j U_ij^2 max(w_j, 0) / (max(w_j, 0) + lam): the exact ridge leverage scores
// diag(K (K + lam I)^-1) from K = U diag(w) U^T (U column-major, thread i walks row i)
__global__ void rls_from_eigen_kernel(const double* __restrict__ U, const double* __restrict__ w, int64_t n, double lam,
                                      double* __restrict__ tau) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    const double wj = fmax(w[j], 0.0);
    const double u = U[j * n + i];
    s = fma(u * u, wj / (wj + lam), s);
  }
  tau[i] = s;
}

// out[a] = sum of in[a * per .. a * per + per - 1], in index order (one thread per group)
__global__ void group_sums_kernel(const double* __restrict__ in, int64_t groups, int per, double* __restrict__ out) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= groups) return;
  double s = 0.0;
  for (int c = 0; c < per; ++c) s += in[a * per + c];
  out[a] = s;
}

}  // namespace

void launch_rls_from_eigen(const double* U, const double* w, int64_t n, double lam, double* tau, cudaStream_t st) {
  { rls_from_eigen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, w, n, lam, tau); count_launch(); }
}

void launch_group_sums(const double* in, int64_t groups, int per, double* out, cudaStream_t st) {
  { group_sums_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(in, groups, per, out); count_launch(); }
}

}  // namespace gdml
