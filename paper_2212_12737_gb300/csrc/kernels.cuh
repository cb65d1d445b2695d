// Internal launcher declarations shared by the libgdml translation units.
#pragma once

#include <cuda.h>

#include <functional>
#include <string>

#include "common.cuh"

namespace gdml {

// scalar slots of the PCG state (device array of doubles)
enum { SC_RHO = 0, SC_PQ = 1, SC_RR = 2, SC_RHO_NEW = 3, SC_YY = 4, SC_TOL2 = 5, SC_COUNT = 8 };
// integer control words of the PCG loop (device int64 array); IC_HCAP: how many iterations of
// the running loop may record their CG coefficients (0: none)
enum { IC_ITER = 0, IC_MAXIT = 1, IC_HCAP = 2, IC_COUNT = 4 };

// geom.cu
void launch_desc_jac(const double* R, int64_t M, int N, int D, double* X, double* G, cudaStream_t st);
void launch_center(const double* X, int64_t M, int D, double* Xc, cudaStream_t st);
void launch_dist_tab(const double* X, int64_t M, int D, double c, double* S, double* A, int64_t ldA,
                     cudaStream_t st);
// kernel columns in double-float (DF64/OZAKI contexts): X2, G2 the float-pair copies of X, G;
// false (nothing launched) when the per-warp staging of 5 D float pairs does not fit in 200 KB
// or ncols > 65535
bool launch_kcol_df(const int64_t* cols, int64_t ncols, const float2* X2, const float2* G2, const double* S,
                    const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                    const int* stop_flag, cudaStream_t st);
// many kernel columns at once in double-float (the Nystrom factor's K_nk); false (nothing
// launched) when geometry a's operands and the per-warp scratch do not fit in 200 KB
bool launch_kcol_bulk_df(const int64_t* cols, int64_t ncols, const float2* X2, const float2* G2, const double* S,
                         const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                         cudaStream_t st);
// permutational symmetries (pis, pinv: S x D descriptor-entry permutations of the group)
void launch_sym_gather(const double* in, int64_t M, int D, const int* pis, int S, const double* xcB, double* out,
                       double* t, cudaStream_t st);
void launch_kdiag_sym(const double* X, const double* G, int64_t M, int N, int D, const int* pis, const int* pinv,
                      int S, double c, double* diag, cudaStream_t st);
bool launch_kcol_sym(const int64_t* cols, int64_t ncols, const double* X, const double* G, const double* Stab,
                     const double* Atab, int64_t ldA, int64_t M, int64_t MB, int N, int D, const int* pis,
                     const int* pinv, int S, double c, double* out, int64_t ldo, const int* stop_flag,
                     cudaStream_t st);
// each double of x as the float pair (hi, lo)
void launch_split_df(const double* x, int64_t count, float2* out, cudaStream_t st);
void launch_kdiag(const double* G, int64_t M, int N, int D, double c, double* diag, cudaStream_t st);
void launch_proj(const double* G, const double* Xc, const double* v, int64_t M, int N, int D, double* W,
                 int64_t ldW, double* t, cudaStream_t st);
void launch_beta(const double* T, const double* S, const double* t, int64_t M, double c, double* Pb,
                 int64_t ldP, double* rowsum, cudaStream_t st);
// beta for `rows` rows of T, S (row stride M) against the M training columns
void launch_beta_rows(const double* T, const double* S, const double* t, int64_t rows, int64_t M, double c,
                      double* Pb, int64_t ldP, double* rowsum, cudaStream_t st);
// force prediction: query-vs-training S, A tables, and query descriptors on the training centre
void launch_dist_tab_cross(const double* Xq, int64_t Q, const double* X, int64_t M, int D, double c, double* S,
                           double* A, int64_t ldA, cudaStream_t st);
void launch_center_like(const double* Xq, int64_t Q, int D, const double* X, const double* Xc, double* Xqc,
                        cudaStream_t st);
template <typename TU>
void launch_backproj(const TU* U, int64_t ldU, int splits, int64_t split_stride, const double* rowsum,
                     const double* Xc, const double* G, const double* v, int64_t M, int N, int D, double lam,
                     int add_lambda, double* out, cudaStream_t st);
void launch_kcol(const int64_t* cols, int64_t ncols, const double* X, const double* G, const double* S,
                 const double* A, int64_t ldA, int64_t M, int N, int D, double c, double* out, int64_t ldo,
                 const int* stop_flag, cudaStream_t st);

// dgemm.cu
template <typename TA, typename TB>
void launch_dgemm(bool nt, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t lda,
                  const TB* B, int64_t ldb, double beta, double* C, int64_t ldc, bool lower_only,
                  cudaStream_t st, int splits = 1, int64_t split_stride = 0);
int dgemm_splits(int64_t M, int64_t N, int64_t K);
// double-float (FP32-pair) GEMM, same layouts as launch_dgemm with alpha = 1, beta = 0
void launch_dfgemm(bool nt, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double* C, int64_t ldc, cudaStream_t st, int splits = 1, int64_t split_stride = 0);

// linalg.cu
void cholesky_inplace(double* A, int64_t k, int* status, cudaStream_t st);
void trsm_left_lower(const double* Lkk, int64_t k, double* Bm, int64_t nrhs, cudaStream_t st, bool lower_rhs = false);
void add_diag(double* A, int64_t lda, int64_t k, double eps, cudaStream_t st);

// woodbury.cu
// C: full symmetric k x k (lambda I + L^T L); t must hold 3k doubles (t, u = C^-1 t, residual)
template <typename TL>
void woodbury_apply(const TL* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                    const double* r, double* z, double* part, double* t, cudaStream_t st);
void mirror_lower(double* A, int64_t k, cudaStream_t st);
// DF64 contexts: FP32-stored L_k, double-float accumulation; C and Cinv hold float
// pairs (split_df_inplace); t holds 6k doubles (t, u, e and three float-pair vectors)
void split_df_inplace(double* a, int64_t count, cudaStream_t st);
// TMA-staged passes over the FP32 factor (n x k, column j at L + j n); valid only for
// n % 4 == 0
struct WsPlan {
  bool ok = false;
  const float* L = nullptr;
  int64_t n = 0, k = 0, nch = 0, nru = 0;
  int rc = 0, grid = 0;                 // L u pass: chunks of rc rows
  int ru = 0, ncr = 0, cpr = 0, grid_t = 0;  // L^T r pass: units of ru rows x cpr columns
  CUtensorMap map;   // box rc rows x (32 * 128 / rc) columns
  CUtensorMap mapT;  // box 256 rows x 16 columns
};
// fills plan for L (plan.ok = false where the staged passes do not apply: n % 4 != 0, k = 0,
// or the CUDA driver rejects the map); rows: 128 or 256 to force the chunk size, else automatic
void ws_plan(WsPlan& plan, const float* L, int64_t n, int64_t k, int rows = 0);
// whether this driver captures cooperative launches into graphs (checked once per process,
// outside any capture; the fused Woodbury core needs it)
bool coop_graph_capture_ok();
// bar: two zeroed words (the fused core's grid barrier; nullptr: separate launches for the
// k-vector steps)
void woodbury_apply_df(const float* L, int64_t n, int64_t k, const double* C, const double* Cinv, double lam,
                       const double* r, double* z, double* part, double* t, float2* rs, const WsPlan* plan,
                       int* err, unsigned* bar, cudaStream_t st);
// the two L passes alone (test hook): t = L^T r and z = (r - L u) / lambda, staged (plan) or
// register-streamed (plan == nullptr); part: woodbury_part_size(n, k) doubles, t2: k float pairs
void df_passes(const float* L, int64_t n, int64_t k, const double* r, const double* u, double lam, double* t,
               double* z, double* part, float2* rs, float2* t2, float2* u2, const WsPlan* plan, int* err,
               cudaStream_t st);
void to_float(const double* a, int64_t n, float* b, cudaStream_t st);
void widen_float(const float* a, int64_t n, double* b, cudaStream_t st);
// lower-triangle-only double-float SYRK of an FP32 matrix: C = A A^T, A (k x n row-major, ld)
void launch_dfsyrk(int64_t k, int64_t n, const float* A, int64_t lda, double* C, int64_t ldc, cudaStream_t st);
void transpose_square(const double* A, int64_t k, double* At, cudaStream_t st);
void set_identity(double* A, int64_t k, cudaStream_t st);
int64_t woodbury_part_size(int64_t n, int64_t k);

// the bounded-wait limit of each translation unit with tcgen05 / TMA pipelines (test hook)
cudaError_t set_wait_limit_oz(uint32_t polls);
cudaError_t set_wait_limit_tc(uint32_t polls);
cudaError_t set_wait_limit_wb(uint32_t polls);
cudaError_t set_wait_limit_pc(uint32_t polls);
uint32_t tc_default_wait_limit();
void launch_check_finite(const double* a, int64_t count, int* flag, cudaStream_t st);

// cg.cu
void launch_dot(const double* x, const double* y, int64_t n, double* partial, unsigned* ticket, double* out,
                cudaStream_t st);
// x += gamma p; r -= gamma q; sc[RR] = r.r (dot_kernel's partition and order); check != 0: also
// the end-of-iteration test of the graph-captured loop (conditional handle h).  hist (may be
// null): hist[2 j] = gamma of loop iteration j while j < ictl[IC_HCAP]
void launch_update_xr_rr(double* x, double* r, const double* p, const double* q, int64_t n, double* sc, int* status,
                         double* partial, unsigned* ticket, int64_t* ictl, cudaGraphConditionalHandle h, int check,
                         double* hist, cudaStream_t st);
// p = z + (rho_new / rho) p; rho <- rho_new.  hist (may be null): hist[2 j + 1] = rho_new / rho of
// loop iteration j = ictl[IC_ITER] - 1 while j < ictl[IC_HCAP]
void launch_update_p_rho(double* p, const double* z, int64_t n, double* sc, unsigned* ticket, const int64_t* ictl,
                         double* hist, cudaStream_t st);
void launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st);
cudaError_t add_pcg_gate_node(cudaGraph_t g, cudaGraphNode_t* node, const double* sc, const int64_t* ictl,
                              cudaGraphConditionalHandle h);

// spectrum.cu
// L[:, j] = U[:, n - 1 - j] sqrt(max(w[n - 1 - j], 0)) for j < k: the factor of the rank-k SVD
// preconditioner from an ascending eigendecomposition (U column-major n x n, L column-major)
void launch_svd_factor(const double* U, const double* w, int64_t n, int64_t k, double* L, cudaStream_t st);
// dense symmetric eigendecomposition in place (A column-major n x n, lower triangle read;
// eigenvectors overwrite A, ascending eigenvalues in w).  Returns an empty string on success,
// else what failed.
std::string eigh_dense(double* A, int64_t n, double* w, cudaStream_t st);
// exact ridge leverage scores tau_i = sum_j U_ij^2 w_j^+ / (w_j^+ + lam) from an ascending
// eigendecomposition (U column-major n x n)
void launch_rls_from_eigen(const double* U, const double* w, int64_t n, double lam, double* tau, cudaStream_t st);
// out[a] = sum of the per consecutive entries of group a (index order)
void launch_group_sums(const double* in, int64_t groups, int per, double* out, cudaStream_t st);
// Ritz values of the Lanczos matrix T_m of m CG steps (gamma_j, beta_j; see gdml_pcg_spectrum):
// its smallest and largest eigenvalue and its `count` largest in descending order
void lanczos_ritz(const double* gamma, const double* beta, int64_t m, int64_t count, double* top, double* tmin,
                  double* tmax);

// select.cu
int64_t select_scratch_len(int64_t n);
void select_uniform(int64_t n, int64_t k, uint64_t seed, uint32_t stream, uint64_t* key, int64_t* idx,
                    int64_t* out, cudaStream_t st);
void select_weighted(int64_t n, int64_t k, uint64_t seed, uint32_t stream, const double* tau, uint64_t* key,
                     int64_t* idx, int64_t* out, cudaStream_t st);

// mlp.cu
void launch_column_weights(const double* score, const double* diag, int64_t n, int B3, double* w, cudaStream_t st);
void launch_destandardize(const float* out, int64_t B, float ym, float ysd, double* dst, cudaStream_t st);

// pivchol.cu
struct PivState {
  double lmm;   // l_{pivot, m} = sqrt(d_pivot)
  double ilmm;  // 1 / lmm
  int64_t piv;
  int64_t rank;
  int stop;
  int pad;
};
struct ArgMaxPart {
  double v;
  int64_t pos;
  double sum;
};
struct PivCholArgs {
  int64_t n, k;
  double* d;
  int64_t* perm;
  unsigned char* chosen;
  int64_t* pivots;
  double* trace;
  PivState* ps;
  ArgMaxPart* part;
  unsigned* ticket;
  double* col;
  std::function<void(const int64_t*, double*, const int*, cudaStream_t)> get_col;
  // DF64 form only: pivot-row gather (k floats) and Schur partials (pivchol_schur_groups() * n pairs)
  float* prow = nullptr;
  float2* schur = nullptr;
  int64_t* posof = nullptr;  // inverse of perm (position of each index)
  int* err = nullptr;        // error word of the staged Schur pass
};
int pivchol_schur_groups();
template <typename TL>
void pivchol_run(const PivCholArgs& a, TL* L, cudaStream_t st);
// Alg. 1 with FP32-stored L and double-float Schur sums (DF64 contexts)
void pivchol_run_df(const PivCholArgs& a, float* L, cudaStream_t st);
int pivchol_part_blocks();

}  // namespace gdml
