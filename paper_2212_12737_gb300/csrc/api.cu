// C ABI of libgdml (declared in include/gdml.h): context, matvec,
// preconditioner build / apply and the PCG solve.  Every step runs in the
// kernels of this library; the host only sequences launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "oz.cuh"
#include "tc.cuh"
#include "../../include/gdml_testing.h"

namespace gdml {

static thread_local std::string g_msg;
static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
gdml_status fail(gdml_status st, const std::string& msg) {
  g_msg = msg;
  return st;
}
const std::string& last_msg() { return g_msg; }
void clear_msg() { g_msg.clear(); }

int num_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace gdml

using namespace gdml;

// iterations of a solve whose CG coefficients are kept for gdml_pcg_spectrum (320 KB per context)
constexpr int64_t kHistCap = 20000;
// largest n of the SVD preconditioner: dense K (8 n^2 bytes) and syevd's workspace of ~2 n^2
// doubles (its size is a 32-bit int)
constexpr int64_t kSvdMaxN = 24576;

struct gdml_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  int64_t M = 0, n = 0;
  int N = 0, D = 0, B = 0;
  double sigma = 0, lam = 0, c = 0;
  int precision = GDML_FP64;
  double inner_rtol = 1e-4;
  int last_outer = 0;
  int inner_lev = 7;       // OZAKI: slice levels of the PCG loop's matvec (gdml_set_inner_levels)
  int last_restarts = 0;   // true-residual restarts of the last pcg_core call
  std::string err;
  std::vector<void*> allocs;

  // kernel state
  double* R = nullptr;    // M*N*3
  double* X = nullptr;    // M*D
  double* G = nullptr;    // M*D*3
  double* S = nullptr;    // M*M
  double* P64 = nullptr;  // M x 2M : [A | beta]
  double* V64 = nullptr;  // 2M x D : [W ; Xc]
  double* T = nullptr;    // M*M
  double* tb = nullptr;   // M
  double* rowsum = nullptr;
  double* U = nullptr;  // splits_cap x M x D (split-K partials of the second contraction)
  int splitsU = 1;
  int splits_cap = 1;
  double* diag = nullptr;  // n
  float2* X2 = nullptr;    // M*D: X as float pairs (DF64/OZAKI kernel columns)
  float2* G2 = nullptr;    // M*D*3: G as float pairs
  // permutational symmetries (sGDML): Ssym atom permutations of a group; the training side of
  // the kernel then has MB = M Ssym rows, row b Ssym + q = P_q applied to geometry b
  int Ssym = 1;
  int64_t MB = 0;
  int* pis = nullptr;     // Ssym x D: pi_q(p)
  int* pinv = nullptr;    // Ssym x D: pi_q^-1(p)
  double* XB = nullptr;   // MB x D: P_q x_b (X itself when Ssym == 1)
  double* XcA = nullptr;  // M x D: centred descriptors of the rows (the bottom of V64 when Ssym == 1)
  double* Wa = nullptr;   // M x D: w_a = J_a v_a (Ssym > 1; the top of V64 holds the training side)
  double* Xc() const { return XcA; }
  double* XcB() const { return V64 + MB * D; }  // MB x D: the training side's centred descriptors
  TcMatvec tc;  // tensor-core matvec state (TF32/BF16 contexts)
  OzMatvec oz;  // sliced-BF16 tensor-core matvec state (OZAKI contexts)

  // preconditioner
  int64_t k = 0;  // rank built (0: none)
  double jitter = 0;
  double* L = nullptr;    // n x k col-major
  float* Lf = nullptr;    // n x k col-major FP32 copy used by DF64 contexts
  double* rsplit = nullptr;  // n float pairs (DF64 apply)
  double* LC = nullptr;   // k x k lower (row-major): Cholesky factor of C = lambda I + L^T L
  double* Cinv = nullptr; // k x k: C^-1 = L_C^-T L_C^-1 (formed once per build)
  double* Cfull = nullptr; // k x k: C itself (for the refinement step of the apply)
  double* wpart = nullptr;
  double* wt = nullptr;
  WsPlan ws;              // TMA-staged passes over Lf (DF64/OZAKI contexts)
  int* werr = nullptr;    // error word of the staged passes
  unsigned* wbar = nullptr;  // [2] grid-barrier counters of the fused Woodbury core (kept zero)
  int64_t cap_k = 0;

  // PCG state
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr, *ys = nullptr;
  double* sc = nullptr;       // SC_COUNT scalars
  double* partial = nullptr;  // dot partials
  unsigned* ticket = nullptr;
  int* status = nullptr;      // device status word
  double* hsc = nullptr;      // pinned host mirror of scalars
  int64_t* ictl = nullptr;    // device loop control (IC_*)
  int64_t* hictl = nullptr;   // pinned host mirror
  // CG coefficients (gamma_j, beta_j) of the first CG run of the last gdml_pcg_solve: the Lanczos
  // matrix behind gdml_pcg_spectrum
  double* hist = nullptr;     // 2 * hist_cap doubles
  int64_t hist_cap = 0;
  int64_t hist_len = 0;       // iterations recorded
  bool hist_arm = false;      // the next pcg_core run records
  cudaStream_t cap = nullptr;             // private stream used only to capture graphs
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // PCG loop graphs: [0] context precision, [1] FP64
  int64_t gbody[2] = {0, 0};                       // kernels per captured iteration
};

namespace {

gdml_status ctx_fail(gdml_ctx* c, gdml_status st, const std::string& m) {
  if (c) c->err = m;
  return fail(st, m);
}

template <typename T>
gdml_status dalloc(gdml_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return ctx_fail(c, GDML_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return GDML_OK;
}

void dfree(gdml_ctx* c, void* p) {
  if (!p) return;
  for (auto& a : c->allocs)
    if (a == p) {
      cudaFree(a);
      a = nullptr;
    }
}

#define TRY(x)                          \
  do {                                  \
    gdml_status _s = (x);               \
    if (_s != GDML_OK) return _s;       \
  } while (0)
#define CTRY(c, expr)                                                                           \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess) return ctx_fail(c, GDML_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

gdml_status check_launch(gdml_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(c, GDML_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return GDML_OK;
}

// FP32-stored L_k with double-float sums (DF64 and OZAKI contexts)
inline bool df_precond(const gdml_ctx* c) { return c->precision == GDML_DF64 || c->precision == GDML_OZAKI; }
// FP64-class matvec: plain PCG with true-residual restarts, no refinement loop
inline bool direct_pcg(const gdml_ctx* c) { return c->precision != GDML_TF32 && c->precision != GDML_BF16; }

// ----------------------------------------------------------------- matvec
gdml_status matvec_fp64(gdml_ctx* c, const double* v, double* out, int add_lambda) {
  const int64_t M = c->M;
  const int D = c->D;
  cudaStream_t st = c->st;
  if (c->Ssym > 1) {  // the same steps with the training side of MB = M S rows
    const int64_t MB = c->MB;
    double* WB = c->V64;  // [W_B ; Xc_B]
    launch_proj(c->G, c->XcA, v, M, c->N, D, c->Wa, D, c->tb, st);
    launch_sym_gather(c->Wa, M, D, c->pis, c->Ssym, c->XcB(), WB, c->tb, st);
    launch_dgemm<double, double>(true, M, MB, D, 1.0, c->XcA, D, WB, D, 0.0, c->T, MB, false, st);
    launch_beta_rows(c->T, c->S, c->tb, M, MB, c->c, c->P64 + MB, 2 * MB, c->rowsum, st);
    launch_dgemm<double, double>(false, M, D, 2 * MB, 1.0, c->P64, 2 * MB, c->V64, D, 0.0, c->U, D, false, st,
                                 c->splitsU, M * D);
    launch_backproj<double>(c->U, D, c->splitsU, M * D, c->rowsum, c->XcA, c->G, v, M, c->N, D, c->lam, add_lambda,
                            out, st);
    return check_launch(c, "matvec_fp64 (symmetries)");
  }
  double* W = c->V64;
  launch_proj(c->G, c->Xc(), v, M, c->N, D, W, D, c->tb, st);
  // T = Xc W^T
  launch_dgemm<double, double>(true, M, M, D, 1.0, c->Xc(), D, W, D, 0.0, c->T, M, false, st);
  launch_beta(c->T, c->S, c->tb, M, c->c, c->P64 + M, 2 * M, c->rowsum, st);
  // U = [A | beta] [W ; Xc]
  launch_dgemm<double, double>(false, M, D, 2 * M, 1.0, c->P64, 2 * M, c->V64, D, 0.0, c->U, D, false, st,
                               c->splitsU, M * D);
  launch_backproj<double>(c->U, D, c->splitsU, M * D, c->rowsum, c->Xc(), c->G, v, M, c->N, D, c->lam, add_lambda,
                          out, st);
  return check_launch(c, "matvec_fp64");
}

// Same steps as matvec_fp64 with both contractions in double-float arithmetic.
gdml_status matvec_df(gdml_ctx* c, const double* v, double* out, int add_lambda) {
  const int64_t M = c->M;
  const int D = c->D;
  cudaStream_t st = c->st;
  double* W = c->V64;
  launch_proj(c->G, c->Xc(), v, M, c->N, D, W, D, c->tb, st);
  launch_dfgemm(true, M, M, D, c->Xc(), D, W, D, c->T, M, st);
  launch_beta(c->T, c->S, c->tb, M, c->c, c->P64 + M, 2 * M, c->rowsum, st);
  launch_dfgemm(false, M, D, 2 * M, c->P64, 2 * M, c->V64, D, c->U, D, st, c->splitsU, M * D);
  launch_backproj<double>(c->U, D, c->splitsU, M * D, c->rowsum, c->Xc(), c->G, v, M, c->N, D, c->lam, add_lambda,
                          out, st);
  return check_launch(c, "matvec_df");
}

// lev: slice levels of an OZAKI context's matvec (7: the full, FP64-class product)
gdml_status matvec_any(gdml_ctx* c, const double* v, double* out, int add_lambda, bool force_fp64, int lev = 7) {
  if (force_fp64 || c->precision == GDML_FP64) return matvec_fp64(c, v, out, add_lambda);
  if (c->precision == GDML_DF64) return matvec_df(c, v, out, add_lambda);
  if (c->precision == GDML_OZAKI) {
    gdml_status s = oz_matvec(c->oz, c->G, c->G2, c->Xc(), v, out, add_lambda, c->lam, c->st, lev);
    if (s != GDML_OK) return ctx_fail(c, s, "sliced tensor-core matvec: " + last_msg());
    return check_launch(c, "matvec_oz");
  }
  gdml_status s = tc_matvec(c->tc, c->G, v, out, add_lambda, c->lam, c->st);
  if (s != GDML_OK) return ctx_fail(c, s, "tensor-core matvec: " + last_msg());
  return check_launch(c, "matvec_tc");
}

// ------------------------------------------------------------ preconditioner
__global__ void gather_kkk_kernel(const double* __restrict__ Knk, int64_t n, const int64_t* __restrict__ S,
                                  int64_t k, double* __restrict__ Kkk) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int64_t r = e / k, cc = e - r * k;
  Kkk[e] = Knk[cc * n + S[r]];
}

__global__ void col_sqnorm_kernel(const double* __restrict__ Z, int64_t k, int64_t n, double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t r = 0; r < k; ++r) {
    double v = Z[r * n + i];
    s = fma(v, v, s);
  }
  out[i] = s;
}

gdml_status read_status(gdml_ctx* c, int* h) {
  CTRY(c, cudaMemcpyAsync(h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  return GDML_OK;
}

// K[:, cols] (n x ncols, column-major) for the Nystrom factor: in double-float with each
// geometry's operands reused across the columns (DF64 / OZAKI contexts, whose preconditioner
// is FP32-stored), else in FP64
gdml_status get_cols(gdml_ctx* c, const int64_t* cols, int64_t ncols, double* out) {
  if (c->Ssym > 1) {
    if (!launch_kcol_sym(cols, ncols, c->X, c->G, c->S, c->P64, 2 * c->MB, c->M, c->MB, c->N, c->D, c->pis, c->pinv,
                         c->Ssym, c->c, out, c->n, nullptr, c->st))
      return ctx_fail(c, GDML_ERR_ARG, "kernel columns with symmetries: descriptor too long for shared memory");
    return check_launch(c, "kcol (symmetries)");
  }
  if (!(c->X2 && launch_kcol_bulk_df(cols, ncols, c->X2, c->G2, c->S, c->P64, 2 * c->M, c->M, c->N, c->D, c->c, out,
                                      c->n, c->st)))
    launch_kcol(cols, ncols, c->X, c->G, c->S, c->P64, 2 * c->M, c->M, c->N, c->D, c->c, out, c->n, nullptr, c->st);
  return check_launch(c, "kcol");
}

struct Scratch {
  gdml_ctx* c;
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) dfree(c, p);
  }
  template <typename T>
  gdml_status get(T** p, size_t count) {
    gdml_status s = dalloc(c, p, count);
    if (s == GDML_OK) ptrs.push_back(*p);
    return s;
  }
};

// In-place lower Cholesky of the k x k work matrix (copy of src) with the
// jitter rule of Eq. 5's factorisation: eps = 1e-14 tr/k, x10 up to 1e-6 tr/k.
gdml_status chol_jitter(gdml_ctx* c, const double* src, double* work, int64_t k, double* eps_out) {
  std::vector<double> hdiag(k);
  CTRY(c, cudaMemcpy2DAsync(hdiag.data(), sizeof(double), src, (k + 1) * sizeof(double), sizeof(double), k,
                            cudaMemcpyDeviceToHost, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  double tr = 0.0;
  for (double v : hdiag) tr += v;
  const double scale = tr / (double)k;
  double eps = 0.0;
  for (;;) {
    CTRY(c, cudaMemcpyAsync(work, src, k * k * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (eps > 0.0) add_diag(work, k, k, eps, c->st);
    CTRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
    cholesky_inplace(work, k, c->status, c->st);
    TRY(check_launch(c, "cholesky"));
    int h = 0;
    TRY(read_status(c, &h));
    if (h == 0) break;
    // the jitter scale tr/k must be positive (a nonzero PSD block has tr > 0); otherwise
    // no retry can help, and eps would stay 0 forever
    if (!(scale > 0.0) || !std::isfinite(scale))
      return ctx_fail(c, GDML_ERR_NOT_SPD, "Cholesky of the inducing block failed and tr/k is not positive");
    eps = (eps == 0.0) ? 1e-14 * scale : eps * 10.0;
    if (!(eps <= 1e-6 * scale * 1.0000001))
      return ctx_fail(c, GDML_ERR_NOT_SPD, "Cholesky of the inducing block failed even with jitter 1e-6 tr/k");
  }
  *eps_out = eps;
  return GDML_OK;
}

// L (k x n row-major = n x k col-major) <- Nystrom factor from columns S (Eq. 5).
// FP64 / DF64 contexts: forward substitution on the FP64 pipe.  OZAKI contexts: the same
// L_k = K_nk L_kk^-T as K_nk times the transposed triangular inverse of L_kk, on the sliced
// BF16 tensor cores (FP64-class products, accumulated over all of k in each tile); only the
// k x k inverse runs on the FP64 pipe.  On return `work` holds L_kk (lower, row-major).
gdml_status nystrom(gdml_ctx* c, const int64_t* S, int64_t k, double* L, double* Kkk, double* work,
                    double* eps_out) {
  TRY(get_cols(c, S, k, L));
  { gather_kkk_kernel<<<(unsigned)cdiv(k * k, 256), 256, 0, c->st>>>(L, c->n, S, k, Kkk); count_launch(); }
  TRY(check_launch(c, "gather_kkk"));
  TRY(chol_jitter(c, Kkk, work, k, eps_out));
  if (c->precision == GDML_OZAKI) {
    Scratch s{c, {}};
    double* Linv = nullptr;
    TRY(s.get(&Linv, (size_t)(k * k)));
    set_identity(Linv, k, c->st);
    trsm_left_lower(work, k, Linv, k, c->st, true);  // L_kk^-1 (lower triangular)
    TRY(check_launch(c, "inducing-block inverse"));
    gdml_status so = oz_gemm_tall(L, c->n, k, Linv, k, k, true, false, L, nullptr, c->st);
    if (so != GDML_OK) return ctx_fail(c, so, "sliced K_nk L_kk^-T: " + last_msg());
    return GDML_OK;
  }
  trsm_left_lower(work, k, L, c->n, c->st);  // rows of K_nk^T -> rows of L_k^T
  return check_launch(c, "trsm");
}

// LC <- chol(lambda I + L^T L) (Eq. 4); with Cinv, also C^-1 = L_C^-T L_C^-1
gdml_status woodbury_core(gdml_ctx* c, const double* L, int64_t k, double* LC, double* Cinv = nullptr,
                          double* Cfull = nullptr, const float* Lf = nullptr) {
  if (Lf && c->precision == GDML_OZAKI) {  // C from the FP32 factor on the sliced tensor cores
    gdml_status s = oz_syrk_lower(Lf, c->n, k, LC, k, c->st);
    if (s != GDML_OK) return ctx_fail(c, s, "sliced syrk: " + last_msg());
  } else if (c->precision == GDML_OZAKI) {  // C from the FP64 factor (columns = rows of L^T), sliced
    gdml_status s = oz_syrk_lower_f64(L, k, c->n, c->n, LC, k, c->st);
    if (s != GDML_OK) return ctx_fail(c, s, "sliced syrk: " + last_msg());
  } else if (Lf)  // DF64: C from the FP32-stored factor, exact products, double-float sums
    launch_dfsyrk(k, c->n, Lf, c->n, LC, k, c->st);
  else
    launch_dgemm<double, double>(true, k, k, c->n, 1.0, L, c->n, L, c->n, 0.0, LC, k, true, c->st);
  add_diag(LC, k, k, c->lam, c->st);
  if (Cfull) {
    CTRY(c, cudaMemcpyAsync(Cfull, LC, k * k * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    mirror_lower(Cfull, k, c->st);
  }
  CTRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
  cholesky_inplace(LC, k, c->status, c->st);
  TRY(check_launch(c, "woodbury_core"));
  int h = 0;
  TRY(read_status(c, &h));
  if (h) return ctx_fail(c, GDML_ERR_NOT_SPD, "Cholesky of lambda I + L^T L failed at column " + std::to_string(h - 1));
  if (Cinv) {
    Scratch s{c, {}};
    double *X = nullptr, *Xt = nullptr;
    TRY(s.get(&X, (size_t)(k * k)));
    TRY(s.get(&Xt, (size_t)(k * k)));
    set_identity(X, k, c->st);
    trsm_left_lower(LC, k, X, k, c->st, true);  // X = L_C^-1 (lower triangular)
    transpose_square(X, k, Xt, c->st);
    if (df_precond(c)) {  // X^T X on the sliced tensor cores (FP64-class), lower triangle mirrored
      TRY(check_launch(c, "woodbury inverse"));
      gdml_status so = oz_syrk_lower_f64(Xt, k, k, k, Cinv, k, c->st);
      if (so != GDML_OK) return ctx_fail(c, so, "sliced X^T X: " + last_msg());
      mirror_lower(Cinv, k, c->st);
    } else {
      launch_dgemm<double, double>(true, k, k, k, 1.0, Xt, k, Xt, k, 0.0, Cinv, k, false, c->st);  // X^T X
    }
    TRY(check_launch(c, "woodbury inverse"));
    if (Lf && Cfull) {  // DF64 apply: the two k x k operators as float pairs
      split_df_inplace(Cinv, k * k, c->st);
      split_df_inplace(Cfull, k * k, c->st);
      TRY(check_launch(c, "woodbury split"));
    }
    CTRY(c, cudaStreamSynchronize(c->st));
  }
  return GDML_OK;
}

gdml_status ensure_precond_buffers(gdml_ctx* c, int64_t k) {
  if (k <= c->cap_k) return GDML_OK;
  dfree(c, c->L);
  dfree(c, c->LC);
  dfree(c, c->wpart);
  dfree(c, c->wt);
  dfree(c, c->Cinv);
  dfree(c, c->Cfull);
  dfree(c, c->Lf);
  c->L = c->LC = c->wpart = c->wt = c->Cinv = c->Cfull = nullptr;
  c->Lf = nullptr;
  c->cap_k = 0;
  TRY(dalloc(c, &c->L, (size_t)(c->n * k)));
  if (df_precond(c)) TRY(dalloc(c, &c->Lf, (size_t)(c->n * k)));
  TRY(dalloc(c, &c->LC, (size_t)(k * k)));
  TRY(dalloc(c, &c->Cinv, (size_t)(k * k)));
  TRY(dalloc(c, &c->Cfull, (size_t)(k * k)));
  TRY(dalloc(c, &c->wpart, (size_t)woodbury_part_size(c->n, k)));
  TRY(dalloc(c, &c->wt, (size_t)(6 * k)));
  c->cap_k = k;
  return GDML_OK;
}



// Nystrom estimate of the ridge leverage scores from a uniform pilot set of
// size k (Philox stream 1): B = K_nS L_S^-T, tau_i = |L_C^-1 b_i|^2 with
// L_C L_C^T = B^T B + lambda I (Sec. 3, "Leverage score sampling").
// Overwrites the context's L / LC buffers (capacity >= k).
gdml_status rls_estimate(gdml_ctx* c, int64_t k, uint64_t seed, int64_t* S, double* Kkk, double* work,
                         uint64_t* key, int64_t* idx, double* tau) {
  const int64_t n = c->n;
  select_uniform(n, k, seed, 1u, key, idx, S, c->st);
  double eps0 = 0.0;
  TRY(nystrom(c, S, k, c->L, Kkk, work, &eps0));  // B (n x k col-major)
  TRY(woodbury_core(c, c->L, k, c->LC));          // chol(B^T B + lambda I)
  if (c->precision == GDML_OZAKI) {
    // tau_i = |L_C^-1 b_i|^2: the row square sums of B X^T with X = L_C^-1 (lower
    // triangular, formed on the FP64 pipe), the product on the sliced tensor cores
    set_identity(work, k, c->st);
    trsm_left_lower(c->LC, k, work, k, c->st, true);
    TRY(check_launch(c, "rls core inverse"));
    gdml_status so = oz_gemm_tall(c->L, n, k, work, k, k, true, true, tau, nullptr, c->st);
    if (so != GDML_OK) return ctx_fail(c, so, "sliced leverage scores: " + last_msg());
    return GDML_OK;
  }
  trsm_left_lower(c->LC, k, c->L, n, c->st);       // Z = L_C^-1 B^T
  { col_sqnorm_kernel<<<(unsigned)cdiv(n, 256), 256, 0, c->st>>>(c->L, k, n, tau); count_launch(); }
  return check_launch(c, "rls scores");
}

// reads (and clears) the error word of the staged Woodbury passes; synchronises the stream
gdml_status ws_check(gdml_ctx* c) {
  int h = 0;
  CTRY(c, cudaMemcpyAsync(&h, c->werr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  if (h) {
    (void)cudaMemsetAsync(c->werr, 0, sizeof(int), c->st);
    return ctx_fail(c, GDML_ERR_TIMEOUT, "a staged Woodbury pass wait timed out (code " + std::to_string(h) + ")");
  }
  return GDML_OK;
}

// ------------------------------------------------------------------ PCG
gdml_status apply_precond(gdml_ctx* c, const double* r, double* z) {
  if (c->k == 0) {
    CTRY(c, cudaMemcpyAsync(z, r, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return GDML_OK;
  }
  if (df_precond(c))
    woodbury_apply_df(c->Lf, c->n, c->k, c->Cfull, c->Cinv, c->lam, r, z, c->wpart, c->wt,
                      reinterpret_cast<float2*>(c->rsplit), &c->ws, c->werr, c->wbar, c->st);
  else
    woodbury_apply<double>(c->L, c->n, c->k, c->Cfull, c->Cinv, c->lam, r, z, c->wpart, c->wt, c->st);
  return check_launch(c, "woodbury_apply");
}

gdml_status dot(gdml_ctx* c, const double* a, const double* b, int slot) {
  launch_dot(a, b, c->n, c->partial, c->ticket, c->sc + slot, c->st);
  return GDML_OK;
}

gdml_status fetch_scalars(gdml_ctx* c) {
  CTRY(c, cudaMemcpyAsync(c->hsc, c->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  return GDML_OK;
}

void drop_graphs(gdml_ctx* c) {
  for (auto& g : c->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Body of one PCG iteration, launched on c->st (captured into the WHILE node):
//   q = K_lam p; pq = p.q; x += g p, r -= g q; rr = r.r; check; z = P^-1 r;
//   rho' = r.z; p = z + (rho'/rho) p; rho = rho'.
gdml_status pcg_body(gdml_ctx* c, double* x, bool fp64_mv, cudaGraphConditionalHandle h) {
  const int64_t n = c->n;
  TRY(matvec_any(c, c->p, c->q, 1, fp64_mv, c->inner_lev));
  TRY(dot(c, c->p, c->q, SC_PQ));
  // x, r update fused with r.r and the loop's end test
  launch_update_xr_rr(x, c->r, c->p, c->q, n, c->sc, c->status, c->partial, c->ticket, c->ictl, h, 1, c->hist, c->st);
  TRY(apply_precond(c, c->r, c->z));
  TRY(dot(c, c->r, c->z, SC_RHO_NEW));
  launch_update_p_rho(c->p, c->z, n, c->sc, c->ticket, c->ictl, c->hist, c->st);
  return check_launch(c, "pcg body");
}

// Capture the PCG loop once as a graph with a conditional WHILE node whose
// body is one iteration; the fused x, r update (with r.r) ends the loop on the device.
gdml_status pcg_graph(gdml_ctx* c, double* x, bool fp64_mv, cudaGraphExec_t* out) {
  const int slot = fp64_mv && c->precision != GDML_FP64 ? 1 : 0;
  if (c->gexec[slot]) {
    *out = c->gexec[slot];
    return GDML_OK;
  }
  if (!c->cap) CTRY(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CTRY(c, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(c->cap, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return ctx_fail(c, GDML_ERR_CUDA, std::string("building the PCG graph: ") + cudaGetErrorString(e));
  }
  cudaStream_t user = c->st;
  c->st = c->cap;
  const int64_t before = launch_count();
  gdml_status bs = pcg_body(c, x, fp64_mv, h);
  const int64_t body_n = launch_count() - before;
  count_launch(-body_n);  // captured, not executed
  c->gbody[slot] = body_n;
  c->st = user;
  cudaGraph_t body = nullptr;
  e = cudaStreamEndCapture(c->cap, &body);
  if (bs != GDML_OK || e != cudaSuccess) {
    cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return bs != GDML_OK ? bs : ctx_fail(c, GDML_ERR_CUDA, std::string("capturing the PCG body: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return ctx_fail(c, GDML_ERR_CUDA, std::string("instantiating the PCG graph: ") + cudaGetErrorString(e));
  c->gexec[slot] = ex;
  *out = ex;
  return GDML_OK;
}

// PCG on K_lambda x = b (x updated in place; the graph is bound to this x).
// Stops when the recurrence residual |r| <= tol_abs; with check_true, the
// true residual is recomputed in FP64 and CG restarts from x if it drifted.
// *iters = iterations used; *res_out = final |r| (the true one if check_true).
gdml_status pcg_core(gdml_ctx* c, const double* b, double* x, double tol_abs, int64_t max_iter, bool fp64_mv,
                     bool check_true, int max_restarts, int64_t* iters, double* res_out) {
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  int64_t it = 0;
  int restarts = 0;
  *iters = 0;
  TRY(matvec_any(c, x, c->r, 1, fp64_mv));  // r = b - K x
  launch_axpby(c->r, b, 1.0, -1.0, n, st);
  TRY(dot(c, c->r, c->r, SC_RR));
  TRY(fetch_scalars(c));
  double res = std::sqrt(c->hsc[SC_RR]);
  gdml_status out = GDML_OK;
  while (res > tol_abs && it < max_iter) {
    TRY(apply_precond(c, c->r, c->z));
    CTRY(c, cudaMemcpyAsync(c->p, c->z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TRY(dot(c, c->r, c->z, SC_RHO));
    c->hictl[IC_ITER] = 0;
    c->hictl[IC_MAXIT] = max_iter - it;
    c->hictl[IC_HCAP] = c->hist_arm ? std::min<int64_t>(c->hist_cap, max_iter - it) : 0;
    c->hsc[SC_TOL2] = tol_abs * tol_abs;
    CTRY(c, cudaMemcpyAsync(c->ictl, c->hictl, 3 * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CTRY(c, cudaMemcpyAsync(c->sc + SC_TOL2, c->hsc + SC_TOL2, sizeof(double), cudaMemcpyHostToDevice, st));
    CTRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), st));
    cudaGraphExec_t ex = nullptr;
    TRY(pcg_graph(c, x, fp64_mv, &ex));
    CTRY(c, cudaGraphLaunch(ex, st));
    CTRY(c, cudaMemcpyAsync(c->hictl, c->ictl, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int hst = 0;
    CTRY(c, cudaMemcpyAsync(&hst, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(fetch_scalars(c));  // synchronises
    it += c->hictl[IC_ITER];
    count_launch(c->hictl[IC_ITER] * c->gbody[fp64_mv && c->precision != GDML_FP64 ? 1 : 0]);
    if (c->hist_arm) {  // only the first run of a solve forms one Lanczos process
      c->hist_len = std::min(c->hictl[IC_ITER], c->hist_cap);
      c->hist_arm = false;
    }
    res = std::sqrt(c->hsc[SC_RR]);
    if (hst || !std::isfinite(res)) {
      // an inner solve of the refinement stops at the last good iterate (its
      // operator is only approximately SPD); a plain FP64 solve reports it
      if (!check_true && std::isfinite(res)) break;
      out = ctx_fail(c, GDML_ERR_BREAKDOWN, "PCG breakdown: p^T K p <= 0 or a non-finite residual");
      break;
    }
    if (!check_true) break;
    TRY(matvec_any(c, x, c->r, 1, true));  // true residual in FP64
    launch_axpby(c->r, b, 1.0, -1.0, n, st);
    TRY(dot(c, c->r, c->r, SC_RR));
    TRY(fetch_scalars(c));
    res = std::sqrt(c->hsc[SC_RR]);
    if (res <= tol_abs || restarts >= max_restarts) break;
    ++restarts;
  }
  *iters = it;
  *res_out = res;
  c->last_restarts = restarts;
  return out;
}

gdml_status validate(const gdml_ctx* c) {
  if (!c) return fail(GDML_ERR_ARG, "null context");
  return GDML_OK;
}

}  // namespace

namespace {

// The symmetries must be a group of atom permutations (identity included, closed under
// composition): only then is K symmetric positive semi-definite.  pis / pinv (S x D) hold the
// descriptor-entry permutation of each element and its inverse.
gdml_status check_symmetry_group(const int32_t* perms, int S, int N, std::vector<int>& pis, std::vector<int>& pinv) {
  if (!perms || S < 1 || S > 256) return fail(GDML_ERR_ARG, "symmetries: need 1 <= S <= 256 permutations");
  std::vector<std::vector<int>> P(S, std::vector<int>(N));
  bool has_id = false;
  for (int q = 0; q < S; ++q) {
    std::vector<char> seen(N, 0);
    bool id = true;
    for (int i = 0; i < N; ++i) {
      const int v = perms[(int64_t)q * N + i];
      if (v < 0 || v >= N || seen[v]) return fail(GDML_ERR_ARG, "symmetries: row " + std::to_string(q) + " is not a permutation of the atoms");
      seen[v] = 1;
      P[q][i] = v;
      id = id && v == i;
    }
    has_id = has_id || id;
    for (int r = 0; r < q; ++r)
      if (P[r] == P[q]) return fail(GDML_ERR_ARG, "symmetries: permutation " + std::to_string(q) + " is listed twice");
  }
  if (!has_id) return fail(GDML_ERR_ARG, "symmetries: the identity permutation must be included");
  std::vector<int> comp(N);
  for (int q1 = 0; q1 < S; ++q1)
    for (int q2 = 0; q2 < S; ++q2) {
      for (int i = 0; i < N; ++i) comp[i] = P[q1][P[q2][i]];
      bool found = false;
      for (int r = 0; r < S && !found; ++r) found = P[r] == comp;
      if (!found) return fail(GDML_ERR_ARG, "symmetries: the permutations are not closed under composition (not a group)");
    }
  const int D = N * (N - 1) / 2;
  pis.assign((size_t)S * D, 0);
  pinv.assign((size_t)S * D, 0);
  for (int q = 0; q < S; ++q)
    for (int i = 1; i < N; ++i)
      for (int j = 0; j < i; ++j) {
        const int p = i * (i - 1) / 2 + j;
        const int a = P[q][i], b = P[q][j];
        const int hi = std::max(a, b), lo = std::min(a, b);
        const int pp = hi * (hi - 1) / 2 + lo;
        pis[(size_t)q * D + p] = pp;
        pinv[(size_t)q * D + pp] = p;
      }
  return GDML_OK;
}

gdml_status setup_impl(gdml_ctx** out, const double* R_dev, int64_t M, int32_t N, double sigma, double lambda,
                       int32_t precision, void* cuda_stream, const int32_t* perms, int32_t Ssym) {
  clear_msg();
  if (!out) return fail(GDML_ERR_ARG, "ctx out-pointer is NULL");
  *out = nullptr;
  if (!R_dev) return fail(GDML_ERR_ARG, "R_dev is NULL");
  if (M < 1 || N < 2 || N > 128) return fail(GDML_ERR_ARG, "need M >= 1 and 2 <= N <= 128");
  if (!(sigma > 0.0) || !(lambda > 0.0) || !std::isfinite(sigma) || !std::isfinite(lambda))
    return fail(GDML_ERR_ARG, "need sigma > 0 and lambda > 0");
  if (precision < GDML_FP64 || precision > GDML_OZAKI) return fail(GDML_ERR_ARG, "unknown precision");
  std::vector<int> hpis, hpinv;
  if (Ssym > 1 || perms) {
    TRY(check_symmetry_group(perms, Ssym, N, hpis, hpinv));
    if (Ssym > 1 && precision != GDML_FP64 && precision != GDML_OZAKI)
      return fail(GDML_ERR_ARG, "symmetries need an FP64 or OZAKI context");
  }
  std::unique_ptr<gdml_ctx, void (*)(gdml_ctx*)> c(new gdml_ctx(), &gdml_destroy);
  CTRY(c.get(), cudaGetDevice(&c->device));
  c->st = static_cast<cudaStream_t>(cuda_stream);
  c->M = M;
  c->N = N;
  c->D = N * (N - 1) / 2;
  c->B = 3 * N;
  c->n = 3 * (int64_t)N * M;
  c->sigma = sigma;
  c->lam = lambda;
  c->c = std::sqrt(5.0) / sigma;
  c->precision = precision;
  c->inner_rtol = precision == GDML_BF16 ? 1e-3 : 1e-4;
  c->Ssym = Ssym > 1 ? Ssym : 1;
  const int64_t D = c->D, n = c->n, MB = M * c->Ssym;
  c->MB = MB;
  gdml_ctx* C = c.get();
  if (c->Ssym > 1 && ((size_t)N + 6 * (size_t)D) * sizeof(double) > 200 * 1024)
    return fail(GDML_ERR_ARG, "symmetries: the kernel columns of molecules with more than ~70 atoms are not supported");
  TRY(dalloc(C, &c->R, (size_t)(M * N * 3)));
  TRY(dalloc(C, &c->X, (size_t)(M * D)));
  TRY(dalloc(C, &c->G, (size_t)(M * D * 3)));
  TRY(dalloc(C, &c->S, (size_t)(M * MB)));
  TRY(dalloc(C, &c->P64, (size_t)(2 * M * MB)));
  TRY(dalloc(C, &c->V64, (size_t)(2 * MB * D)));
  TRY(dalloc(C, &c->T, (size_t)(M * MB)));
  TRY(dalloc(C, &c->tb, (size_t)MB));
  TRY(dalloc(C, &c->rowsum, (size_t)M));
  if (c->Ssym > 1) {
    TRY(dalloc(C, &c->pis, hpis.size()));
    TRY(dalloc(C, &c->pinv, hpinv.size()));
    TRY(dalloc(C, &c->XB, (size_t)(MB * D)));
    TRY(dalloc(C, &c->XcA, (size_t)(M * D)));
    TRY(dalloc(C, &c->Wa, (size_t)(M * D)));
    CTRY(C, cudaMemcpyAsync(c->pis, hpis.data(), hpis.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CTRY(C, cudaMemcpyAsync(c->pinv, hpinv.data(), hpinv.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  } else {
    c->XB = c->X;
    c->XcA = c->V64 + M * D;
    c->Wa = c->V64;
  }
  c->splitsU = dgemm_splits(M, D, 2 * MB);
  c->splits_cap = std::max(c->splitsU, 8);
  TRY(dalloc(C, &c->U, (size_t)(c->splits_cap * M * D)));
  TRY(dalloc(C, &c->diag, (size_t)n));
  for (double** v : {&c->r, &c->z, &c->p, &c->q, &c->x, &c->ys, &c->rsplit}) TRY(dalloc(C, v, (size_t)n));
  TRY(dalloc(C, &c->sc, SC_COUNT));
  TRY(dalloc(C, &c->partial, 4096));
  TRY(dalloc(C, &c->ticket, 1));
  TRY(dalloc(C, &c->status, 1));
  TRY(dalloc(C, &c->werr, 1));
  CTRY(C, cudaMemsetAsync(c->werr, 0, sizeof(int), c->st));
  TRY(dalloc(C, &c->wbar, 2));
  CTRY(C, cudaMemsetAsync(c->wbar, 0, 2 * sizeof(unsigned), c->st));
  if (df_precond(C)) (void)coop_graph_capture_ok();  // once per process, before any capture
  TRY(dalloc(C, &c->ictl, IC_COUNT));
  CTRY(C, cudaMemsetAsync(c->ictl, 0, IC_COUNT * sizeof(int64_t), c->st));
  c->hist_cap = kHistCap;
  TRY(dalloc(C, &c->hist, (size_t)(2 * c->hist_cap)));
  CTRY(C, cudaMallocHost(&c->hsc, SC_COUNT * sizeof(double)));
  CTRY(C, cudaMallocHost(&c->hictl, IC_COUNT * sizeof(int64_t)));
  CTRY(C, cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), c->st));
  CTRY(C, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
  CTRY(C, cudaMemsetAsync(c->sc, 0, SC_COUNT * sizeof(double), c->st));
  CTRY(C, cudaMemcpyAsync(c->R, R_dev, M * N * 3 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  launch_desc_jac(c->R, M, N, (int)D, c->X, c->G, c->st);
  {  // non-finite coordinates or two atoms at one place give non-finite descriptors
    int bad = 0;
    CTRY(C, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
    launch_check_finite(c->X, M * D, c->status, c->st);
    launch_check_finite(c->G, M * D * 3, c->status, c->st);
    TRY(check_launch(C, "descriptor check"));
    TRY(read_status(C, &bad));
    if (bad) return fail(GDML_ERR_ARG, "geometries must be finite with no two atoms of a geometry at one place");
  }
  launch_center(c->X, M, (int)D, c->XcA, c->st);
  if (c->Ssym > 1) {  // the training side: rows b S + q = P_q x_b, centred on the rows' mean
    launch_sym_gather(c->X, M, (int)D, c->pis, c->Ssym, nullptr, c->XB, nullptr, c->st);
    launch_center_like(c->XB, MB, (int)D, c->X, c->XcA, c->XcB(), c->st);
    launch_dist_tab_cross(c->X, M, c->XB, MB, (int)D, c->c, c->S, c->P64, 2 * MB, c->st);
    launch_kdiag_sym(c->X, c->G, M, N, (int)D, c->pis, c->pinv, c->Ssym, c->c, c->diag, c->st);
  } else {
    launch_dist_tab(c->X, M, (int)D, c->c, c->S, c->P64, 2 * M, c->st);
    launch_kdiag(c->G, M, N, (int)D, c->c, c->diag, c->st);
  }
  if (df_precond(c.get())) {
    TRY(dalloc(C, &c->X2, (size_t)(M * D)));
    TRY(dalloc(C, &c->G2, (size_t)(M * D * 3)));
    launch_split_df(c->X, M * D, c->X2, c->st);
    launch_split_df(c->G, M * D * 3, c->G2, c->st);
  }
  TRY(check_launch(C, "setup kernels"));
  if (precision == GDML_TF32 || precision == GDML_BF16) {
    gdml_status s = tc_setup(c->tc, precision, M, N, (int)D, c->Xc(), c->P64, 2 * M, c->S, c->G, c->c, c->st);
    if (s != GDML_OK) return ctx_fail(C, s, "tensor-core setup: " + last_msg());
  }
  if (precision == GDML_OZAKI) {
    gdml_status s = oz_setup(c->oz, M, N, (int)D, c->XcA, c->P64, 2 * MB, c->S, c->c, c->st, c->Ssym, c->pis,
                             c->XcB());
    if (s != GDML_OK) return ctx_fail(C, s, "sliced tensor-core setup: " + last_msg());
  }
  CTRY(C, cudaStreamSynchronize(c->st));
  *out = c.release();
  return GDML_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

gdml_status gdml_kernel_setup(gdml_ctx** out, const double* R_dev, int64_t M, int32_t N, double sigma,
                              double lambda, int32_t precision, void* cuda_stream) {
  return setup_impl(out, R_dev, M, N, sigma, lambda, precision, cuda_stream, nullptr, 1);
}

gdml_status gdml_kernel_setup_sym(gdml_ctx** out, const double* R_dev, int64_t M, int32_t N,
                                  const int32_t* perms_host, int32_t S, double sigma, double lambda,
                                  int32_t precision, void* cuda_stream) {
  if (!perms_host) {
    clear_msg();
    if (out) *out = nullptr;
    return fail(GDML_ERR_ARG, "perms_host is NULL");
  }
  return setup_impl(out, R_dev, M, N, sigma, lambda, precision, cuda_stream, perms_host, S);
}

gdml_status gdml_matvec(gdml_ctx* c, const double* v, double* out, int32_t add_lambda) {
  TRY(validate(c));
  if (!v || !out || v == out) return ctx_fail(c, GDML_ERR_ARG, "matvec: bad pointers");
  return matvec_any(c, v, out, add_lambda ? 1 : 0, false);
}

gdml_status gdml_matvec_fp64(gdml_ctx* c, const double* v, double* out, int32_t add_lambda) {
  TRY(validate(c));
  if (!v || !out || v == out) return ctx_fail(c, GDML_ERR_ARG, "matvec: bad pointers");
  return matvec_fp64(c, v, out, add_lambda ? 1 : 0);
}

// f_q = sum_b J_q^T H(x_q, x_b) J_b alpha_b: the FP64 matvec's steps with query rows against
// the training columns (T = Xq_c W^T is Q x M, U = [A | beta] [W ; Xc] is Q x D).
gdml_status gdml_predict_forces(gdml_ctx* c, const double* R_query, int64_t Q, const double* alpha, double* f) {
  TRY(validate(c));
  if (!R_query || !alpha || !f || alpha == f) return ctx_fail(c, GDML_ERR_ARG, "predict_forces: bad pointers");
  if (Q < 1 || Q > ((int64_t)1 << 20)) return ctx_fail(c, GDML_ERR_ARG, "predict_forces: need 1 <= Q <= 2^20");
  const int64_t M = c->M;
  const int N = c->N, D = c->D;
  cudaStream_t st = c->st;
  const int64_t MB = c->MB;  // the training side: M geometries, or M S with symmetries
  Scratch s{c, {}};
  double *Xq = nullptr, *Gq = nullptr, *Xqc = nullptr, *Sq = nullptr, *Tq = nullptr, *Pq = nullptr, *Uq = nullptr,
         *rs = nullptr;
  TRY(s.get(&Xq, (size_t)(Q * D)));
  TRY(s.get(&Gq, (size_t)(Q * D * 3)));
  TRY(s.get(&Xqc, (size_t)(Q * D)));
  TRY(s.get(&Sq, (size_t)(Q * MB)));
  TRY(s.get(&Tq, (size_t)(Q * MB)));
  TRY(s.get(&Pq, (size_t)(Q * 2 * MB)));
  TRY(s.get(&Uq, (size_t)(Q * D)));
  TRY(s.get(&rs, (size_t)Q));
  double* W = c->V64;  // [W ; Xc] of the training side: W_b = J_b alpha_b (permuted copies with symmetries)
  launch_desc_jac(R_query, Q, N, D, Xq, Gq, st);
  launch_center_like(Xq, Q, D, c->X, c->XcA, Xqc, st);
  launch_dist_tab_cross(Xq, Q, c->XB, MB, D, c->c, Sq, Pq, 2 * MB, st);
  if (c->Ssym > 1) {
    launch_proj(c->G, c->XcA, alpha, M, N, D, c->Wa, D, c->tb, st);
    launch_sym_gather(c->Wa, M, D, c->pis, c->Ssym, c->XcB(), W, c->tb, st);
  } else {
    launch_proj(c->G, c->XcA, alpha, M, N, D, W, D, c->tb, st);
  }
  launch_dgemm<double, double>(true, Q, MB, D, 1.0, Xqc, D, W, D, 0.0, Tq, MB, false, st);
  launch_beta_rows(Tq, Sq, c->tb, Q, MB, c->c, Pq + MB, 2 * MB, rs, st);
  launch_dgemm<double, double>(false, Q, D, 2 * MB, 1.0, Pq, 2 * MB, c->V64, D, 0.0, Uq, D, false, st);
  launch_backproj<double>(Uq, D, 1, Q * D, rs, Xqc, Gq, nullptr, Q, N, D, 0.0, 0, f, st);
  return check_launch(c, "predict_forces");
}

// Dense K (column-major n x n, from the kernel columns in blocks of 4096) and its ascending
// eigendecomposition in place: Kd holds the eigenvectors, w the eigenvalues (n <= kSvdMaxN)
static gdml_status dense_eigh(gdml_ctx* c, double* Kd, double* w, int64_t* cols) {
  const int64_t n = c->n;
  std::vector<int64_t> hcols(n);
  for (int64_t i = 0; i < n; ++i) hcols[i] = i;
  CTRY(c, cudaMemcpyAsync(cols, hcols.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
  constexpr int64_t kBlock = 4096;
  for (int64_t j0 = 0; j0 < n; j0 += kBlock) TRY(get_cols(c, cols + j0, std::min(kBlock, n - j0), Kd + j0 * n));
  const std::string e = eigh_dense(Kd, n, w, c->st);
  if (!e.empty()) return ctx_fail(c, GDML_ERR_CUDA, "dense eigendecomposition of K: " + e);
  return GDML_OK;
}

static gdml_status precond_build_impl(gdml_ctx* c, int32_t method, int64_t k, uint64_t seed, int64_t* pivots_dev,
                                      double* resid_trace_dev, const double* geometry_scores) {
  TRY(validate(c));
  const int64_t n = c->n;
  if (k < 1 || k > n || k > 16384) return ctx_fail(c, GDML_ERR_ARG, "need 1 <= k <= min(n, 16384)");
  if (method < GDML_SEL_UNIFORM || method > GDML_SEL_SVD) return ctx_fail(c, GDML_ERR_ARG, "unknown method");
  if (method == GDML_SEL_WEIGHTED && !geometry_scores) return ctx_fail(c, GDML_ERR_ARG, "scores are NULL");
  if (method == GDML_SEL_SVD && n > kSvdMaxN)
    return ctx_fail(c, GDML_ERR_ARG, "the SVD preconditioner needs n <= " + std::to_string(kSvdMaxN) +
                                         " (a dense eigendecomposition of K)");
  c->k = 0;
  c->ws = WsPlan();
  c->jitter = 0.0;
  drop_graphs(c);
  TRY(ensure_precond_buffers(c, k));
  Scratch s{c, {}};
  int64_t* S = nullptr;
  TRY(s.get(&S, (size_t)k));
  double* trace = nullptr;
  TRY(s.get(&trace, (size_t)k));
  CTRY(c, cudaMemsetAsync(trace, 0, k * sizeof(double), c->st));
  CTRY(c, cudaMemsetAsync(S, 0xFF, k * sizeof(int64_t), c->st));
  int64_t rank = k;
  double* weights = nullptr;
  if (method == GDML_SEL_WEIGHTED) {
    TRY(s.get(&weights, (size_t)n));
    launch_column_weights(geometry_scores, c->diag, n, c->B, weights, c->st);
  }
  if (method == GDML_SEL_PIVCHOL) {
    double* d = nullptr;
    int64_t* perm = nullptr;
    unsigned char* chosen = nullptr;
    PivState* ps = nullptr;
    ArgMaxPart* part = nullptr;
    unsigned* ticket = nullptr;
    double* col = nullptr;
    TRY(s.get(&d, (size_t)n));
    TRY(s.get(&perm, (size_t)n));
    TRY(s.get(&chosen, (size_t)n));
    TRY(s.get(&ps, 1));
    TRY(s.get(&part, (size_t)pivchol_part_blocks()));
    TRY(s.get(&ticket, 1));
    TRY(s.get(&col, (size_t)n));
    CTRY(c, cudaMemcpyAsync(d, c->diag, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    std::vector<int64_t> hperm(n);
    for (int64_t i = 0; i < n; ++i) hperm[i] = i;
    CTRY(c, cudaMemcpyAsync(perm, hperm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
    CTRY(c, cudaMemsetAsync(chosen, 0, n, c->st));
    CTRY(c, cudaMemsetAsync(ps, 0, sizeof(PivState), c->st));
    CTRY(c, cudaMemsetAsync(ticket, 0, sizeof(unsigned), c->st));
    if (!df_precond(c)) CTRY(c, cudaMemsetAsync(c->L, 0, n * k * sizeof(double), c->st));
    PivCholArgs a;
    a.n = n;
    a.k = k;
    a.d = d;
    a.perm = perm;
    a.chosen = chosen;
    a.pivots = S;
    a.trace = trace;
    a.ps = ps;
    a.part = part;
    a.ticket = ticket;
    a.col = col;
    a.get_col = [c](const int64_t* cols, double* out, const int* stop, cudaStream_t st) {
      if (c->Ssym > 1) {  // checked to fit at setup
        (void)launch_kcol_sym(cols, 1, c->X, c->G, c->S, c->P64, 2 * c->MB, c->M, c->MB, c->N, c->D, c->pis, c->pinv,
                              c->Ssym, c->c, out, c->n, stop, st);
        return;
      }
      if (!c->X2 || !launch_kcol_df(cols, 1, c->X2, c->G2, c->S, c->P64, 2 * c->M, c->M, c->N, c->D, c->c, out,
                                    c->n, stop, st))
        launch_kcol(cols, 1, c->X, c->G, c->S, c->P64, 2 * c->M, c->M, c->N, c->D, c->c, out, c->n, stop, st);
    };
    if (df_precond(c)) {
      TRY(s.get(&a.schur, (size_t)(pivchol_schur_groups() * n)));
      TRY(s.get(&a.prow, (size_t)k));
      TRY(s.get(&a.posof, (size_t)n));
      CTRY(c, cudaMemcpyAsync(a.posof, hperm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
      CTRY(c, cudaMemsetAsync(c->Lf, 0, n * k * sizeof(float), c->st));
      a.err = c->werr;
      pivchol_run_df(a, c->Lf, c->st);
    } else {
      pivchol_run<double>(a, c->L, c->st);
    }
    TRY(check_launch(c, "pivoted cholesky"));
    PivState hps;
    CTRY(c, cudaMemcpyAsync(&hps, ps, sizeof(PivState), cudaMemcpyDeviceToHost, c->st));
    CTRY(c, cudaStreamSynchronize(c->st));
    rank = hps.rank;
    if (rank < 1) return ctx_fail(c, GDML_ERR_NOT_SPD, "diag(K) has no positive entry");
  } else if (method == GDML_SEL_SVD) {
    // dense K from the kernel columns, its eigendecomposition, L_k = U_k Sigma_k^(1/2); no
    // pivots (left at -1); trace[m] = tr(K) - (sum of the m + 1 largest eigenvalues)
    double *Kd = nullptr, *w = nullptr;
    int64_t* cols = nullptr;
    TRY(s.get(&Kd, (size_t)(n * n)));
    TRY(s.get(&w, (size_t)n));
    TRY(s.get(&cols, (size_t)n));
    TRY(dense_eigh(c, Kd, w, cols));
    launch_svd_factor(Kd, w, n, k, c->L, c->st);
    TRY(check_launch(c, "SVD factor"));
    std::vector<double> hw(n), htr(k);
    CTRY(c, cudaMemcpyAsync(hw.data(), w, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CTRY(c, cudaStreamSynchronize(c->st));
    double rest = 0.0;  // ascending: the eigenvalues below the top m + 1
    for (int64_t i = 0; i < n - k; ++i) rest += hw[i];
    for (int64_t m = k - 1; m >= 0; --m) {
      htr[m] = rest;
      if (m > 0) rest += hw[n - 1 - m];
    }
    CTRY(c, cudaMemcpyAsync(trace, htr.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->st));
    if (df_precond(c)) to_float(c->L, n * k, c->Lf, c->st);
  } else {
    uint64_t* key = nullptr;
    int64_t* idx = nullptr;
    const int64_t P = select_scratch_len(n);
    TRY(s.get(&key, (size_t)P));
    TRY(s.get(&idx, (size_t)P));
    double* Kkk = nullptr;
    double* work = nullptr;
    TRY(s.get(&Kkk, (size_t)(k * k)));
    TRY(s.get(&work, (size_t)(k * k)));
    if (method == GDML_SEL_RLS) {
      double* tau = nullptr;
      TRY(s.get(&tau, (size_t)n));
      TRY(rls_estimate(c, k, seed, S, Kkk, work, key, idx, tau));
      select_weighted(n, k, seed, 2u, tau, key, idx, S, c->st);
    } else if (method == GDML_SEL_WEIGHTED) {
      select_weighted(n, k, seed, 3u, weights, key, idx, S, c->st);
    } else {
      select_uniform(n, k, seed, 0u, key, idx, S, c->st);
    }
    TRY(check_launch(c, "selection"));
    TRY(nystrom(c, S, k, c->L, Kkk, work, &c->jitter));
    if (df_precond(c)) to_float(c->L, n * k, c->Lf, c->st);
  }
  TRY(woodbury_core(c, c->L, rank, c->LC, c->Cinv, c->Cfull, df_precond(c) ? c->Lf : nullptr));
  if (pivots_dev) CTRY(c, cudaMemcpyAsync(pivots_dev, S, k * sizeof(int64_t), cudaMemcpyDeviceToDevice, c->st));
  if (resid_trace_dev)
    CTRY(c, cudaMemcpyAsync(resid_trace_dev, trace, k * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  if (df_precond(c)) TRY(ws_check(c));
  c->k = rank;
  if (df_precond(c)) ws_plan(c->ws, c->Lf, n, rank);
  return GDML_OK;
}

gdml_status gdml_precond_build(gdml_ctx* c, int32_t method, int64_t k, uint64_t seed, int64_t* pivots_dev,
                               double* resid_trace_dev) {
  if (method == GDML_SEL_WEIGHTED) return ctx_fail(c, GDML_ERR_ARG, "use gdml_precond_build_scored for scores");
  return precond_build_impl(c, method, k, seed, pivots_dev, resid_trace_dev, nullptr);
}

gdml_status gdml_precond_build_scored(gdml_ctx* c, const double* geometry_scores_dev, int64_t k, uint64_t seed,
                                      int64_t* pivots_dev) {
  return precond_build_impl(c, GDML_SEL_WEIGHTED, k, seed, pivots_dev, nullptr, geometry_scores_dev);
}

gdml_status gdml_rls_scores(gdml_ctx* c, int64_t k, uint64_t seed, double* tau_dev) {
  TRY(validate(c));
  const int64_t n = c->n;
  if (!tau_dev) return ctx_fail(c, GDML_ERR_ARG, "tau_dev is NULL");
  if (k < 1 || k > n || k > 16384) return ctx_fail(c, GDML_ERR_ARG, "need 1 <= k <= min(n, 16384)");
  c->k = 0;
  c->ws = WsPlan();
  drop_graphs(c);
  TRY(ensure_precond_buffers(c, k));
  Scratch s{c, {}};
  int64_t* S = nullptr;
  uint64_t* key = nullptr;
  int64_t* idx = nullptr;
  double *Kkk = nullptr, *work = nullptr;
  const int64_t P = select_scratch_len(n);
  TRY(s.get(&S, (size_t)k));
  TRY(s.get(&key, (size_t)P));
  TRY(s.get(&idx, (size_t)P));
  TRY(s.get(&Kkk, (size_t)(k * k)));
  TRY(s.get(&work, (size_t)(k * k)));
  TRY(rls_estimate(c, k, seed, S, Kkk, work, key, idx, tau_dev));
  CTRY(c, cudaStreamSynchronize(c->st));
  return GDML_OK;
}

gdml_status gdml_rls_labels(gdml_ctx* c, int32_t exact, int64_t k, uint64_t seed, double* labels_dev) {
  TRY(validate(c));
  const int64_t n = c->n;
  if (!labels_dev) return ctx_fail(c, GDML_ERR_ARG, "labels_dev is NULL");
  Scratch s{c, {}};
  double* tau = nullptr;
  TRY(s.get(&tau, (size_t)n));
  if (exact) {
    if (n > kSvdMaxN)
      return ctx_fail(c, GDML_ERR_ARG, "exact leverage scores need n <= " + std::to_string(kSvdMaxN) +
                                           " (a dense eigendecomposition of K)");
    double *Kd = nullptr, *w = nullptr;
    int64_t* cols = nullptr;
    TRY(s.get(&Kd, (size_t)(n * n)));
    TRY(s.get(&w, (size_t)n));
    TRY(s.get(&cols, (size_t)n));
    TRY(dense_eigh(c, Kd, w, cols));
    launch_rls_from_eigen(Kd, w, n, c->lam, tau, c->st);
  } else {
    TRY(gdml_rls_scores(c, k, seed, tau));
  }
  launch_group_sums(tau, c->M, c->B, labels_dev, c->st);
  TRY(check_launch(c, "rls labels"));
  CTRY(c, cudaStreamSynchronize(c->st));
  return GDML_OK;
}

gdml_status gdml_descriptors(const gdml_ctx* c, double* X_dev) {
  TRY(validate(c));
  if (!X_dev) return fail(GDML_ERR_ARG, "X_dev is NULL");
  if (cudaMemcpyAsync(X_dev, c->X, c->M * c->D * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "copying descriptors");
  return GDML_OK;
}

gdml_status gdml_precond_info(const gdml_ctx* c, int64_t* rank_out, double* jitter_out) {
  TRY(validate(c));
  if (rank_out) *rank_out = c->k;
  if (jitter_out) *jitter_out = c->jitter;
  return GDML_OK;
}

gdml_status gdml_precond_apply(gdml_ctx* c, const double* r, double* z) {
  TRY(validate(c));
  if (!r || !z || r == z) return ctx_fail(c, GDML_ERR_ARG, "precond_apply: bad pointers");
  if (c->k == 0) return ctx_fail(c, GDML_ERR_STATE, "no preconditioner built");
  return apply_precond(c, r, z);
}

gdml_status gdml_pcg_spectrum(gdml_ctx* c, int32_t count, double* ritz_host, double* theta_min, double* theta_max,
                              int32_t* steps_out) {
  TRY(validate(c));
  if (count < 0 || count > 1024 || (count > 0 && !ritz_host))
    return ctx_fail(c, GDML_ERR_ARG, "pcg_spectrum: need 0 <= count <= 1024 and ritz_host for count > 0");
  if (c->hist_len < 1) return ctx_fail(c, GDML_ERR_STATE, "pcg_spectrum: no recorded PCG run (solve first)");
  const int64_t m_rec = c->hist_len;
  std::vector<double> h(2 * m_rec);
  CTRY(c, cudaMemcpyAsync(h.data(), c->hist, 2 * m_rec * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CTRY(c, cudaStreamSynchronize(c->st));
  std::vector<double> g(m_rec), b(m_rec);
  int64_t m = 0;  // the valid prefix: positive finite steps, non-negative finite ratios between them
  for (; m < m_rec; ++m) {
    g[m] = h[2 * m];
    b[m] = h[2 * m + 1];
    if (!(g[m] > 0.0 && std::isfinite(g[m]))) break;
    if (m > 0 && !(b[m - 1] >= 0.0 && std::isfinite(b[m - 1]))) break;
  }
  if (m < 1) return ctx_fail(c, GDML_ERR_STATE, "pcg_spectrum: the recorded run has no valid CG step");
  double tmin = 0.0, tmax = 0.0;
  lanczos_ritz(g.data(), b.data(), m, count, ritz_host, &tmin, &tmax);
  if (theta_min) *theta_min = tmin;
  if (theta_max) *theta_max = tmax;
  if (steps_out) *steps_out = (int32_t)m;
  return GDML_OK;
}

gdml_status gdml_set_inner_levels(gdml_ctx* c, int32_t levels) {
  TRY(validate(c));
  if (c->precision != GDML_OZAKI) return ctx_fail(c, GDML_ERR_ARG, "inner levels apply to OZAKI contexts only");
  if (levels < 1 || levels > 7) return ctx_fail(c, GDML_ERR_ARG, "inner levels must be in 1..7");
  if (levels != c->inner_lev) drop_graphs(c);  // the captured loop bakes the GEMMs' level count in
  c->inner_lev = levels;
  return GDML_OK;
}

gdml_status gdml_set_inner_rtol(gdml_ctx* c, double v) {
  TRY(validate(c));
  if (!(v > 0.0 && v < 1.0)) return ctx_fail(c, GDML_ERR_ARG, "inner_rtol must be in (0, 1)");
  c->inner_rtol = v;
  return GDML_OK;
}

gdml_status gdml_last_outer_steps(const gdml_ctx* c, int32_t* o) {
  TRY(validate(c));
  if (o) *o = c->last_outer;
  return GDML_OK;
}

gdml_status gdml_pcg_solve(gdml_ctx* c, const double* y, double* alpha, double rtol, int32_t max_iter,
                           int32_t* iters_out, double* relres_out) {
  TRY(validate(c));
  if (!y || !alpha || y == alpha) return ctx_fail(c, GDML_ERR_ARG, "pcg_solve: bad pointers");
  if (!(rtol > 0.0) || max_iter < 1) return ctx_fail(c, GDML_ERR_ARG, "need rtol > 0 and max_iter >= 1");
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  // |y|
  CTRY(c, cudaMemcpyAsync(c->ys, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(dot(c, c->ys, c->ys, SC_YY));
  TRY(fetch_scalars(c));
  const double ynorm = std::sqrt(c->hsc[SC_YY]);
  if (!std::isfinite(ynorm)) return ctx_fail(c, GDML_ERR_ARG, "pcg_solve: y is not finite");
  int64_t iters = 0;
  double res = 0.0;
  gdml_status stat = GDML_OK;
  c->hist_len = 0;
  c->hist_arm = true;  // the first CG run below records its coefficients
  if (ynorm == 0.0) {
    CTRY(c, cudaMemsetAsync(alpha, 0, n * sizeof(double), st));
    c->last_outer = 0;
  } else if (direct_pcg(c)) {
    // the captured loop is bound to the context's own x buffer; DF64 / OZAKI
    // iterate with their FP64-class matvec and refine through FP64 true-residual restarts
    const bool fp64 = c->precision == GDML_FP64;
    CTRY(c, cudaMemcpyAsync(c->x, alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    stat = pcg_core(c, c->ys, c->x, rtol * ynorm, max_iter, fp64, true, fp64 ? 3 : 10, &iters, &res);
    CTRY(c, cudaMemcpyAsync(alpha, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    c->last_outer = 1 + c->last_restarts;
  } else {
    // FP64 iterative refinement around the tensor-core PCG
    double* dx = c->x;
    double* rhs = nullptr;
    Scratch s{c, {}};
    TRY(s.get(&rhs, (size_t)n));
    // r = y - K alpha (FP64)
    TRY(matvec_any(c, alpha, rhs, 1, true));
    launch_axpby(rhs, c->ys, 1.0, -1.0, n, st);
    TRY(dot(c, rhs, rhs, SC_RR));
    TRY(fetch_scalars(c));
    res = std::sqrt(c->hsc[SC_RR]);
    int outer = 0, stalls = 0;
    while (res > rtol * ynorm && outer < 20 && iters < max_iter) {
      ++outer;
      CTRY(c, cudaMemsetAsync(dx, 0, n * sizeof(double), st));
      int64_t it_in = 0;
      double res_in = 0.0;
      const double tol_in = std::max(c->inner_rtol * res, 0.5 * rtol * ynorm);
      stat = pcg_core(c, rhs, dx, tol_in, max_iter - iters, false, false, 0, &it_in, &res_in);
      iters += it_in;
      if (stat != GDML_OK) break;
      launch_axpby(alpha, dx, 1.0, 1.0, n, st);
      TRY(matvec_any(c, alpha, rhs, 1, true));  // FP64 residual y - K_lambda alpha
      launch_axpby(rhs, c->ys, 1.0, -1.0, n, st);
      TRY(dot(c, rhs, rhs, SC_RR));
      TRY(fetch_scalars(c));
      const double rnew = std::sqrt(c->hsc[SC_RR]);
      TRY(check_launch(c, "refinement"));
      if (!(rnew < res)) {  // the correction did not help: undo it and stop
        launch_axpby(alpha, dx, -1.0, 1.0, n, st);
        break;
      }
      // stagnation: the low-precision operator cannot resolve what is left
      stalls = rnew > 0.5 * res ? stalls + 1 : 0;
      res = rnew;
      if (stalls >= 3) break;
    }
    c->last_outer = outer;
  }
  c->hist_arm = false;
  CTRY(c, cudaStreamSynchronize(st));
  if (c->precision == GDML_TF32 || c->precision == GDML_BF16 || c->precision == GDML_OZAKI) {
    gdml_status ts = c->precision == GDML_OZAKI ? oz_check(c->oz, st) : tc_check(c->tc, st);
    if (ts != GDML_OK) return ctx_fail(c, ts, last_msg());
  }
  if (df_precond(c)) TRY(ws_check(c));
  if (iters_out) *iters_out = (int32_t)iters;
  const double rel = ynorm > 0 ? res / ynorm : 0.0;
  if (relres_out) *relres_out = rel;
  if (stat != GDML_OK) return stat;
  if (rel > rtol) return ctx_fail(c, GDML_ERR_NOT_CONVERGED, "PCG did not reach rtol within max_iter");
  return GDML_OK;
}

gdml_status gdml_test_tc_gemm(int32_t bf16, const double* A_dev, const double* B_dev, int32_t M, int32_t N,
                              int32_t K, double* C_dev, void* stream) {
  clear_msg();
  if (!A_dev || !B_dev || !C_dev || M < 1 || N < 1 || K < 1) return fail(GDML_ERR_ARG, "bad gemm test arguments");
  return tc_gemm_test(bf16, A_dev, B_dev, M, N, K, C_dev, static_cast<cudaStream_t>(stream));
}

gdml_status gdml_test_df_passes(const float* L_dev, int64_t n, int64_t k, const double* r_dev, const double* u_dev,
                                double lambda, int32_t staged, double* t_dev, double* z_dev, void* stream) {
  clear_msg();
  if (!L_dev || !r_dev || !u_dev || !t_dev || !z_dev || n < 1 || k < 1 || !(lambda > 0.0))
    return fail(GDML_ERR_ARG, "bad apply-pass test arguments");
  if (n > ((int64_t)1 << 30) || k > 16384) return fail(GDML_ERR_ARG, "apply-pass test sizes too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsPlan plan;
  if (staged) {
    ws_plan(plan, L_dev, n, k, staged);
    if (!plan.ok) return fail(GDML_ERR_ARG, "staged passes need n % 4 == 0 and a valid TMA map");
  }
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };  // 256-byte aligned sub-buffers
  const size_t part_b = al((size_t)woodbury_part_size(n, k) * sizeof(double));
  const size_t rs_b = al((size_t)n * sizeof(float2)), kv_b = al((size_t)k * sizeof(float2));
  void* buf = nullptr;
  if (cudaMalloc(&buf, part_b + rs_b + 2 * kv_b + 256) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GDML_ERR_OOM, "apply-pass test scratch");
  }
  char* b = static_cast<char*>(buf);
  double* part = reinterpret_cast<double*>(b);
  float2* rs = reinterpret_cast<float2*>(b + part_b);
  float2* t2 = reinterpret_cast<float2*>(b + part_b + rs_b);
  float2* u2 = reinterpret_cast<float2*>(b + part_b + rs_b + kv_b);
  int* err = reinterpret_cast<int*>(b + part_b + rs_b + 2 * kv_b);
  gdml_status s = GDML_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) s = fail(GDML_ERR_CUDA, "apply-pass test memset");
  if (s == GDML_OK) {
    df_passes(L_dev, n, k, r_dev, u_dev, lambda, t_dev, z_dev, part, rs, t2, u2, staged ? &plan : nullptr, err, st);
    int h = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = fail(GDML_ERR_CUDA, "apply-pass test launch");
    else if (h)
      s = fail(GDML_ERR_TIMEOUT, "a staged Woodbury pass wait timed out (code " + std::to_string(h) + ")");
  }
  cudaFree(buf);
  return s;
}

gdml_status gdml_test_oz_gemm(const double* A_dev, const double* B_dev, int64_t M, int64_t N, int64_t K,
                              int32_t chunks_per_cta, int32_t levels, double* C_dev, void* stream) {
  clear_msg();
  if (!A_dev || !B_dev || !C_dev || M < 1 || N < 1 || K < 1) return fail(GDML_ERR_ARG, "bad gemm test arguments");
  if (M > ((int64_t)1 << 24) || N > ((int64_t)1 << 24) || K > ((int64_t)1 << 24))
    return fail(GDML_ERR_ARG, "gemm test sizes too large");
  if (levels < 1 || levels > 7) return fail(GDML_ERR_ARG, "gemm test: levels outside 1..7");
  return oz_gemm_test(A_dev, B_dev, M, N, K, chunks_per_cta, levels, C_dev, static_cast<cudaStream_t>(stream));
}

gdml_status gdml_test_oz_gemm_tall(const double* A_dev, int64_t n, int64_t K, const double* B_dev, int64_t NB,
                                   int64_t ldb, int32_t tri_b, int32_t rowsq, double* out_dev, float* out32_dev,
                                   void* stream) {
  clear_msg();
  if (!A_dev || !B_dev || !out_dev || n < 1 || K < 1 || NB < 1 || ldb < K)
    return fail(GDML_ERR_ARG, "bad tall gemm test arguments");
  if (n > ((int64_t)1 << 31)) return fail(GDML_ERR_ARG, "tall gemm test: n too large");
  return oz_gemm_tall(A_dev, n, K, B_dev, NB, ldb, tri_b != 0, rowsq != 0, out_dev, rowsq ? nullptr : out32_dev,
                      static_cast<cudaStream_t>(stream));
}

gdml_status gdml_test_precond_factor(gdml_ctx* c, double* L_out) {
  TRY(validate(c));
  if (!L_out) return ctx_fail(c, GDML_ERR_ARG, "precond_factor: NULL output");
  if (c->k == 0) return ctx_fail(c, GDML_ERR_STATE, "no preconditioner built");
  const int64_t count = c->n * c->k;
  if (df_precond(c)) {
    widen_float(c->Lf, count, L_out, c->st);
    TRY(check_launch(c, "precond_factor"));
  } else {
    CTRY(c, cudaMemcpyAsync(L_out, c->L, count * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  }
  CTRY(c, cudaStreamSynchronize(c->st));
  return GDML_OK;
}

gdml_status gdml_test_set_wait_limit(uint32_t polls) {
  clear_msg();
  const uint32_t v = polls == 0xFFFFFFFFu ? tc_default_wait_limit() : polls;
  for (auto fn : {set_wait_limit_oz, set_wait_limit_tc, set_wait_limit_wb, set_wait_limit_pc}) {
    cudaError_t e = fn(v);
    if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("set_wait_limit: ") + cudaGetErrorString(e));
  }
  return GDML_OK;
}

gdml_status gdml_test_cholesky_jitter(const double* A_dev, int64_t k, double* L_dev, double* eps_out, void* stream) {
  clear_msg();
  if (!A_dev || !L_dev || !eps_out || k < 1 || k > 16384) return fail(GDML_ERR_ARG, "bad cholesky test arguments");
  gdml_ctx tmp;  // carries the stream, the status word and the error text only
  tmp.st = static_cast<cudaStream_t>(stream);
  if (cudaMalloc(&tmp.status, sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GDML_ERR_OOM, "cholesky test status word");
  }
  double eps = 0.0;
  gdml_status s = chol_jitter(&tmp, A_dev, L_dev, k, &eps);
  cudaStreamSynchronize(tmp.st);
  cudaFree(tmp.status);
  tmp.status = nullptr;
  *eps_out = eps;
  return s;
}

gdml_status gdml_test_set_lambda(gdml_ctx* c, double lambda) {
  TRY(validate(c));
  if (!std::isfinite(lambda)) return ctx_fail(c, GDML_ERR_ARG, "set_lambda: lambda must be finite");
  c->lam = lambda;
  c->k = 0;  // the preconditioner was built for the old lambda
  c->ws = WsPlan();
  drop_graphs(c);
  return GDML_OK;
}

int64_t gdml_launch_count(void) { return launch_count(); }

// Many independent FP64 systems, one CUDA graph: per system a gate kernel and a
// conditional WHILE node whose body is that system's PCG iteration.  The
// systems are independent branches of the graph, so their loops run
// concurrently on the device; the host only prepares each round and checks
// the true residuals between launches (restarting drifted systems).
gdml_status gdml_pcg_solve_batched(gdml_ctx* const* ctxs, int32_t count, const double* const* y_dev,
                                   double* const* alpha_dev, double rtol, int32_t max_iter, int32_t* iters_out,
                                   double* relres_out) {
  clear_msg();
  if (!ctxs || !y_dev || !alpha_dev || count < 1) return fail(GDML_ERR_ARG, "batched solve: bad arguments");
  if (!(rtol > 0.0) || max_iter < 1) return fail(GDML_ERR_ARG, "batched solve: need rtol > 0 and max_iter >= 1");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !y_dev[i] || !alpha_dev[i]) return fail(GDML_ERR_ARG, "batched solve: null entry");
    if (!direct_pcg(ctxs[i]))
      return fail(GDML_ERR_ARG, "batched solve: FP64, DF64 or OZAKI contexts only");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(GDML_ERR_ARG, "batched solve: a context appears twice");
  }
  std::vector<double> ynorm(count), res(count);
  std::vector<int64_t> iters(count, 0);
  std::vector<int> restarts(count, 0), active(count, 0);
  // initial residuals
  for (int i = 0; i < count; ++i) {
    gdml_ctx* c = ctxs[i];
    const int64_t n = c->n;
    CTRY(c, cudaMemcpyAsync(c->ys, y_dev[i], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    CTRY(c, cudaMemcpyAsync(c->x, alpha_dev[i], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    TRY(dot(c, c->ys, c->ys, SC_YY));
    TRY(matvec_any(c, c->x, c->r, 1, true));
    launch_axpby(c->r, c->ys, 1.0, -1.0, n, c->st);
    TRY(dot(c, c->r, c->r, SC_RR));
  }
  for (int i = 0; i < count; ++i) {
    gdml_ctx* c = ctxs[i];
    TRY(fetch_scalars(c));
    ynorm[i] = std::sqrt(c->hsc[SC_YY]);
    res[i] = std::sqrt(c->hsc[SC_RR]);
    if (!std::isfinite(ynorm[i]) || !std::isfinite(res[i]))
      return fail(GDML_ERR_ARG, "batched solve: y or alpha of system " + std::to_string(i) + " is not finite");
  }
  // one graph for all systems
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return fail(GDML_ERR_CUDA, "cudaGraphCreate");
  std::vector<int64_t> body_n(count, 0);
  gdml_status bs = GDML_OK;
  for (int i = 0; i < count && bs == GDML_OK; ++i) {
    gdml_ctx* c = ctxs[i];
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
      bs = fail(GDML_ERR_CUDA, "capture stream");
      break;
    }
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    // gate kernel node, then the WHILE node depending on it
    cudaGraphNode_t gate_tail = nullptr;
    if (e == cudaSuccess) e = add_pcg_gate_node(g, &gate_tail, c->sc, c->ictl, h);
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, &gate_tail, nullptr, 1, &prm);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(c->cap, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      bs = fail(GDML_ERR_CUDA, std::string("building the batched graph: ") + cudaGetErrorString(e));
      break;
    }
    cudaStream_t user = c->st;
    c->st = c->cap;
    const int64_t before = launch_count();
    bs = pcg_body(c, c->x, c->precision == GDML_FP64, h);
    body_n[i] = launch_count() - before;
    count_launch(-body_n[i]);
    c->st = user;
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(c->cap, &body);
    if (bs == GDML_OK && e != cudaSuccess) bs = fail(GDML_ERR_CUDA, "capturing a batched PCG body");
  }
  cudaGraphExec_t ex = nullptr;
  if (bs == GDML_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess)
    bs = fail(GDML_ERR_CUDA, "instantiating the batched graph");
  cudaGraphDestroy(g);
  if (bs != GDML_OK) {
    (void)cudaGetLastError();
    return bs;
  }
  cudaStream_t st0 = ctxs[0]->st;
  gdml_status out = GDML_OK;
  for (int round = 0; round < 12; ++round) {
    int n_active = 0;
    for (int i = 0; i < count; ++i) {
      gdml_ctx* c = ctxs[i];
      const double tol = rtol * ynorm[i];
      const int max_rs = c->precision == GDML_FP64 ? 3 : 10;
      active[i] = ynorm[i] > 0.0 && res[i] > tol && iters[i] < max_iter && restarts[i] <= max_rs;
      c->hictl[IC_ITER] = 0;
      c->hictl[IC_MAXIT] = active[i] ? max_iter - iters[i] : 0;
      c->hictl[IC_HCAP] = 0;  // batched solves record no Lanczos coefficients
      c->hist_len = 0;
      c->hsc[SC_TOL2] = tol * tol;
      if (active[i]) {
        ++n_active;
        TRY(apply_precond(c, c->r, c->z));
        CTRY(c, cudaMemcpyAsync(c->p, c->z, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        TRY(dot(c, c->r, c->z, SC_RHO));
      }
      CTRY(c, cudaMemcpyAsync(c->ictl, c->hictl, 3 * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
      CTRY(c, cudaMemcpyAsync(c->sc + SC_TOL2, c->hsc + SC_TOL2, sizeof(double), cudaMemcpyHostToDevice, c->st));
      CTRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
      CTRY(c, cudaStreamSynchronize(c->st));
    }
    if (!n_active) break;
    CTRY(ctxs[0], cudaGraphLaunch(ex, st0));
    CTRY(ctxs[0], cudaStreamSynchronize(st0));
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      gdml_ctx* c = ctxs[i];
      int hst = 0;
      CTRY(c, cudaMemcpyAsync(c->hictl, c->ictl, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
      CTRY(c, cudaMemcpyAsync(&hst, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      TRY(fetch_scalars(c));
      iters[i] += c->hictl[IC_ITER];
      count_launch(c->hictl[IC_ITER] * body_n[i] + 1);
      if (hst) {
        out = ctx_fail(c, GDML_ERR_BREAKDOWN, "PCG breakdown in a batched system");
        restarts[i] = 99;
        continue;
      }
      TRY(matvec_any(c, c->x, c->r, 1, true));  // true FP64 residual
      launch_axpby(c->r, c->ys, 1.0, -1.0, c->n, c->st);
      TRY(dot(c, c->r, c->r, SC_RR));
      TRY(fetch_scalars(c));
      res[i] = std::sqrt(c->hsc[SC_RR]);
      if (res[i] > rtol * ynorm[i]) ++restarts[i];
    }
  }
  cudaGraphExecDestroy(ex);
  bool all = true;
  for (int i = 0; i < count; ++i) {
    gdml_ctx* c = ctxs[i];
    if (ynorm[i] == 0.0) {
      CTRY(c, cudaMemsetAsync(alpha_dev[i], 0, c->n * sizeof(double), c->st));
    } else {
      CTRY(c, cudaMemcpyAsync(alpha_dev[i], c->x, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    }
    CTRY(c, cudaStreamSynchronize(c->st));
    const double rel = ynorm[i] > 0 ? res[i] / ynorm[i] : 0.0;
    if (iters_out) iters_out[i] = (int32_t)iters[i];
    if (relres_out) relres_out[i] = rel;
    c->last_outer = 1;
    if (rel > rtol) all = false;
  }
  if (out != GDML_OK) return out;
  if (!all) return fail(GDML_ERR_NOT_CONVERGED, "batched solve: some systems did not reach rtol");
  return GDML_OK;
}

// Tile autotuner: time the candidate K-splits of the matvec's second
// contraction (FP64: DGEMM split-K; TF32/BF16: tcgen05 split-K) on this
// context's shapes and keep the fastest.  *choice_out = chosen split count.
gdml_status gdml_autotune(gdml_ctx* c, int32_t* choice_out) {
  TRY(validate(c));
  double* v = c->z;
  double* out = c->q;
  CTRY(c, cudaMemsetAsync(v, 0, c->n * sizeof(double), c->st));
  cudaEvent_t e0, e1;
  CTRY(c, cudaEventCreate(&e0));
  CTRY(c, cudaEventCreate(&e1));
  if (c->precision == GDML_OZAKI) {
    // the sliced GEMMs' K chunks per CTA (GEMM 1: T = Xc W^T, GEMM 2: U = A W + beta Xc)
    auto time_mv = [&](float* ms) -> gdml_status {
      for (int w = 0; w < 2; ++w) TRY(matvec_any(c, v, out, 1, false));
      CTRY(c, cudaEventRecord(e0, c->st));
      for (int w = 0; w < 5; ++w) TRY(matvec_any(c, v, out, 1, false));
      CTRY(c, cudaEventRecord(e1, c->st));
      CTRY(c, cudaEventSynchronize(e1));
      cudaEventElapsedTime(ms, e0, e1);
      return GDML_OK;
    };
    const int n1 = (int)c->oz.W1.nchunks, n2 = (int)c->oz.nch2;
    std::vector<int> cand2;
    for (int g = 1; g <= n2; g = g < 4 ? g + 1 : g * 2) cand2.push_back(g);
    if (cand2.back() != n2) cand2.push_back(n2);
    int best1 = c->oz.g1, best2 = c->oz.g2;
    float best_ms = 1e30f;
    for (int g1 : {1, n1}) {
      for (int g2 : cand2) {
        c->oz.g1 = g1;
        c->oz.g2 = g2;
        float ms = 0.f;
        gdml_status ts = time_mv(&ms);
        if (ts != GDML_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return ts;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best1 = g1;
          best2 = g2;
        }
      }
      if (n1 == 1) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->oz.g1 = best1;
    c->oz.g2 = best2;
    drop_graphs(c);
    if (choice_out) *choice_out = best1 * 65536 + best2;
    return GDML_OK;
  }
  int best = 1;
  float best_ms = 1e30f;
  const bool tcm = c->precision == GDML_TF32 || c->precision == GDML_BF16;
  const int max_s = tcm ? c->tc.splits_cap : c->splits_cap;
  for (int s = 1; s <= max_s; s *= 2) {
    if (!tcm) c->splitsU = s;
    else c->tc.splits2 = s;
    for (int w = 0; w < 2; ++w) TRY(matvec_any(c, v, out, 1, false));
    CTRY(c, cudaEventRecord(e0, c->st));
    for (int w = 0; w < 5; ++w) TRY(matvec_any(c, v, out, 1, false));
    CTRY(c, cudaEventRecord(e1, c->st));
    CTRY(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!tcm) c->splitsU = best;
  else c->tc.splits2 = best;
  drop_graphs(c);
  if (choice_out) *choice_out = best;
  return GDML_OK;
}

gdml_status gdml_set_tuning(gdml_ctx* c, int32_t splits) {
  TRY(validate(c));
  if (c->precision == GDML_OZAKI) {  // g1 * 65536 + g2: K chunks per CTA of the two sliced GEMMs
    const int g1 = splits >> 16, g2 = splits & 0xFFFF;
    if (g1 < 1 || g1 > c->oz.W1.nchunks || g2 < 1 || g2 > c->oz.nch2)
      return ctx_fail(c, GDML_ERR_ARG, "chunks per CTA out of range");
    c->oz.g1 = g1;
    c->oz.g2 = g2;
    drop_graphs(c);
    return GDML_OK;
  }
  const bool tcm = c->precision == GDML_TF32 || c->precision == GDML_BF16;
  const int cap = tcm ? c->tc.splits_cap : c->splits_cap;
  if (splits < 1 || splits > cap) return ctx_fail(c, GDML_ERR_ARG, "split count out of range");
  if (!tcm) c->splitsU = splits;
  else c->tc.splits2 = splits;
  drop_graphs(c);
  return GDML_OK;
}

gdml_status gdml_tc_check(gdml_ctx* c) {
  TRY(validate(c));
  if (df_precond(c)) TRY(ws_check(c));
  if (c->precision != GDML_TF32 && c->precision != GDML_BF16 && c->precision != GDML_OZAKI) return GDML_OK;
  gdml_status s = c->precision == GDML_OZAKI ? oz_check(c->oz, c->st) : tc_check(c->tc, c->st);
  if (s != GDML_OK) return ctx_fail(c, s, last_msg());
  return GDML_OK;
}

const char* gdml_last_error(const gdml_ctx* c) {
  if (c) return c->err.c_str();
  return last_msg().c_str();
}

void gdml_destroy(gdml_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  tc_destroy(c->tc);
  oz_destroy(c->oz);
  for (void* p : c->allocs)
    if (p) cudaFree(p);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->hictl) cudaFreeHost(c->hictl);
  delete c;
}

}  // extern "C"
