/*
 * gdml.h -- C ABI of libgdml: preconditioned conjugate-gradient training of
 * a GDML force-field kernel model on one NVIDIA GB300 (sm_103a).
 *
 * The problem (Sec. 2.1, Eq. 1): given M training geometries of N atoms and
 * force labels y, solve  (K + lambda I_n) alpha = y,  n = 3 N M, where K is
 * the force kernel made of 3N x 3N blocks K_ab = J_a^T H_ab J_b:
 *   descriptor  x_p = 1/|R_i - R_j| (pairs i > j, p = i(i-1)/2 + j, D = N(N-1)/2),
 *   J_a = dx_a/dR_a,  H_ab = (c^2/3) e^{-c r} [(1 + c r) I - c^2 d d^T],
 *   d = x_a - x_b, r = |d|, c = sqrt(5)/sigma  (Matern-5/2 kernel).
 * The solve is PCG (Sec. 2.1, Eq. 2) with the Nystrom-type preconditioner
 *   P = L_k L_k^T + lambda I                                (Eq. 3),
 *   P^-1 = lambda^-1 [I - L_k (lambda I + L_k^T L_k)^-1 L_k^T]  (Eq. 4),
 * whose k inducing columns are chosen by uniform sampling, ridge leverage
 * scores, or the incomplete (pivoted) Cholesky of App. A.2, Algorithm 1.
 *
 * Conventions for every entry point
 *  - Vector layout: index a*3N + 3*i + q (geometry a, atom i, coordinate q);
 *    this is the reshape n -> (n_train, d, 3) of App. A.
 *  - Pointers named *_dev are device pointers on the context's device, at
 *    least 8-byte aligned; all work is ordered on the context's stream.
 *    The caller owns every pointer it passes; the context keeps none of them
 *    after the call returns.  The context owns its own device workspace.
 *  - Nothing throws across the ABI.  Every call returns a gdml_status;
 *    gdml_last_error() gives a message for the last failure on a context.
 *  - Calls on one context must not run concurrently from several host threads.
 */
#ifndef GDML_H
#define GDML_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gdml_ctx gdml_ctx;

typedef enum {
  GDML_OK = 0,
  GDML_ERR_ARG = 1,           /* invalid argument (sizes, pointers, enum values) */
  GDML_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  GDML_ERR_OOM = 3,           /* device allocation failed */
  GDML_ERR_NOT_SPD = 4,       /* a Cholesky pivot was not positive (even after jitter) */
  GDML_ERR_BREAKDOWN = 5,     /* PCG: p^T K p <= 0 or not finite */
  GDML_ERR_NOT_CONVERGED = 6, /* PCG hit max_iter; alpha holds the last iterate */
  GDML_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  GDML_ERR_STATE = 8          /* call order violated (e.g. apply before build) */
} gdml_status;

/* Arithmetic of the kernel matvec K v (Sec. 2.1: CG only needs matvecs).
 * FP64: every step in IEEE double.
 * TF32 / BF16: the two descriptor contractions of the matvec run on the
 * tcgen05 tensor cores (TF32 or BF16 operands, FP32 accumulation); PCG then
 * runs as the inner solver of an FP64 iterative refinement whose residual
 * y - K_lambda alpha is recomputed with the FP64 matvec. */
/* DF64: the two descriptor contractions run in double-float arithmetic on
 * the FP32 lanes (each FP64 operand split into two floats, exact products by
 * FMA, (hi, lo) accumulation by TwoSum; ~2^-46 relative per term), i.e.
 * FP64-class accuracy at the FP32 rate.  PCG uses it inside the loop and
 * recomputes the TRUE residual with the FP64 matvec, restarting (refining)
 * from the current iterate until it converges (at most 10 restarts). */
/* OZAKI: the two descriptor contractions run on the BF16 tensor cores with
 * FP64-class accuracy.  Each 256-entry chunk of an operand row is scaled by a
 * power of two and cut into 7 exact BF16 integer slices of 7 bits (49 bits);
 * slice pairs whose products are kept (i + j <= 8 counting slices from 1: 28 of 49) are accumulated exactly in
 * FP32 per level, combined in double-float and summed across chunks (the
 * error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012; ~1e-14 relative
 * matvec error).  Preconditioner and PCG as for DF64.  Operand magnitudes must
 * stay inside the FP32 range (|x| < 1e38). */
typedef enum { GDML_FP64 = 0, GDML_TF32 = 1, GDML_BF16 = 2, GDML_DF64 = 3, GDML_OZAKI = 4 } gdml_precision;

/* Inducing-column selection rule (Sec. 3, "Column selection strategies"). */
typedef enum {
  GDML_SEL_UNIFORM = 0, /* k distinct columns, uniformly at random */
  GDML_SEL_RLS = 1,     /* sampled without replacement by estimated ridge leverage scores */
  GDML_SEL_PIVCHOL = 2, /* incomplete Cholesky with greedy diagonal pivoting (Alg. 1) */
  GDML_SEL_WEIGHTED = 3, /* sampled without replacement by given per-geometry scores (learned scorer) */
  GDML_SEL_SVD = 4       /* the k dominant eigenpairs of K: the optimal rank-k reference (Sec. 2.2, App. A.1) */
} gdml_select;

/* Build a context for one kernel system (Sec. 2.1, Eq. 1).
 *  R_dev:  M*N*3 doubles, geometry a atom i coordinate q at (a*N + i)*3 + q, Angstrom.
 *  M >= 1 geometries, 2 <= N <= 128 atoms, sigma > 0 (Matern length scale),
 *  lambda > 0 (ridge), precision: a gdml_precision value.
 *  cuda_stream: a cudaStream_t on the current device, or NULL for the legacy stream.
 * Computes descriptors, Jacobians, the M x M descriptor-distance tables and
 * diag(K) on the device.  On success *ctx owns that state until gdml_destroy.
 * Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA (then *ctx is NULL). */
gdml_status gdml_kernel_setup(gdml_ctx** ctx, const double* R_dev, int64_t M, int32_t N,
                              double sigma, double lambda, int32_t precision, void* cuda_stream);

/* A context for the symmetric (sGDML) force kernel.  The paper's runtimes include the
 * molecules' permutational symmetries, and its kernel's forward pass grows with their number
 * (Sec. 4.3, "Remarks on runtime").  The kernel is
 *   K_ab = sum_q J_a^T H(x_a, P_q x_b) P_q J_b,
 * the force kernel of kappa_S(R_a, R_b) = sum_q kappa(x(R_a), x(R_b with its atoms permuted by
 * sigma_q)), where P_q permutes descriptor entries: (P_q x)_(i,j) = x_(sigma_q(i), sigma_q(j)).
 *  perms_host: S x N int32 (host memory), row q = sigma_q; sigma_q[i] is the atom that takes
 *    atom i's place.  The S rows must form a group: each a permutation of 0..N-1, the identity
 *    among them, closed under composition, and no row repeated.  1 <= S <= 256.
 *  precision: GDML_FP64 or GDML_OZAKI when S > 1.
 *  Every other argument is as for gdml_kernel_setup.
 * Every entry point then uses the symmetric kernel: matvec, preconditioner builds, PCG and
 * prediction.  Costs:
 *  - the matvec's two contractions and the M x M setup tables grow by a factor S;
 *  - kernel columns (the preconditioner builds) are computed in FP64, which limits N to about
 *    70 atoms.
 * S = 1 (the identity alone) gives the plain kernel.
 * Errors: GDML_ERR_ARG (as gdml_kernel_setup, or perms_host NULL / not a group / a precision
 * other than FP64 or OZAKI with S > 1), GDML_ERR_OOM, GDML_ERR_CUDA (then *ctx is NULL). */
gdml_status gdml_kernel_setup_sym(gdml_ctx** ctx, const double* R_dev, int64_t M, int32_t N,
                                  const int32_t* perms_host, int32_t S, double sigma, double lambda,
                                  int32_t precision, void* cuda_stream);

/* out = K v (+ lambda v if add_lambda), both length n = 3 N M, in the
 * context's precision (FP64 contexts: FP64; TF32/BF16: tensor-core matvec
 * with FP32 accumulation, result stored as double; DF64: double-float
 * contractions; OZAKI: sliced-BF16 tensor-core contractions).  v_dev and out_dev must
 * not overlap.  The matvec is matrix-free: w_b = J_b v_b, u_a = sum_b H_ab w_b,
 * (K v)_a = J_a^T u_a (Sec. 2.1: CG touches K only through such products,
 * so K is never formed).
 * Errors: GDML_ERR_ARG (NULL context, NULL or equal pointers), GDML_ERR_CUDA; a timed-out
 * tensor-core pipeline wait is reported by gdml_tc_check. */
gdml_status gdml_matvec(gdml_ctx* ctx, const double* v_dev, double* out_dev, int32_t add_lambda);

/* Same as gdml_matvec but always in FP64, whatever the context precision.
 * Errors as gdml_matvec. */
gdml_status gdml_matvec_fp64(gdml_ctx* ctx, const double* v_dev, double* out_dev, int32_t add_lambda);

/* Forces the trained model predicts for Q query geometries of the context's molecule
 * (Sec. 2.1: predictions cost time linear in the training set):
 *   f_q = sum_b J_q^T H(x_q, x_b) J_b alpha_b,
 * the force-kernel blocks of the queries against the M training geometries applied to
 * alpha, the solution of Eq. 1 (for example from gdml_pcg_solve).  Computed in FP64 in
 * every context precision.  No lambda term: at a training geometry f = (K alpha)_q.
 *  R_query_dev: Q*N*3 doubles, layout as R_dev of gdml_kernel_setup (same N).
 *  alpha_dev: n = 3 N M doubles.  f_dev: Q*N*3 doubles (layout as R_query_dev),
 *  must not overlap alpha_dev.  1 <= Q <= 2^20; temporary device memory of about
 *  8 Q (4 M + 6 D) bytes is allocated and freed inside the call.
 * Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA. */
gdml_status gdml_predict_forces(gdml_ctx* ctx, const double* R_query_dev, int64_t Q, const double* alpha_dev,
                                double* f_dev);

/* Build the Nystrom-type preconditioner (Eqs. 3-5, Sec. 3, Alg. 1).
 *  method: gdml_select; 1 <= k <= min(n, 16384); seed: Philox4x32-10 key
 *  (uniform: counter (i, 0), rls pilot: (i, 1), rls sampling: (i, 2)).
 *  pivots_dev (may be NULL): k int64 column indices in selection order
 *    (uniform/rls: ascending key; pivchol: pivot order of Alg. 1).
 *  resid_trace_dev (may be NULL): k doubles; for pivchol the sum of the
 *    residual diagonal after each step (monotone, Sec. 3), for SVD see below,
 *    else zeros.
 * Uniform/RLS: L_k = K_nk L_kk^-T with K_kk = L_kk L_kk^T (Eq. 5); if that
 * Cholesky fails, jitter eps = 1e-14 tr(K_kk)/k is added and multiplied by 10
 * per retry up to 1e-6 tr(K_kk)/k.  Pivchol: L_k from Alg. 1 (stops early,
 * with a smaller rank, if the largest residual diagonal is <= 0).
 * SVD (GDML_SEL_SVD; the paper's optimal but O(n^3)-costly reference, for small n): K is
 * PSD, so its SVD is its eigendecomposition K = U Sigma U^T; the preconditioner is
 * P = U_k Sigma_k U_k^T + lambda I, i.e. L_k = U_k Sigma_k^(1/2) (the k largest eigenvalues,
 * negative rounding clamped to 0).  K is assembled densely from the kernel columns and
 * decomposed by cuSOLVER's syevd (loaded from libcusolver on first use); n <= 24576, and
 * about 24 n^2 bytes of device memory are allocated and freed inside the call.  No pivots
 * (pivots_dev receives -1); resid_trace_dev[m] = tr(K) minus the m + 1 largest eigenvalues.
 * Then C = lambda I + L_k^T L_k and its FP64 Cholesky factor (Eq. 4).
 * Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_NOT_SPD, GDML_ERR_CUDA (also when libcusolver
 * cannot be loaded for GDML_SEL_SVD). */
gdml_status gdml_precond_build(gdml_ctx* ctx, int32_t method, int64_t k, uint64_t seed,
                               int64_t* pivots_dev, double* resid_trace_dev);

/* Number of inducing columns k for gdml_precond_build by the rule of thumb of
 * Sec. 4.3 (Eqs. 7-8): the integer k in [1, n] that minimises the runtime model
 *   (k_min / k)^m + (k / n)^2,
 * a PCG cost that falls as a power law in k plus a k^2 n build cost.  A tie
 * between two integers goes to the smaller k.  m and k_min are the molecule's
 * fitted parameters (Table 1); the default row is m = 1, k_min = 100.
 * Host arithmetic only (no context, no device); *k_out is a host int64.
 * Errors: GDML_ERR_ARG unless n >= 1, m and k_min finite and > 0, k_out != NULL
 * (message through gdml_last_error(NULL)). */
gdml_status gdml_rule_of_thumb_k(int64_t n, double m, double k_min, int64_t* k_out);

/* Preconditioner from k columns sampled without replacement with weights
 * w_i = max(score_a, 0) * K_ii for column i of geometry a (keys -ln(u_i)/w_i,
 * Philox stream 3), then the Nystrom factor and Woodbury core exactly as for
 * GDML_SEL_UNIFORM / GDML_SEL_RLS (Eqs. 3-5).  geometry_scores_dev: M doubles,
 * e.g. a learned scorer's prediction of each geometry's ridge leverage mass
 * (the paper samples by the leverage scores themselves, Sec. 3).
 * Errors as gdml_precond_build. */
gdml_status gdml_precond_build_scored(gdml_ctx* ctx, const double* geometry_scores_dev, int64_t k, uint64_t seed,
                                      int64_t* pivots_dev);

/* The Nystrom estimate of the ridge leverage scores tau_i = (K (K + lambda I)^-1)_ii
 * (Sec. 3) that GDML_SEL_RLS samples by: pilot of k uniform columns (Philox
 * stream 1), B = K_nS L_S^-T, tau_i = b_i^T (B^T B + lambda I)^-1 b_i.
 * tau_dev: n doubles.  Invalidates any built preconditioner (rank 0).
 * Errors: GDML_ERR_ARG (NULL tau_dev, k outside [1, min(n, 16384)]), GDML_ERR_OOM,
 * GDML_ERR_NOT_SPD, GDML_ERR_CUDA. */
gdml_status gdml_rls_scores(gdml_ctx* ctx, int64_t k, uint64_t seed, double* tau_dev);

/* Per-geometry ridge-leverage mass, the training label of the learned scorer:
 * labels[a] = sum over the 3N columns i of geometry a of tau_i (summed in index order).
 *  exact != 0: the exact scores tau_i = (K (K + lambda I)^-1)_ii = sum_j U_ij^2 s_j / (s_j + lambda)
 *    from the eigendecomposition K = U diag(s) U^T (dense K from the kernel columns, cuSOLVER
 *    syevd; negative rounding of s clamped to 0; n <= 24576, ~24 n^2 bytes of temporary device
 *    memory).  At lambda far below the rounding of K's small eigenvalues (~n eps |K|) the scores
 *    of those eigen-directions are as uncertain as the eigenvalues themselves.  k, seed unused.
 *  exact == 0: the Nystrom estimate of gdml_rls_scores (pilot k, seed), which invalidates any
 *    built preconditioner.
 * labels_dev: M doubles.  Synchronises the stream.
 * Errors: GDML_ERR_ARG (NULL labels_dev, n too large for exact, k outside [1, min(n, 16384)]),
 * GDML_ERR_OOM, GDML_ERR_NOT_SPD, GDML_ERR_CUDA. */
gdml_status gdml_rls_labels(gdml_ctx* ctx, int32_t exact, int64_t k, uint64_t seed, double* labels_dev);

/* The inverse-distance descriptors x_a (M x D doubles, row a = geometry a).
 * Errors: GDML_ERR_ARG (NULL context or X_dev), GDML_ERR_CUDA. */
gdml_status gdml_descriptors(const gdml_ctx* ctx, double* X_dev);

/* Rank actually built by the last gdml_precond_build (pivchol may stop early),
 * and the jitter added to K_kk (0 if none).  Host outputs; either may be NULL.
 * Errors: GDML_ERR_ARG (NULL context). */
gdml_status gdml_precond_info(const gdml_ctx* ctx, int64_t* rank_out, double* jitter_out);

/* z = P^-1 r by the Woodbury identity (Eq. 4).  r_dev, z_dev: length n, may
 * not overlap.  Errors: GDML_ERR_STATE if no preconditioner was built. */
gdml_status gdml_precond_apply(gdml_ctx* ctx, const double* r_dev, double* z_dev);

/* Solve K_lambda alpha = y by PCG (Sec. 2.1, Eq. 2), x0 = alpha_dev's
 * contents on entry (pass zeros for the paper's cold start).  The stopping
 * test is the TRUE relative residual |y - K_lambda alpha|_2 / |y|_2 <= rtol,
 * recomputed in FP64 when the recurrence residual passes (restart from alpha
 * if it has drifted: at most 3 times in FP64 contexts, 10 times in DF64 and
 * OZAKI contexts, whose FP64-class matvec drifts more).  TF32/BF16 contexts run FP64 iterative
 * refinement: the inner PCG uses the tensor-core matvec and stops at
 * inner_rtol relative to its own right-hand side; the outer loop recomputes
 * r = y - K_lambda alpha with the FP64 matvec (at most 20 outer steps).
 * Uses the preconditioner if one was built, else P = I.
 *  iters_out (host, may be NULL): total inner PCG iterations.
 *  relres_out (host, may be NULL): final true relative residual (FP64).
 * Synchronises the context's stream before returning.
 * Errors: GDML_ERR_NOT_CONVERGED (alpha holds the best iterate),
 * GDML_ERR_BREAKDOWN, GDML_ERR_ARG, GDML_ERR_CUDA. */
gdml_status gdml_pcg_solve(gdml_ctx* ctx, const double* y_dev, double* alpha_dev, double rtol,
                           int32_t max_iter, int32_t* iters_out, double* relres_out);

/* Spectrum diagnostics of the last gdml_pcg_solve (Sec. 4.1, Fig. 3: the convergence of PCG
 * follows the spectrum of P^-1 K_lambda).  The first CG run of that solve (before any
 * true-residual restart; for TF32/BF16 contexts the first inner solve) recorded its step
 * lengths gamma_j = rho_j / p_j^T K_lambda p_j and ratios beta_j = rho_(j+1) / rho_j on the
 * device.  They define the Lanczos tridiagonal matrix T_m of P^-1 K_lambda,
 *   T[0,0] = 1/gamma_0, T[j,j] = 1/gamma_j + beta_(j-1)/gamma_(j-1),
 *   T[j,j+1] = T[j+1,j] = sqrt(beta_j)/gamma_j   (m = the run's iterations, at most 20000),
 * whose eigenvalues (Ritz values) lie within the spectrum of P^-1 K_lambda and converge to its
 * extreme eigenvalues as the run proceeds; theta_max / theta_min estimates cond(P^-1 K_lambda)
 * from below.  Host arithmetic (bisection on Sturm counts, O(m) per bisection step).
 *  count (0..1024): how many of the largest Ritz values to write to ritz_host (host array,
 *    descending; entries beyond m are NaN); ritz_host may be NULL when count is 0.
 *  theta_min, theta_max, steps_out (host, each may be NULL): the extreme Ritz values and m.
 * Errors: GDML_ERR_STATE (no solve recorded coefficients: none yet, the last solve had y = 0
 * or was batched), GDML_ERR_ARG, GDML_ERR_CUDA. */
gdml_status gdml_pcg_spectrum(gdml_ctx* ctx, int32_t count, double* ritz_host, double* theta_min, double* theta_max,
                              int32_t* steps_out);

/* Inner tolerance of the mixed-precision refinement (default 1e-3 for BF16,
 * 1e-4 for TF32; ignored in FP64 contexts).
 * Errors: GDML_ERR_ARG unless 0 < inner_rtol < 1. */
gdml_status gdml_set_inner_rtol(gdml_ctx* ctx, double inner_rtol);

/* Slice levels of the matvec inside the PCG loop of an OZAKI context: mixed precision with a
 * cheaper inner operator and FP64 true residuals.  levels = 7 (the default) is the full product;
 * levels < 7 keeps only the slice pairs i + j < levels (slices counted from 0) in both
 * contractions: fewer tensor-core products (28, 21, 15, 10 for 7, 6, 5, 4 levels) and a matvec
 * error of roughly 2^-(7 levels - 2) relative to |K||v| instead of ~1e-14.  The recurrence then
 * solves a slightly perturbed system; gdml_pcg_solve recomputes the true residual with the FP64
 * matvec whenever the recurrence passes and restarts PCG from alpha (at most 10 times), so the
 * reported residual is the FP64 one.  gdml_matvec and the build are not affected.
 * Errors: GDML_ERR_ARG (not an OZAKI context, levels outside 1..7). */
gdml_status gdml_set_inner_levels(gdml_ctx* ctx, int32_t levels);

/* Outer refinement steps of the last gdml_pcg_solve: for FP64, DF64 and OZAKI contexts the
 * number of PCG runs (1 + true-residual restarts); for TF32/BF16 the refinement steps.
 * Errors: GDML_ERR_ARG (NULL context). */
gdml_status gdml_last_outer_steps(const gdml_ctx* ctx, int32_t* outer_out);

/* Solve count independent systems (each set up by its own FP64, DF64 or OZAKI
 * context, any sizes, sigma and lambda) with ONE CUDA graph launch per round: the graph
 * holds, per system, a gate kernel and a conditional WHILE node whose body is
 * that system's PCG iteration (Sec. 2.1, Eq. 2, as in gdml_pcg_solve), so the
 * loops of all systems run concurrently on the device.  Between rounds the
 * host recomputes each active system's TRUE FP64 residual and restarts the
 * ones that drifted (at most 3 restarts for FP64 contexts, 10 for DF64 and
 * OZAKI, as gdml_pcg_solve; at most 12 rounds in all).
 *  ctxs, y_dev, alpha_dev: host arrays of count entries (device vectors of
 *    each context's length n_i; alpha_dev holds x0 on entry, the solution on exit).
 *  iters_out, relres_out (host arrays of count entries, may be NULL).
 * All contexts must be FP64, DF64 or OZAKI contexts on the current device, each at most once
 * (TF32 / BF16 contexts, whose solve is an iterative refinement, are rejected).
 * Synchronises every context's stream.  Errors: GDML_ERR_ARG,
 * GDML_ERR_NOT_CONVERGED (some system above rtol), GDML_ERR_BREAKDOWN, GDML_ERR_CUDA. */
gdml_status gdml_pcg_solve_batched(gdml_ctx* const* ctxs, int32_t count, const double* const* y_dev,
                                   double* const* alpha_dev, double rtol, int32_t max_iter,
                                   int32_t* iters_out, double* relres_out);

/* Tile autotuner for the matvec of this context's shapes.  FP64, DF64, TF32 and BF16
 * contexts: times every power-of-two K-split (1 .. 8 or more) of the second descriptor
 * contraction (FP64 DGEMM or tcgen05 GEMM) and keeps the fastest.  OZAKI contexts: times the
 * number of 256-entry K chunks each CTA of the two sliced GEMMs accumulates in registers
 * (GEMM 1: 1 or all; GEMM 2: 1, 2, 3, 4, 8, ... up to all, counting the chunks of both of its
 * K segments when they run as one product) and keeps the fastest pair.
 * *choice_out (host, may be NULL) receives the choice (OZAKI: g1 * 65536 + g2) so that a
 * caller can cache it and restore it later with gdml_set_tuning.  Synchronises the
 * context's stream.  Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA. */
gdml_status gdml_autotune(gdml_ctx* ctx, int32_t* choice_out);
gdml_status gdml_set_tuning(gdml_ctx* ctx, int32_t splits);

/* out = K v (+ lambda v if add_lambda) for M geometries R_dev (same layout as
 * gdml_kernel_setup), computed in FP64 WITHOUT a context and WITHOUT any device
 * allocation -- for callers that cannot call cudaMalloc: code that runs while
 * another runtime owns the device memory (a framework's caching allocator or
 * a fixed pre-reserved budget), real-time loops where an allocation could
 * block or fail, or work recorded between pre-allocated buffers only.
 * The paper has no counterpart; this is a deployment variant of gdml_matvec.
 *  Limits: 1 <= M <= 128 geometries, 2 <= N <= 24 atoms (GDML_ERR_ARG beyond).
 *  Working memory: one static device array of 2.5 MB that every GPU loading
 *    this library holds until process exit; every call overwrites what it uses,
 *    so nothing needs clearing between calls.
 *  The first call on each device looks the array's address up (with that
 *    device current), so make that first call before any stream capture.
 *  The looked-up address belongs to the device's primary context: it does not
 *    survive cudaDeviceReset, and code running under another context of the
 *    device must not call this entry point.
 *  Calls that overlap on the GPU (two streams, or two host threads on one
 *    device) share the array and race; serialise them.
 *  R_dev, v_dev, out_dev: caller-owned device arrays on the current device
 *    (v_dev != out_dev), v_dev and out_dev holding 3 N M doubles each;
 *  cuda_stream: a cudaStream_t of the current device, or NULL.
 * Errors: GDML_ERR_ARG (sizes beyond the limits, NULL or equal pointers, a stream
 * of another device), GDML_ERR_CUDA. */
gdml_status gdml_matvec_noalloc(const double* R_dev, int64_t M, int32_t N, double sigma, double lambda,
                                const double* v_dev, double* out_dev, int32_t add_lambda, void* cuda_stream);

/* Learned inducing-column scorer: a BF16 MLP D -> hidden -> hidden -> 1 with
 * exact-erf GELU, FP32 master weights and accumulation, trained by Adam
 * (beta 0.9 / 0.999) on mean-squared error.  Its per-geometry scores feed
 * gdml_precond_build_scored; pivoted Cholesky (Alg. 1) stays the fallback and
 * the referee (by PCG iteration count) of its selections.  The paper has no
 * learned selection; its leverage-score sampling (Sec. 3) supplies the labels. */
typedef struct gdml_scorer gdml_scorer;
/* A scorer for D descriptor features with two hidden layers of width `hidden`, weights drawn
 * from `seed`; *s owns its device memory until gdml_scorer_destroy.
 * Errors: GDML_ERR_ARG (NULL s, D outside [1, 65536], hidden outside [1, 4096]), GDML_ERR_OOM,
 * GDML_ERR_CUDA. */
gdml_status gdml_scorer_create(gdml_scorer** s, int32_t D, int32_t hidden, uint64_t seed, void* cuda_stream);
/* feature mean/std per column and label mean/std from training data X (B x D), y (B)
 * Errors: GDML_ERR_ARG (NULL arguments, B < 2), GDML_ERR_CUDA. */
gdml_status gdml_scorer_fit_scaling(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B);
/* `epochs` passes of Adam (learning rate lr) over the B rows of X (B x D) and labels y (B) in
 * mini-batches of `batch`; last_loss_out (host, may be NULL) gets the last mini-batch's
 * mean-squared error on standardised labels.
 * Errors: GDML_ERR_ARG (NULL arguments, B, epochs or batch < 1, lr <= 0), GDML_ERR_OOM,
 * GDML_ERR_CUDA. */
gdml_status gdml_scorer_train(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B, int32_t epochs,
                              int32_t batch, double lr, double* last_loss_out);
/* out (B doubles) = the scorer's prediction for the B rows of X (B x D), in label units.
 * Errors: GDML_ERR_ARG (NULL arguments, B < 1), GDML_ERR_OOM, GDML_ERR_CUDA. */
gdml_status gdml_scorer_predict(gdml_scorer* s, const double* X_dev, int64_t B, double* out_dev);
/* flat FP32 parameters [W1 (h x D) | b1 | W2 (h x h) | b2 | w3 | b3]: get (set = 0) or set (set = 1)
 * params_dev = NULL only reports the count. Errors: GDML_ERR_ARG (NULL scorer), GDML_ERR_CUDA. */
gdml_status gdml_scorer_params(gdml_scorer* s, float* params_dev, int32_t set, int64_t* nparam_out);
/* loss (host) and its gradient w.r.t. the flat parameters (device) on one batch
 * Errors: GDML_ERR_ARG (NULL arguments, B < 1), GDML_ERR_OOM, GDML_ERR_CUDA. */
gdml_status gdml_scorer_grad(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B, double* loss_out,
                             float* grad_dev);
/* Waits for the scorer's stream and frees its device memory (NULL is allowed). Never fails. */
void gdml_scorer_destroy(gdml_scorer* s);

/* Message describing the last error on ctx (or, when ctx is NULL, the last
 * failed call without a context on this thread: setup, rule_of_thumb_k).
 * Never NULL; valid until the next call on the context.
 * Never fails. */
const char* gdml_last_error(const gdml_ctx* ctx);

/* Release all device memory owned by ctx (NULL is allowed).
 * Never fails. */
void gdml_destroy(gdml_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GDML_H */
