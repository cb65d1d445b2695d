/*
 * gdml_testing.h -- diagnostic entry points of libgdml, used by the test suite.
 * Same conventions as gdml.h (device pointers, status codes, no exceptions).
 */
#ifndef GDML_TESTING_H
#define GDML_TESTING_H

#include "gdml.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = A B^T on the tcgen05 tensor cores, the building block of the TF32/BF16
 * matvec (Sec. 2.1: the matvec's descriptor contractions).  A: M x K, B: N x K,
 * C: M x N, all row-major FP64 device arrays; A and B are rounded to TF32
 * (bf16 = 0) or BF16 (bf16 = 1) and accumulated in FP32.  Synchronises the
 * stream.  Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA, GDML_ERR_TIMEOUT
 * (a bounded pipeline wait gave up). */
gdml_status gdml_test_tc_gemm(int32_t bf16, const double* A_dev, const double* B_dev, int32_t M, int32_t N,
                              int32_t K, double* C_dev, void* cuda_stream);

/* C = A B^T through the sliced-BF16 tensor-core GEMM of OZAKI contexts (the
 * matvec's descriptor contractions, Sec. 2.1, at FP64-class accuracy).  A: M x K,
 * B: N x K, C: M x N, row-major FP64 device arrays, 1 <= M, N, K <= 2^24; every
 * 256-entry chunk of a row of A and B is split into 7 BF16 slices of 7 bits,
 * chunk products are accumulated exactly in FP32 per slice level, each CTA adds
 * chunks_per_cta consecutive chunks in double-float (< 1: the contexts' automatic
 * choice) and the groups' partials are summed into C as FP64.  levels (1..7) keeps the
 * slice pairs i + j < levels only (0-based slices; 7 is the full product, fewer give the
 * cheaper product of gdml_set_inner_levels).  Synchronises the stream.
 * Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA, GDML_ERR_TIMEOUT (a bounded pipeline
 * wait gave up). */
gdml_status gdml_test_oz_gemm(const double* A_dev, const double* B_dev, int64_t M, int64_t N, int64_t K,
                              int32_t chunks_per_cta, int32_t levels, double* C_dev, void* cuda_stream);

/* The tall product of the OZAKI preconditioner build (Eq. 5's L_k = K_nk L_kk^-T as K_nk
 * times the transposed triangular inverse, and the leverage-score row norms of Sec. 3's
 * estimate): C = A B^T on the sliced-BF16 tensor cores, accumulated over all of K inside
 * each output tile (FP64-class).  A: n x K FP64, COLUMN-major (entry (r, j) at A[j n + r]);
 * B: NB x K FP64, row-major with row stride ldb >= K; tri_b != 0 declares B lower
 * triangular (zero above its diagonal, which must hold: whole K blocks past each tile's
 * diagonal are skipped).  rowsq = 0: out (n x NB, column-major: C[r][c] at out[c n + r])
 * and, if out32 is not NULL, the same as FP32 at out32; out may equal A.  rowsq != 0:
 * out[r] = sum_c C[r][c]^2 (n doubles), out32 unused.  1 <= n <= 2^31, 1 <= K, NB <= 2^24.
 * Synchronises the stream.  Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA,
 * GDML_ERR_TIMEOUT (a bounded pipeline wait gave up). */
gdml_status gdml_test_oz_gemm_tall(const double* A_dev, int64_t n, int64_t K, const double* B_dev, int64_t NB,
                                   int64_t ldb, int32_t tri_b, int32_t rowsq, double* out_dev, float* out32_dev,
                                   void* cuda_stream);

/* The two passes over the FP32-stored factor L_k of the Woodbury apply (Eq. 4) in
 * DF64/OZAKI contexts: t = L^T r and z = (r - L u) / lambda, with exact FP32
 * products of L and the float-pair split of r (u) and double-float sums.  L: n x k
 * FP32 column-major (column j at L + j n), r, z: n FP64, u, t: k FP64, all device
 * arrays owned by the caller.  staged = 1: the TMA-staged kernels the contexts use
 * when n % 4 == 0 (GDML_ERR_ARG otherwise), with their automatic row-chunk size;
 * staged = 128 or 256: the same kernels with that chunk size; staged = 0: the
 * register-streamed kernels used for other n.  Synchronises the stream.  Errors: GDML_ERR_ARG
 * (NULL pointers, n < 1, k < 1 or k > 16384, lambda <= 0), GDML_ERR_OOM,
 * GDML_ERR_CUDA, GDML_ERR_TIMEOUT (a bounded pipeline wait gave up). */
gdml_status gdml_test_df_passes(const float* L_dev, int64_t n, int64_t k, const double* r_dev, const double* u_dev,
                                double lambda, int32_t staged, double* t_dev, double* z_dev, void* cuda_stream);

/* The built preconditioner's factor L_k (Eqs. 3-5) as FP64: n x rank, column-major (column
 * j at L_out_dev + j n, columns in selection / pivot order; rank from gdml_precond_info).
 * DF64 and OZAKI contexts store L_k in FP32; it is widened exactly.  L_out_dev: n * rank
 * doubles owned by the caller.  Synchronises the context's stream.
 * Errors: GDML_ERR_ARG (NULL arguments), GDML_ERR_STATE (nothing built), GDML_ERR_CUDA. */
gdml_status gdml_test_precond_factor(gdml_ctx* ctx, double* L_out_dev);

/* Reads and clears the error words of the tensor-core kernels of a TF32/BF16/OZAKI
 * context and of the staged Woodbury passes of a DF64/OZAKI context (synchronises
 * its stream); GDML_ERR_TIMEOUT if a pipeline wait gave up since the last check.
 * FP64 contexts: always GDML_OK. */
gdml_status gdml_tc_check(gdml_ctx* ctx);

/* Fault injection from the host for the bounded device waits: every mbarrier wait of the
 * library's tcgen05 / TMA pipelines (the TF32/BF16 and sliced GEMMs, the staged Woodbury
 * passes and Schur sums) gives up after `polls` polls instead of its default (about 2^26,
 * seconds).  polls = 0 makes each wait give up at once: the waiting role then issues no copy
 * and no MMA, records GDML_ERR_TIMEOUT in the kernel's error word (read by gdml_tc_check) and
 * the CTA still releases its tensor memory, so the context stays usable.  polls = 0xFFFFFFFF
 * restores the default.  Applies to all contexts and devices' kernels launched after the call
 * on the current device; not thread-safe with concurrent launches.  Errors: GDML_ERR_CUDA. */
gdml_status gdml_test_set_wait_limit(uint32_t polls);

/* The FP64 Cholesky of the preconditioner build with the jitter rule of Eq. 5's reading
 * (if A is not positive definite, eps = 1e-14 tr(A)/k is added to the diagonal and
 * multiplied by 10 per retry up to 1e-6 tr(A)/k) on a caller matrix: A_dev k x k row-major
 * FP64 (only its lower triangle is read), L_dev k x k receives the factor in its lower
 * triangle (the strict upper triangle is unspecified), *eps_out (host) the jitter used.
 * Synchronises the stream.  Errors: GDML_ERR_ARG, GDML_ERR_OOM, GDML_ERR_CUDA,
 * GDML_ERR_NOT_SPD (still not positive definite at the largest jitter). */
gdml_status gdml_test_cholesky_jitter(const double* A_dev, int64_t k, double* L_dev, double* eps_out,
                                      void* cuda_stream);

/* Replaces the context's lambda by any finite value -- zero or negative included, which makes
 * K + lambda I indefinite, so that a test can drive PCG into its breakdown status
 * (GDML_ERR_BREAKDOWN: p^T K_lambda p <= 0).  Drops the built preconditioner (rank 0) and the
 * captured PCG graphs.  Errors: GDML_ERR_ARG (NULL context, non-finite lambda). */
gdml_status gdml_test_set_lambda(gdml_ctx* ctx, double lambda);

/* Kernel launches this library has executed since it was loaded (all
 * contexts and threads; a kernel inside a CUDA graph counts once per replay).
 * Host-side counter, never fails. */
int64_t gdml_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GDML_TESTING_H */
