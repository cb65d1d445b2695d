// FP64-accurate force-kernel matvec on the BF16 tensor cores (GDML_OZAKI contexts).
//
// The two descriptor contractions of K v (the same algebra as the FP64 path),
//   GEMM 1:  T = Xc W^T                              (M x M, K = D)
//   GEMM 2:  U = A W + beta Xc                       (M x D, K = M, two segments run as
//                                                     one product over the concatenated K)
// are computed by an error-free splitting in the manner of Ozaki, Ogita, Oishi and
// Rump (2012), "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications":
//
//   * every operand row is cut into chunks of KC = 256 entries along K; within a
//     chunk the row is scaled by a power of two 2^e (e from the chunk's largest
//     magnitude) and written as  x = 2^e * sum_{i<7} s_i 2^{-7(i+1)}  with integer
//     slices |s_1| <= 128, |s_i| <= 64 (i > 1), each exact in BF16 (49 bits in all);
//   * the product of one slice pair is an integer of magnitude at most 2^14, so the FP32
//     tensor-core accumulation of one chunk is exact: every level sum
//     sum_{i+j=l} s_i t_j over 256 K entries stays below 2^24;
//   * slice pairs with i + j <= 8 (1-based) are kept, one TMEM accumulator per
//     level i + j; the levels are combined in double-float arithmetic and scaled by
//     2^(eA + eB), giving one double-float partial per chunk; partials are summed
//     by the consumer.
//
// The projection, the nonlinear step between the GEMMs (beta = c^2 S (T - t)) and the
// back-projection run in double-float arithmetic (GB300's FP64 pipe is ~1/64 of its FP32 rate).  Relative error of the matvec is
// ~1e-14 (FP64-class), so the plain PCG reaches 1e-8 at lambda = 1e-10.
#pragma once
#include <cuda.h>

#include <vector>

#include "common.cuh"

namespace gdml {

namespace oz {
constexpr int S = 7;         // slices per operand
constexpr int BITS = 7;      // bits per slice
constexpr int KC = 256;      // K entries per exactly accumulated chunk
constexpr int KB = 64;       // K entries per k-block (one 128-byte BF16 span)
constexpr int BM = 128;      // rows per tile (UMMA M)
constexpr int BN = 64;       // columns per tile (UMMA N)
}  // namespace oz

// one operand in sliced form: S slice matrices of rows x Kp BF16 (zero padded),
// stacked as S * Rp rows, plus an exponent per (chunk, row)
struct OzOperand {
  void* slices = nullptr;  // __nv_bfloat16[S][Rp][Kp]
  int* e = nullptr;        // [nchunks][rows]
  int64_t rows = 0, Rp = 0, K = 0, Kp = 0, nchunks = 0;
  CUtensorMap map;
};

struct OzMatvec {
  bool ready = false;
  int64_t M = 0;   // rows a (the geometries)
  int64_t MB = 0;  // training-side rows: M, or M S with S permutational symmetries (row b S + q)
  int N = 0, D = 0;
  int S = 1;                     // symmetries
  const int* pis = nullptr;      // S x D descriptor-entry permutations (S > 1)
  const double* XcB = nullptr;   // MB x D centred training-side descriptors (S > 1)
  OzOperand Xc1;  // GEMM 1 A: Xc (rows a, K = D), fixed
  OzOperand W1;   // GEMM 1 B: W (rows b, K = D), per matvec
  OzOperand A2;   // GEMM 2 segment 1 A: A (rows a, K = b), fixed
  OzOperand WT2;  // GEMM 2 segment 1 B: W^T (rows d, K = b), per matvec
  OzOperand B2;   // GEMM 2 segment 2 A: beta (rows a, K = b), per matvec
  OzOperand XT2;  // GEMM 2 segment 2 B: Xc^T (rows d, K = b), fixed
  double* W = nullptr;    // M x D (FP64 projection)
  float2* Wf = nullptr;   // M x D: the projection as float pairs (double-float path, S = 1)
  float2* Xc2 = nullptr;  // M x D: the centred descriptors as float pairs
  double* WB = nullptr;   // MB x D: the projection on the training side (S > 1)
  double* WT = nullptr;   // D x MB
  double* t = nullptr;    // M: t_b = xc_b . w_b
  float2* t2 = nullptr;   // M: t_b as a double-float pair
  float2* S2 = nullptr;   // M x M: c^2 S_ab as double-float pairs
  float2* Tp = nullptr;   // [W1.nchunks][M][M] partials of T
  float2* Up = nullptr;   // [2 * A2.nchunks][M][D] partials of U
  float2* rs2 = nullptr;  // [A2.nchunks][M] partial row sums of beta
  int* err = nullptr;
  int g1 = 1, g2 = 1;  // K chunks per CTA of GEMM 1 and GEMM 2 (tuned by gdml_autotune)
  // GEMM 2's two segments (A W and beta Xc) run as one product over the concatenated K when
  // the first ends on a 256-entry chunk boundary; nch2 = GEMM 2's chunks per output
  bool u_merged = false;
  int64_t nch2 = 0;
  std::vector<void*> allocs;
};

// Xc: the M rows' centred descriptors.  Without symmetries (S = 1) the training side is the
// same M geometries (XcB = Xc, A and S are M x M).  With S > 1 symmetries the training side has
// MB = M S rows b S + q (XcB: MB x D, pis: S x D device permutations), A and S are M x MB.
gdml_status oz_setup(OzMatvec& oz, int64_t M, int N, int D, const double* Xc, const double* A, int64_t ldA,
                     const double* S, double c, cudaStream_t st, int Ssym = 1, const int* pis = nullptr,
                     const double* XcB = nullptr);
// out = K v (+ lambda v); G, Xc: the context's FP64 Jacobian factors and centred descriptors,
// G2 the Jacobian factors as float pairs (the projection and back-projection run in
// double-float arithmetic).  lev < 7 keeps only the slice pairs i + j < lev in both
// contractions (a cheaper, less accurate matvec for an inner solve)
gdml_status oz_matvec(OzMatvec& oz, const double* G, const float2* G2, const double* Xc, const double* v,
                      double* out, int add_lambda, double lam, cudaStream_t st, int lev = oz::S);
gdml_status oz_check(OzMatvec& oz, cudaStream_t st);
void oz_destroy(OzMatvec& oz);

// lower triangle of C = L^T L (k x k, FP64, row stride ldc) for the FP32 n x k factor L
// (column j at L + j n), through the sliced tensor-core GEMM with in-CTA accumulation
// over all 256-entry chunks of n.  Synchronises the stream.
gdml_status oz_syrk_lower(const float* L, int64_t n, int64_t k, double* C, int64_t ldc, cudaStream_t st);
// lower triangle of C = X X^T (rows x rows, FP64, row stride ldc) for FP64 X (rows x K, row
// stride ldx), through the same sliced GEMM.  Synchronises the stream.
gdml_status oz_syrk_lower_f64(const double* X, int64_t rows, int64_t K, int64_t ldx, double* C, int64_t ldc,
                              cudaStream_t st);

// C = A B^T for a tall A (n x K, column-major: entry (r, j) at A[j n + r]) and B (NB x K,
// row-major, row stride ldb; lower triangular when tri_b, so K entries past each row's
// diagonal are skipped) through the sliced tensor-core GEMM with in-CTA accumulation over
// all of K (FP64-class).  A is sliced in panels of rows.  rowsq = false: C stored
// column-major, out[c n + r] (and as FP32 at out32[c n + r] when out32 is not null); out may
// alias A.  rowsq = true: out[r] = sum_c C[r][c]^2 (n doubles).  Synchronises the stream.
gdml_status oz_gemm_tall(const double* A, int64_t n, int64_t K, const double* B, int64_t NB, int64_t ldb, bool tri_b,
                         bool rowsq, double* out, float* out32, cudaStream_t st);

// test hook: C (M x N, FP64) = A (M x K) B (N x K)^T through the sliced tensor-core GEMM with G
// K-chunks per CTA (G < 1: the automatic choice), keeping the slice pairs i + j < nlev
gdml_status oz_gemm_test(const double* A, const double* B, int64_t M, int64_t N, int64_t K, int G, int nlev,
                         double* C, cudaStream_t st);
// K chunks per CTA that keep about 8 waves of CTAs for `tiles` output tiles
int oz_auto_chunks_per_cta(int64_t tiles, int64_t nchunks);

}  // namespace gdml
