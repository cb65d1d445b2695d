// Tensor-core (tcgen05) form of the force-kernel matvec for TF32 / BF16 contexts.
//
// The two descriptor contractions of K v run as tcgen05 GEMMs with FP32
// accumulation (operands rounded to TF32 or BF16):
//   GEMM 1:  T = Xc W^T                      (M x M, K = D)   epilogue: beta_ab = c^2 S_ab (T_ab - t_b)
//   GEMM 2:  U = [A | beta] [W ; Xc]         (M x D, K = 2M)
// with Xc the centred descriptors, W = J v, t_b = xc_b . w_b, A_ab = S_ab (1 + c r_ab);
// projection, the beta epilogue and back-projection (J_a^T (U_a - rowsum_a xc_a))
// run in FP32: the contractions' operands carry 8-11 bits, so FP64 there would
// only add GB300's slow FP64 pipe to the critical path.
#pragma once
#include <cuda.h>

#include <vector>

#include "common.cuh"

namespace gdml {

struct TcMatvec {
  int precision = 0;  // GDML_TF32 or GDML_BF16
  bool ready = false;
  int64_t M = 0;
  int N = 0, D = 0, Dp = 0;  // Dp: D padded to one 128-byte swizzle span
  int64_t K2p = 0;           // 2M padded likewise
  double c = 0;
  void* Xc_lp = nullptr;  // M x Dp
  void* W_lp = nullptr;   // M x Dp
  void* P_lp = nullptr;   // M x K2p : [A | beta]
  void* Vt_lp = nullptr;  // Dp x K2p : [W^T | Xc^T]
  float* S32 = nullptr;   // M x M
  float* U = nullptr;     // splits x M x Dp
  double* rs_part = nullptr;  // rowsum partials: ceil(M/32) x M
  float* tb = nullptr;        // t_b = xc~_b . w~_b
  float* G32 = nullptr;       // M x D x 3 FP32 copy of the Jacobian factors
  int* err = nullptr;
  int bn2 = 256, splits2 = 1, splits_cap = 1;
  std::vector<void*> allocs;
  CUtensorMap mapXc, mapW, mapP, mapVt;
};

gdml_status tc_setup(TcMatvec& tc, int precision, int64_t M, int N, int D, const double* Xc, const double* A,
                     int64_t ldA, const double* S, const double* G, double c, cudaStream_t st);
gdml_status tc_matvec(TcMatvec& tc, const double* G, const double* v, double* out, int add_lambda, double lam,
                      cudaStream_t st);
// reads (and clears) the device error word of the tensor-core kernels; synchronises st
gdml_status tc_check(TcMatvec& tc, cudaStream_t st);
void tc_destroy(TcMatvec& tc);

// 2D K-major TMA map with 128-byte swizzle: inner dim K (elements), outer dim rows, row stride
// ld_elems; box = one 128-byte span of K x box_rows rows.  False if the CUDA driver rejects it.
bool make_kmajor_map(CUtensorMap* m, const void* base, bool bf16, uint64_t K, uint64_t rows, uint64_t ld_elems,
                     uint32_t box_rows);

// 2D FP32 TMA map without swizzle: inner dim (contiguous elements), outer dim, outer stride
// ld_elems (ld_elems * 4 a multiple of 16 bytes); box = box_inner x box_outer elements,
// zero fill outside the tensor.  False if the CUDA driver rejects it.
bool make_f32_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                  uint32_t box_inner, uint32_t box_outer);

// C (M x N, FP32, row stride ldc) = A B^T (+ bias per column) on the tcgen05 tensor cores (BF16
// operands, FP32 accumulation): A M x K, B N x K, row-major BF16 with row strides lda, ldb that
// are multiples of 8 elements and 16-byte aligned bases; any M, N, K.  err: a device int that a
// bounded pipeline wait sets (checked by the caller).
gdml_status tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, float* C,
                         int64_t ldc, const float* bias, int* err, cudaStream_t st);
// test hook: C (M x N, fp64) = A (M x K) B (N x K)^T with operands rounded to TF32 / BF16
gdml_status tc_gemm_test(int bf16, const double* A, const double* B, int M, int N, int K, double* C,
                         cudaStream_t st);

}  // namespace gdml
