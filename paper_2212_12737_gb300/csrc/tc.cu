// Tensor-core matvec for TF32 / BF16 contexts (see tc.cuh for the split into
// two tcgen05 GEMMs).  Data layout in HBM (all K-major, zero padded):
//   Xc_lp  M x Dp        centred descriptors          (A of GEMM 1, fixed)
//   W_lp   M x Dp        w = J v                      (B of GEMM 1, per matvec)
//   P_lp   M x K2p       [A | beta]                   (A of GEMM 2; A fixed, beta per matvec)
//   Vt_lp  Dp x K2p      [W^T | Xc^T]                 (B of GEMM 2; Xc^T fixed)
//   S32    M x M  fp32   S_ab = (c^2/3) e^{-c r_ab}
//   U      splits x M x Dp fp32 (split-K partials of GEMM 2, summed in order)
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tc.cuh"
#include "tc_gemm.cuh"

namespace gdml {

using namespace tc;

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <bool BF16>
struct Lp;
template <>
struct Lp<false> {
  using T = float;
  static __device__ __forceinline__ T from(double x) { return round_tf32((float)x); }
  static __device__ __forceinline__ double to(T x) { return (double)x; }
};
template <>
struct Lp<true> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ T from(double x) { return __double2bfloat16(x); }
  static __device__ __forceinline__ double to(T x) { return (double)__bfloat162float(x); }
};

// ------------------------------------------------------------ setup kernels
template <bool BF16>
__global__ void tc_setup_kernel(const double* __restrict__ Xc, const double* __restrict__ A, int64_t ldA,
                                const double* __restrict__ S, const double* __restrict__ G, int64_t M, int D, int Dp,
                                int64_t K2p, typename Lp<BF16>::T* __restrict__ Xc_lp,
                                typename Lp<BF16>::T* __restrict__ P_lp, typename Lp<BF16>::T* __restrict__ Vt_lp,
                                float* __restrict__ S32, float* __restrict__ G32) {
  using L = Lp<BF16>;
  const int64_t a = blockIdx.x;
  for (int p = threadIdx.x; p < D; p += blockDim.x) {
    const auto x = L::from(Xc[a * D + p]);
    Xc_lp[a * Dp + p] = x;
    Vt_lp[(int64_t)p * K2p + M + a] = x;
  }
  for (int e = threadIdx.x; e < 3 * D; e += blockDim.x) G32[a * 3 * D + e] = (float)G[a * 3 * D + e];
  for (int64_t b = threadIdx.x; b < M; b += blockDim.x) {
    P_lp[a * K2p + b] = L::from(A[a * ldA + b]);
    S32[a * M + b] = (float)S[a * M + b];
  }
}

// w_a = J_a v_a (FP32) rounded to the operand type; t_a = xc~_a . w~_a (FP32).
// Row-major W only; the transposed copy for GEMM 2 is written by tc_transpose_kernel.
template <bool BF16, int THREADS>
__global__ void tc_proj_kernel(const float* __restrict__ G, const double* __restrict__ v, int N, int D, int Dp,
                               const typename Lp<BF16>::T* __restrict__ Xc_lp, typename Lp<BF16>::T* __restrict__ W_lp,
                               float* __restrict__ t) {
  using L = Lp<BF16>;
  extern __shared__ float sh_vf[];
  __shared__ float red[THREADS / 32];
  const int64_t a = blockIdx.x;
  const int B = 3 * N;
  for (int l = threadIdx.x; l < B; l += THREADS) sh_vf[l] = (float)v[a * B + l];
  __syncthreads();
  const float* Ga = G + a * D * 3;
  float part = 0.f;
  for (int p = threadIdx.x; p < D; p += THREADS) {
    int i = (int)((1.f + sqrtf(1.f + 8.f * (float)p)) * 0.5f);
    while (i * (i - 1) / 2 > p) --i;
    while ((i + 1) * i / 2 <= p) ++i;
    const int j = p - i * (i - 1) / 2;
    const float w = -(Ga[3 * p] * (sh_vf[3 * i] - sh_vf[3 * j]) + Ga[3 * p + 1] * (sh_vf[3 * i + 1] - sh_vf[3 * j + 1]) +
                      Ga[3 * p + 2] * (sh_vf[3 * i + 2] - sh_vf[3 * j + 2]));
    const auto wl = L::from((double)w);
    W_lp[a * Dp + p] = wl;
    part = fmaf((float)L::to(Xc_lp[a * Dp + p]), (float)L::to(wl), part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < THREADS / 32; ++q) s += red[q];
    t[a] = s;
  }
}

// Vt[p][a] = W[a][p] for a < M, p < D (32 x 32 tiles through shared memory)
template <typename T>
__global__ void tc_transpose_kernel(const T* __restrict__ W, int64_t M, int D, int Dp, int64_t K2p,
                                    T* __restrict__ Vt) {
  __shared__ T tile[32][33];
  const int64_t a0 = (int64_t)blockIdx.y * 32;
  const int p0 = blockIdx.x * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t a = a0 + yy;
    const int p = p0 + threadIdx.x;
    if (a < M && p < D) tile[yy][threadIdx.x] = W[a * Dp + p];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int p = p0 + yy;
    const int64_t a = a0 + threadIdx.x;
    if (a < M && p < D) Vt[(int64_t)p * K2p + a] = tile[threadIdx.x][yy];
  }
}

// GEMM 1 epilogue: beta_ab = c^2 S_ab (T_ab - t_b) -> P[:, M + b]; per-32-column row sums
template <bool BF16>
struct EpiBeta {
  const float* S32;
  const float* t;
  typename Lp<BF16>::T* P;
  int64_t K2p;
  int M;
  float c2;
  double* rs_part;
  __device__ __forceinline__ void operator()(int row, int col0, float (&v)[32], int valid, int) const {
    float s = 0.f;
    const float* Srow = S32 + (int64_t)row * M;
    auto* Prow = P + (int64_t)row * K2p + M;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j < valid) {
        const int b = col0 + j;
        const float beta = c2 * Srow[b] * (v[j] - t[b]);
        const auto bl = Lp<BF16>::from((double)beta);
        Prow[b] = bl;
        s += (float)Lp<BF16>::to(bl);
      }
    }
    rs_part[(int64_t)(col0 >> 5) * M + row] = (double)s;
  }
};

// GEMM 2 epilogue: U partial (fp32)
struct EpiStore {
  float* U;
  int64_t ld;
  int64_t split_stride;
  __device__ __forceinline__ void operator()(int row, int col0, float (&v)[32], int valid, int split) const {
    float* dst = U + split * split_stride + (int64_t)row * ld + col0;
    if (valid == 32) {  // ld and col0 are multiples of 32 floats: 16-byte aligned
#pragma unroll
      for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < valid) dst[j] = v[j];
    }
  }
};

// test epilogue: FP64 output
struct EpiStoreD {
  double* C;
  int64_t ld;
  __device__ __forceinline__ void operator()(int row, int col0, float (&v)[32], int valid, int) const {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < valid) C[(int64_t)row * ld + col0 + j] = (double)v[j];
  }
};

// (K v)_a = J_a^T (sum_s U_s[a] - rowsum_a xc~_a) (+ lambda v_a); FP32 arithmetic, FP64 output
template <bool BF16>
__global__ void tc_backproj_kernel(const float* __restrict__ U, int splits, int64_t split_stride, int Dp,
                                   const double* __restrict__ rs_part, int nslots, int64_t M,
                                   const typename Lp<BF16>::T* __restrict__ Xc_lp, const float* __restrict__ G,
                                   const double* __restrict__ v, int N, int D, double lam, int add_lambda,
                                   double* __restrict__ out) {
  extern __shared__ float sh_uf[];
  __shared__ float rs;
  const int64_t a = blockIdx.x;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nslots; k += 32) s += rs_part[(int64_t)k * M + a];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) rs = (float)s;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < D; p += blockDim.x) {
    float u = 0.f;
    for (int s = 0; s < splits; ++s) u += U[s * split_stride + a * Dp + p];
    sh_uf[p] = u - rs * (float)Lp<BF16>::to(Xc_lp[a * Dp + p]);
  }
  __syncthreads();
  const int B = 3 * N;
  const float* Ga = G + a * D * 3;
  for (int l = threadIdx.x; l < B; l += blockDim.x) {
    const int i = l / 3, q = l - 3 * i;
    float s = 0.f;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {  // branch-free: independent loads of successive j
      const bool skip = j == i;
      const int p = skip ? 0 : (i > j ? i * (i - 1) / 2 + j : j * (j - 1) / 2 + i);
      const float gj = Ga[3 * p + q] * sh_uf[p];
      s += skip ? 0.f : ((i > j) ? -gj : gj);
    }
    double o = (double)s;
    if (add_lambda) o = fma(lam, v[a * B + l], o);
    out[a * B + l] = o;
  }
}

template <bool BF16>
__global__ void to_lp_padded_kernel(const double* __restrict__ src, int rows, int cols, int ldp,
                                    typename Lp<BF16>::T* __restrict__ dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * ldp) return;
  int r = (int)(e / ldp), c = (int)(e % ldp);
  dst[e] = Lp<BF16>::from(c < cols ? src[(int64_t)r * cols + c] : 0.0);
}

// ------------------------------------------------------------ host helpers
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D K-major map: inner dim K (elements), outer dim rows; box = one 128-byte span x box_rows
bool make_kmajor_map(CUtensorMap* m, const void* base, bool bf16, uint64_t K, uint64_t rows, uint64_t ld_elems,
                     uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const uint32_t esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {ld_elems * esz};
  cuuint32_t box[2] = {128u / esz, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2D FP32 map without swizzle: inner dim contiguous, outer stride ld_elems (a multiple
// of 4 elements); box = box_inner x box_outer; zero fill outside the tensor
bool make_f32_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                  uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld_elems * 4};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool BF16, int BN, int STAGES, typename Epi>
static gdml_status launch_gemm(const CUtensorMap& mA, const CUtensorMap& mB, int M, int N, int num_kb, int splits,
                               const Epi& epi, int* err, cudaStream_t st) {
  using SM = Smem<BN, STAGES>;
  auto kern = gemm_kernel<BF16, BN, STAGES, Epi>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::TOTAL) != cudaSuccess)
      return fail(GDML_ERR_CUDA, "cudaFuncSetAttribute(tcgen05 gemm)");
    attr_set = true;
  }
  const int kb_per_split = (int)cdiv(num_kb, splits);
  splits = (int)cdiv(num_kb, kb_per_split);
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)cdiv(M, BM), (unsigned)splits);
  { kern<<<grid, NUM_THREADS, SM::TOTAL, st>>>(mA, mB, M, N, num_kb, kb_per_split, epi, err); count_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("tcgen05 gemm launch: ") + cudaGetErrorString(e));
  return GDML_OK;
}

template <bool BF16, typename Epi>
static gdml_status gemm_dispatch_bn(int bn, const CUtensorMap& mA, const CUtensorMap& mB, int M, int N, int num_kb,
                                    int splits, const Epi& epi, int* err, cudaStream_t st) {
  switch (bn) {
    case 64:
      return launch_gemm<BF16, 64, 6>(mA, mB, M, N, num_kb, splits, epi, err, st);
    case 128:
      return launch_gemm<BF16, 128, 5>(mA, mB, M, N, num_kb, splits, epi, err, st);
    default:
      return launch_gemm<BF16, 256, 4>(mA, mB, M, N, num_kb, splits, epi, err, st);
  }
}

template <typename T>
static gdml_status tc_alloc(TcMatvec& tc, T** p, size_t count) {
  void* v = nullptr;
  if (cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GDML_ERR_OOM, "tensor-core buffers: cudaMalloc failed");
  }
  tc.allocs.push_back(v);
  *p = static_cast<T*>(v);
  return GDML_OK;
}

#define TC_TRY(x)                    \
  do {                               \
    gdml_status _s = (x);            \
    if (_s != GDML_OK) return _s;    \
  } while (0)

template <bool BF16>
static gdml_status setup_impl(TcMatvec& tc, const double* Xc, const double* A, int64_t ldA, const double* S,
                              const double* G, cudaStream_t st) {
  using T = typename Lp<BF16>::T;
  const int64_t M = tc.M;
  const int span = BF16 ? 64 : 32;  // elements per 128-byte swizzle span
  tc.Dp = (int)(cdiv(tc.D, span) * span);
  tc.K2p = cdiv(2 * M, span) * span;
  T *xc, *w, *p, *vt;
  TC_TRY(tc_alloc(tc, &xc, (size_t)(M * tc.Dp)));
  TC_TRY(tc_alloc(tc, &w, (size_t)(M * tc.Dp)));
  TC_TRY(tc_alloc(tc, &p, (size_t)(M * tc.K2p)));
  TC_TRY(tc_alloc(tc, &vt, (size_t)(tc.Dp * tc.K2p)));
  TC_TRY(tc_alloc(tc, &tc.S32, (size_t)(M * M)));
  TC_TRY(tc_alloc(tc, &tc.rs_part, (size_t)(cdiv(M, 32) * M)));
  TC_TRY(tc_alloc(tc, &tc.err, 1));
  TC_TRY(tc_alloc(tc, &tc.tb, (size_t)M));
  TC_TRY(tc_alloc(tc, &tc.G32, (size_t)(M * tc.D * 3)));
  tc.Xc_lp = xc;
  tc.W_lp = w;
  tc.P_lp = p;
  tc.Vt_lp = vt;
  // GEMM 2 tiling: N tile covers Dp (<= 256), split K to fill the 152 SMs
  tc.bn2 = tc.Dp <= 64 ? 64 : (tc.Dp <= 128 ? 128 : 256);
  const int64_t tiles = cdiv(tc.Dp, tc.bn2) * cdiv(M, BM);
  const int64_t num_kb2 = tc.K2p / span;
  // split K until the grid covers ~3 waves of the SMs (the autotuner can refine it)
  tc.splits2 = (int)std::max<int64_t>(1, std::min<int64_t>(num_kb2 / 8, cdiv(3 * (int64_t)num_sms(), std::max<int64_t>(tiles, 1))));
  tc.splits_cap = std::max(tc.splits2, 8);
  TC_TRY(tc_alloc(tc, &tc.U, (size_t)(tc.splits_cap * M * tc.Dp)));
  if (cudaMemsetAsync(xc, 0, M * tc.Dp * sizeof(T), st) != cudaSuccess ||
      cudaMemsetAsync(w, 0, M * tc.Dp * sizeof(T), st) != cudaSuccess ||
      cudaMemsetAsync(p, 0, M * tc.K2p * sizeof(T), st) != cudaSuccess ||
      cudaMemsetAsync(vt, 0, tc.Dp * tc.K2p * sizeof(T), st) != cudaSuccess ||
      cudaMemsetAsync(tc.err, 0, sizeof(int), st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "tensor-core buffer memset");
  { tc_setup_kernel<BF16><<<(unsigned)M, 256, 0, st>>>(Xc, A, ldA, S, G, M, tc.D, tc.Dp, tc.K2p, xc, p, vt, tc.S32, tc.G32); count_launch(); }
  if (cudaGetLastError() != cudaSuccess) return fail(GDML_ERR_CUDA, "tensor-core setup kernel");
  bool ok = make_kmajor_map(&tc.mapXc, xc, BF16, tc.Dp, M, tc.Dp, BM) && make_kmajor_map(&tc.mapW, w, BF16, tc.Dp, M, tc.Dp, 128) &&
            make_kmajor_map(&tc.mapP, p, BF16, tc.K2p, M, tc.K2p, BM) &&
            make_kmajor_map(&tc.mapVt, vt, BF16, tc.K2p, tc.Dp, tc.K2p, tc.bn2);
  if (!ok) return fail(GDML_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  tc.ready = true;
  return GDML_OK;
}

gdml_status tc_setup(TcMatvec& tc, int precision, int64_t M, int N, int D, const double* Xc, const double* A,
                     int64_t ldA, const double* S, const double* G, double c, cudaStream_t st) {
  if (M > (int64_t)1 << 30) return fail(GDML_ERR_ARG, "M too large for the tensor-core path");
  tc.precision = precision;
  tc.M = M;
  tc.N = N;
  tc.D = D;
  tc.c = c;
  return precision == GDML_BF16 ? setup_impl<true>(tc, Xc, A, ldA, S, G, st)
                                : setup_impl<false>(tc, Xc, A, ldA, S, G, st);
}

template <bool BF16>
static gdml_status matvec_impl(TcMatvec& tc, const double* G, const double* v, double* out, int add_lambda,
                               double lam, cudaStream_t st) {
  using T = typename Lp<BF16>::T;
  (void)G;
  const int64_t M = tc.M;
  const int span = BF16 ? 64 : 32;
  { tc_proj_kernel<BF16, 256><<<(unsigned)M, 256, 3 * tc.N * sizeof(float), st>>>(tc.G32, v, tc.N, tc.D, tc.Dp, (const T*)tc.Xc_lp, (T*)tc.W_lp, tc.tb); count_launch(); }
  {
    dim3 g((unsigned)cdiv(tc.D, 32), (unsigned)cdiv(M, 32));
    { tc_transpose_kernel<T><<<g, dim3(32, 8), 0, st>>>((const T*)tc.W_lp, M, tc.D, tc.Dp, tc.K2p, (T*)tc.Vt_lp); count_launch(); }
  }
  EpiBeta<BF16> e1{tc.S32, tc.tb, (T*)tc.P_lp, tc.K2p, (int)M, (float)(tc.c * tc.c), tc.rs_part};
  // short K: 3 stages (97 KB) so that two CTAs share an SM and epilogues overlap mainloops
  TC_TRY((launch_gemm<BF16, 128, 3>(tc.mapXc, tc.mapW, (int)M, (int)M, tc.Dp / span, 1, e1, tc.err, st)));
  EpiStore e2{tc.U, tc.Dp, M * tc.Dp};
  TC_TRY((gemm_dispatch_bn<BF16>(tc.bn2, tc.mapP, tc.mapVt, (int)M, tc.D, (int)(tc.K2p / span), tc.splits2, e2,
                                 tc.err, st)));
  const int kb_per_split = (int)cdiv(tc.K2p / span, tc.splits2);
  const int splits = (int)cdiv(tc.K2p / span, kb_per_split);
  const size_t smem = tc.D * sizeof(float);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(tc_backproj_kernel<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { tc_backproj_kernel<BF16><<<(unsigned)M, 128, smem, st>>>(tc.U, splits, M * tc.Dp, tc.Dp, tc.rs_part, (int)cdiv(M, 32), M, (const T*)tc.Xc_lp, tc.G32, v, tc.N, tc.D, lam, add_lambda, out); count_launch(); }
  if (cudaGetLastError() != cudaSuccess) return fail(GDML_ERR_CUDA, "tensor-core matvec kernels");
  return GDML_OK;
}

gdml_status tc_matvec(TcMatvec& tc, const double* G, const double* v, double* out, int add_lambda, double lam,
                      cudaStream_t st) {
  if (!tc.ready) return fail(GDML_ERR_STATE, "tensor-core matvec not set up");
  return tc.precision == GDML_BF16 ? matvec_impl<true>(tc, G, v, out, add_lambda, lam, st)
                                   : matvec_impl<false>(tc, G, v, out, add_lambda, lam, st);
}

gdml_status tc_check(TcMatvec& tc, cudaStream_t st) {
  if (!tc.ready) return GDML_OK;
  int h = 0;
  if (cudaMemcpyAsync(&h, tc.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "reading the tensor-core error word");
  if (h) {
    cudaMemsetAsync(tc.err, 0, sizeof(int), st);
    return fail(GDML_ERR_TIMEOUT, "a tcgen05 pipeline wait timed out (code " + std::to_string(h) + ")");
  }
  return GDML_OK;
}

void tc_destroy(TcMatvec& tc) {
  for (void* p : tc.allocs) cudaFree(p);
  tc.allocs.clear();
  tc.ready = false;
}

template <bool BF16>
static gdml_status gemm_test_impl(const double* A, const double* B, int M, int N, int K, double* C, cudaStream_t st) {
  using T = typename Lp<BF16>::T;
  const int span = BF16 ? 64 : 32;
  const int Kp = (int)(cdiv(K, span) * span);
  T *a = nullptr, *b = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&a, (size_t)M * Kp * sizeof(T)) != cudaSuccess || cudaMalloc(&b, (size_t)N * Kp * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaFree(a);
    cudaFree(b);
    return fail(GDML_ERR_OOM, "gemm test buffers");
  }
  cudaMemsetAsync(err, 0, sizeof(int), st);
  { to_lp_padded_kernel<BF16><<<(unsigned)cdiv((int64_t)M * Kp, 256), 256, 0, st>>>(A, M, K, Kp, a); count_launch(); }
  { to_lp_padded_kernel<BF16><<<(unsigned)cdiv((int64_t)N * Kp, 256), 256, 0, st>>>(B, N, K, Kp, b); count_launch(); }
  CUtensorMap mA, mB;
  const int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  gdml_status s = GDML_OK;
  if (!make_kmajor_map(&mA, a, BF16, Kp, M, Kp, BM) || !make_kmajor_map(&mB, b, BF16, Kp, N, Kp, bn)) {
    s = fail(GDML_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  } else {
    EpiStoreD e{C, N};
    s = gemm_dispatch_bn<BF16>(bn, mA, mB, M, N, Kp / span, 1, e, err, st);
  }
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFree(a);
  cudaFree(b);
  cudaFree(err);
  if (s == GDML_OK && h) s = fail(GDML_ERR_TIMEOUT, "tcgen05 gemm wait timed out");
  return s;
}

// C[row][col] = bias[col] + sum_k A[row][k] B[col][k], FP32, for any M, N, K (rows beyond M and
// columns beyond N are masked; K beyond the operands reads the TMA fill value, zero)
struct EpiStoreBias {
  float* C;
  int64_t ld;
  const float* bias;
  __device__ __forceinline__ void operator()(int row, int col0, float (&v)[32], int valid, int) const {
    float* dst = C + (int64_t)row * ld + col0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < valid) dst[j] = v[j] + (bias ? bias[col0 + j] : 0.f);
  }
};

gdml_status tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, float* C,
                         int64_t ldc, const float* bias, int* err, cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || lda % 8 || ldb % 8 || lda < K || ldb < K ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return fail(GDML_ERR_ARG, "tc_gemm_bf16: operands need 16-byte aligned bases and strides >= K, multiples of 8");
  CUtensorMap mA, mB;
  const int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  if (!make_kmajor_map(&mA, A, true, (uint64_t)K, (uint64_t)M, (uint64_t)lda, BM) ||
      !make_kmajor_map(&mB, B, true, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, (uint32_t)bn))
    return fail(GDML_ERR_CUDA, "tc_gemm_bf16: cuTensorMapEncodeTiled failed");
  EpiStoreBias e{C, ldc, bias};
  return gemm_dispatch_bn<true>(bn, mA, mB, M, N, (int)cdiv(K, 64), 1, e, err, st);
}

gdml_status tc_gemm_test(int bf16, const double* A, const double* B, int M, int N, int K, double* C,
                         cudaStream_t st) {
  return bf16 ? gemm_test_impl<true>(A, B, M, N, K, C, st) : gemm_test_impl<false>(A, B, M, N, K, C, st);
}

cudaError_t set_wait_limit_tc(uint32_t polls) { return tc::set_wait_limit_here(polls); }

}  // namespace gdml
