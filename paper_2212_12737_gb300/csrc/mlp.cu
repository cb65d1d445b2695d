// Learned inducing-column scorer: a BF16 MLP D -> H -> H -> 1 (exact-erf GELU)
// that maps a geometry's descriptor to a score, trained with MSE + Adam on the
// per-geometry ridge leverage scores this library computes (Sec. 3, "Leverage
// score sampling"; the scorer replaces their O(k^2 n) estimate at selection time).
//
// Storage: FP32 master parameters and Adam moments; BF16 copies of the weights, of the
// activations and of the back-propagated gradients feed the five contractions (two forward,
// three backward), which run on the tcgen05 tensor cores with FP32 accumulation
// (tc_gemm_bf16); none of them is on the PCG solve's loop.
#include <cuda_bf16.h>

#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "../../include/gdml.h"

namespace gdml {
namespace mlp {

using bf16 = __nv_bfloat16;

template <typename T>
__device__ __forceinline__ float ld(const T* p, int64_t i) {
  if constexpr (sizeof(T) == 2) return __bfloat162float(p[i]);
  else return (float)p[i];
}

// Operand layouts for the tcgen05 GEMMs (C = A B^T, BF16 operands with row strides that are
// multiples of 8 elements): the weights as BF16 copies W1b (H x Dp), W2b (H x Hp) and W2t = W2^T;
// per batch Xs (B x Dp), A1 (B x Hp), dZ2b (B x Hp) and the transposed XsT (D x Bt),
// A1T (H x Bt), dZ2T (H x Bt), dZ1T (H x Bt) for the weight gradients, whose K is the batch.
inline int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Xs = bf16((X - mu) / sd), row stride ldx, and (XsT) its transpose with row stride ldt
__global__ void standardize_kernel(const double* __restrict__ X, int64_t B, int D, const float* __restrict__ mu,
                                   const float* __restrict__ sd, bf16* __restrict__ Xs, int64_t ldx,
                                   bf16* __restrict__ XsT, int64_t ldt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B * D) return;
  const int64_t b = e / D;
  const int d = (int)(e - b * D);
  const bf16 v = __float2bfloat16(((float)X[e] - mu[d]) / sd[d]);
  Xs[b * ldx + d] = v;
  if (XsT) XsT[d * ldt + b] = v;
}

// A = bf16(gelu(Z)) (Z: B x H FP32, kept for the backward pass) with row stride lda, and (AT)
// its transpose with row stride ldt
__global__ void gelu_kernel(const float* __restrict__ Z, int64_t B, int H, bf16* __restrict__ A, int64_t lda,
                            bf16* __restrict__ AT, int64_t ldt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B * H) return;
  const int64_t b = e / H;
  const int h = (int)(e - b * H);
  const bf16 v = __float2bfloat16(gelu(Z[e]));
  A[b * lda + h] = v;
  if (AT) AT[h * ldt + b] = v;
}

// BF16 copies of the weights in the GEMMs' layouts: W1b (H x Dp), W2b (H x Hp), W2t = W2^T
__global__ void pack_weights_kernel(const float* __restrict__ W1, const float* __restrict__ W2, int D, int H,
                                    int64_t Dp, int64_t Hp, bf16* __restrict__ W1b, bf16* __restrict__ W2b,
                                    bf16* __restrict__ W2t) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n1 = (int64_t)H * D, n2 = (int64_t)H * H;
  if (e < n1) {
    const int64_t h = e / D, d = e - h * D;
    W1b[h * Dp + d] = __float2bfloat16(W1[e]);
  } else if (e < n1 + n2) {
    const int64_t f = e - n1, r = f / H, c = f - r * H;
    const bf16 v = __float2bfloat16(W2[f]);
    W2b[r * Hp + c] = v;
    W2t[c * Hp + r] = v;
  }
}

// out[b] = A2[b,:] . w3 + b3   (one warp per row)
__global__ void head_kernel(const bf16* __restrict__ A2, int64_t B, int H, const bf16* __restrict__ w3,
                            const float* __restrict__ b3, float* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  float s = 0.f;
  for (int h = lane; h < H; h += 32) s = fmaf(__bfloat162float(A2[b * H + h]), __bfloat162float(w3[h]), s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[b] = s + b3[0];
}

// dout = 2 (out - (y - ym)/ysd) / B; loss partial = sum (out - ys)^2 / B (last-block total)
__global__ void loss_kernel(const float* __restrict__ out, const double* __restrict__ y, int64_t B, float ym,
                            float ysd, float* __restrict__ dout, float* __restrict__ loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t b = threadIdx.x; b < B; b += 256) {
    const float r = out[b] - ((float)y[b] - ym) / ysd;
    dout[b] = 2.f * r / (float)B;
    s += r * r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)B;
}

// dZ2[b,h] = dout[b] * w3[h] * gelu'(Z2[b,h]) (FP32, for the bias gradient) and its BF16
// roundings for the GEMMs: dZ2b (row stride ldb) and the transpose dZ2T (row stride ldt)
__global__ void head_back_kernel(const float* __restrict__ dout, const bf16* __restrict__ w3,
                                 const float* __restrict__ Z2, int64_t B, int H, float* __restrict__ dZ2,
                                 bf16* __restrict__ dZ2b, int64_t ldb, bf16* __restrict__ dZ2T, int64_t ldt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B * H) return;
  const int64_t b = e / H;
  const int h = (int)(e - b * H);
  const float g = dout[b] * __bfloat162float(w3[h]) * gelu_grad(Z2[e]);
  dZ2[e] = g;
  const bf16 gb = __float2bfloat16(g);
  dZ2b[b * ldb + h] = gb;
  dZ2T[h * ldt + b] = gb;
}

// dZ1 = dA1 * gelu'(Z1) in place (FP32) and its BF16 transpose dZ1T (row stride ldt)
__global__ void gelu_back_kernel(float* __restrict__ dA, const float* __restrict__ Z, int64_t B, int H,
                                 bf16* __restrict__ dZT, int64_t ldt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B * H) return;
  const float g = dA[e] * gelu_grad(Z[e]);
  dA[e] = g;
  const int64_t b = e / H;
  dZT[(e - b * H) * ldt + b] = __float2bfloat16(g);
}

// g[j] = sum_b M[b, j] (column sums, fixed order per column)
__global__ void colsum_kernel(const float* __restrict__ Mx, int64_t B, int H, float* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= H) return;
  float s = 0.f;
  for (int64_t b = 0; b < B; ++b) s += Mx[b * H + j];
  g[j] = s;
}

// dw3[h] = sum_b A2[b,h] dout[b]
__global__ void head_wgrad_kernel(const bf16* __restrict__ A2, const float* __restrict__ dout, int64_t B, int H,
                                  float* __restrict__ dw3, float* __restrict__ db3) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < H) {
    float s = 0.f;
    for (int64_t b = 0; b < B; ++b) s = fmaf(__bfloat162float(A2[b * H + h]), dout[b], s);
    dw3[h] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int64_t b = 0; b < B; ++b) s += dout[b];
    *db3 = s;
  }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master parameters; refresh BF16 copies
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, bf16* __restrict__ pb, int64_t n, float lr, float bc1,
                            float bc2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float upd = lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
  p[i] -= upd;
  pb[i] = __float2bfloat16(p[i]);
}

__global__ void to_bf16_kernel(const float* __restrict__ p, bf16* __restrict__ pb, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16(p[i]);
}

// uniform init in [-a, a] from a 64-bit mix of (seed, index)
__global__ void init_kernel(float* __restrict__ p, int64_t n, float a, uint64_t seed) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((z >> 40) * (1.0 / 16777216.0));  // [0, 1)
  p[i] = a * (2.f * u - 1.f);
}

// column weight w_i = max(score_{geometry(i)}, 0) * diag_i
__global__ void column_weights_kernel(const double* __restrict__ score, const double* __restrict__ diag, int64_t n,
                                      int B3, double* __restrict__ w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = score[i / B3];
  w[i] = (s > 0.0 ? s : 0.0) * diag[i];
}

__global__ void destandardize_kernel(const float* __restrict__ out, int64_t B, float ym, float ysd,
                                     double* __restrict__ dst) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < B) dst[b] = (double)out[b] * (double)ysd + (double)ym;
}

}  // namespace mlp

void launch_destandardize(const float* out, int64_t B, float ym, float ysd, double* dst, cudaStream_t st) {
  { mlp::destandardize_kernel<<<(unsigned)cdiv(B, 256), 256, 0, st>>>(out, B, ym, ysd, dst); count_launch(); }
}

void launch_column_weights(const double* score, const double* diag, int64_t n, int B3, double* w, cudaStream_t st) {
  { mlp::column_weights_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(score, diag, n, B3, w); count_launch(); }
}

}  // namespace gdml

// ============================================================ scorer object
using namespace gdml;
using namespace gdml::mlp;

struct gdml_scorer {
  int D = 0, H = 0;
  cudaStream_t st = nullptr;
  int64_t nparam = 0;
  // flat FP32 parameters: [W1 (H x D) | b1 (H) | W2 (H x H) | b2 (H) | w3 (H) | b3 (1)]
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16* pb = nullptr;
  float *mu = nullptr, *sd = nullptr;  // feature standardisation (device, D)
  float ym = 0.f, ysd = 1.f;           // label standardisation
  int64_t Dp = 0, Hp = 0;              // row strides of the BF16 GEMM operands (multiples of 8)
  bf16 *W1b = nullptr, *W2b = nullptr, *W2t = nullptr;  // BF16 weights in the GEMMs' layouts
  int* err = nullptr;                  // device word set by a timed-out tensor-core pipeline wait
  int64_t cap = 0, Bt = 0;             // batch capacity of the buffers below; Bt = pad8(cap)
  bf16 *Xs = nullptr, *A1 = nullptr, *A2 = nullptr, *dZ2b = nullptr;
  bf16 *XsT = nullptr, *A1T = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *out = nullptr, *dout = nullptr, *dZ1 = nullptr, *dZ2 = nullptr,
        *loss = nullptr;
  int64_t step = 0;
  std::vector<void*> allocs;
  float* W1() { return p; }
  float* b1() { return p + (int64_t)H * D; }
  float* W2() { return b1() + H; }
  float* b2() { return W2() + (int64_t)H * H; }
  float* w3() { return b2() + H; }
  float* b3() { return w3() + H; }
  int64_t off_W2() const { return (int64_t)H * D + H; }
  int64_t off_w3() const { return off_W2() + (int64_t)H * H + H; }
};

namespace {

template <typename T>
gdml_status salloc(gdml_scorer* s, T** ptr, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GDML_ERR_OOM, "scorer: cudaMalloc failed");
  }
  s->allocs.push_back(q);
  *ptr = static_cast<T*>(q);
  return GDML_OK;
}

#define STRY(x)                     \
  do {                              \
    gdml_status _q = (x);           \
    if (_q != GDML_OK) return _q;   \
  } while (0)

gdml_status ensure_batch(gdml_scorer* s, int64_t B) {
  if (B <= s->cap) return GDML_OK;
  for (void** q : {(void**)&s->Xs, (void**)&s->A1, (void**)&s->A2, (void**)&s->Z1, (void**)&s->Z2, (void**)&s->out,
                   (void**)&s->dout, (void**)&s->dZ1, (void**)&s->dZ2, (void**)&s->dZ2b, (void**)&s->XsT,
                   (void**)&s->A1T, (void**)&s->dZ2T, (void**)&s->dZ1T}) {
    if (*q) {
      cudaFree(*q);
      for (auto& a : s->allocs)
        if (a == *q) a = nullptr;
      *q = nullptr;
    }
  }
  const int D = s->D, H = s->H;
  const int64_t Bt = pad8(B);
  STRY(salloc(s, &s->Xs, (size_t)(B * s->Dp)));
  STRY(salloc(s, &s->A1, (size_t)(B * s->Hp)));
  STRY(salloc(s, &s->dZ2b, (size_t)(B * s->Hp)));
  STRY(salloc(s, &s->XsT, (size_t)(D * Bt)));
  STRY(salloc(s, &s->A1T, (size_t)(H * Bt)));
  STRY(salloc(s, &s->dZ2T, (size_t)(H * Bt)));
  STRY(salloc(s, &s->dZ1T, (size_t)(H * Bt)));
  STRY(salloc(s, &s->A2, (size_t)(B * H)));
  STRY(salloc(s, &s->Z1, (size_t)(B * H)));
  STRY(salloc(s, &s->Z2, (size_t)(B * H)));
  STRY(salloc(s, &s->out, (size_t)B));
  STRY(salloc(s, &s->dout, (size_t)B));
  STRY(salloc(s, &s->dZ1, (size_t)(B * H)));
  STRY(salloc(s, &s->dZ2, (size_t)(B * H)));
  s->cap = B;
  s->Bt = Bt;
  return GDML_OK;
}

// BF16 copies of W1 and W2 in the GEMMs' layouts, after every change of the FP32 parameters
void pack_weights(gdml_scorer* s) {
  const int64_t n = (int64_t)s->H * s->D + (int64_t)s->H * s->H;
  { pack_weights_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s->st>>>(s->W1(), s->W2(), s->D, s->H, s->Dp, s->Hp, s->W1b, s->W2b, s->W2t); count_launch(); }
}

// read (and clear) the device error word after the stream has drained
gdml_status check_err(gdml_scorer* s) {
  int h = 0;
  if (cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "scorer: reading the error word");
  if (h) {
    cudaMemsetAsync(s->err, 0, sizeof(int), s->st);
    return fail(GDML_ERR_TIMEOUT, "scorer: a tensor-core pipeline wait timed out");
  }
  return GDML_OK;
}

// forward on rows X[0..B) (FP64, B x D) -> s->out (standardised prediction); with `keep_t` the
// transposed BF16 activations for the weight gradients are written too
gdml_status forward(gdml_scorer* s, const double* X, int64_t B, bool keep_t) {
  const int D = s->D, H = s->H;
  const int64_t Dp = s->Dp, Hp = s->Hp, Bt = s->Bt;
  cudaStream_t st = s->st;
  { standardize_kernel<<<(unsigned)cdiv(B * D, 256), 256, 0, st>>>(X, B, D, s->mu, s->sd, s->Xs, Dp, keep_t ? s->XsT : nullptr, Bt); count_launch(); }
  // Z1 = Xs W1^T + b1
  STRY(tc_gemm_bf16(s->Xs, Dp, s->W1b, Dp, (int)B, H, D, s->Z1, H, s->b1(), s->err, st));
  { gelu_kernel<<<(unsigned)cdiv(B * H, 256), 256, 0, st>>>(s->Z1, B, H, s->A1, Hp, keep_t ? s->A1T : nullptr, Bt); count_launch(); }
  // Z2 = A1 W2^T + b2
  STRY(tc_gemm_bf16(s->A1, Hp, s->W2b, Hp, (int)B, H, H, s->Z2, H, s->b2(), s->err, st));
  { gelu_kernel<<<(unsigned)cdiv(B * H, 256), 256, 0, st>>>(s->Z2, B, H, s->A2, H, nullptr, 0); count_launch(); }
  { head_kernel<<<(unsigned)cdiv(B, 8), 256, 0, st>>>(s->A2, B, H, s->pb + s->off_w3(), s->b3(), s->out); count_launch(); }
  return GDML_OK;
}

// loss and gradient (into s->g) on one batch
gdml_status backward(gdml_scorer* s, const double* X, const double* y, int64_t B) {
  const int D = s->D, H = s->H;
  const int64_t Hp = s->Hp, Bt = s->Bt;
  cudaStream_t st = s->st;
  STRY(forward(s, X, B, true));
  { loss_kernel<<<1, 256, 0, st>>>(s->out, y, B, s->ym, s->ysd, s->dout, s->loss); count_launch(); }
  float* g = s->g;
  float* gW1 = g;
  float* gb1 = g + (int64_t)H * D;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * H;
  float* gw3 = gb2 + H;
  float* gb3 = gw3 + H;
  { head_wgrad_kernel<<<(unsigned)cdiv(H, 256), 256, 0, st>>>(s->A2, s->dout, B, H, gw3, gb3); count_launch(); }
  { head_back_kernel<<<(unsigned)cdiv(B * H, 256), 256, 0, st>>>(s->dout, s->pb + s->off_w3(), s->Z2, B, H, s->dZ2, s->dZ2b, Hp, s->dZ2T, Bt); count_launch(); }
  // gW2[h][k] = sum_b dZ2[b][h] A1[b][k]
  STRY(tc_gemm_bf16(s->dZ2T, Bt, s->A1T, Bt, H, H, (int)B, gW2, H, nullptr, s->err, st));
  { colsum_kernel<<<(unsigned)cdiv(H, 256), 256, 0, st>>>(s->dZ2, B, H, gb2); count_launch(); }
  // dA1[b][k] = sum_h dZ2[b][h] W2[h][k]; dZ1 = dA1 * gelu'(Z1)
  STRY(tc_gemm_bf16(s->dZ2b, Hp, s->W2t, Hp, (int)B, H, H, s->dZ1, H, nullptr, s->err, st));
  { gelu_back_kernel<<<(unsigned)cdiv(B * H, 256), 256, 0, st>>>(s->dZ1, s->Z1, B, H, s->dZ1T, Bt); count_launch(); }
  // gW1[h][d] = sum_b dZ1[b][h] Xs[b][d]
  STRY(tc_gemm_bf16(s->dZ1T, Bt, s->XsT, Bt, H, D, (int)B, gW1, D, nullptr, s->err, st));
  { colsum_kernel<<<(unsigned)cdiv(H, 256), 256, 0, st>>>(s->dZ1, B, H, gb1); count_launch(); }
  return GDML_OK;
}

}  // namespace

extern "C" {

gdml_status gdml_scorer_create(gdml_scorer** out, int32_t D, int32_t hidden, uint64_t seed, void* stream) {
  clear_msg();
  if (!out || D < 1 || D > 65536 || hidden < 1 || hidden > 4096) return fail(GDML_ERR_ARG, "scorer: bad sizes");
  std::unique_ptr<gdml_scorer, void (*)(gdml_scorer*)> s(new gdml_scorer(), &gdml_scorer_destroy);
  s->D = D;
  s->H = hidden;
  s->st = static_cast<cudaStream_t>(stream);
  s->nparam = (int64_t)hidden * D + hidden + (int64_t)hidden * hidden + hidden + hidden + 1;
  gdml_scorer* S = s.get();
  STRY(salloc(S, &S->p, (size_t)S->nparam));
  STRY(salloc(S, &S->g, (size_t)S->nparam));
  STRY(salloc(S, &S->m, (size_t)S->nparam));
  STRY(salloc(S, &S->v, (size_t)S->nparam));
  STRY(salloc(S, &S->pb, (size_t)S->nparam));
  STRY(salloc(S, &S->mu, (size_t)D));
  STRY(salloc(S, &S->sd, (size_t)D));
  STRY(salloc(S, &S->loss, 1));
  S->Dp = pad8(D);
  S->Hp = pad8(hidden);
  STRY(salloc(S, &S->W1b, (size_t)(hidden * S->Dp)));
  STRY(salloc(S, &S->W2b, (size_t)(hidden * S->Hp)));
  STRY(salloc(S, &S->W2t, (size_t)(hidden * S->Hp)));
  STRY(salloc(S, &S->err, 1));
  cudaStream_t st = S->st;
  cudaMemsetAsync(S->err, 0, sizeof(int), st);
  auto init = [&](float* q, int64_t n, float a, uint64_t sd) {
    { init_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(q, n, a, sd); count_launch(); }
  };
  init(S->W1(), (int64_t)hidden * D, 1.f / std::sqrt((float)D), seed * 4 + 0);
  init(S->W2(), (int64_t)hidden * hidden, 1.f / std::sqrt((float)hidden), seed * 4 + 1);
  init(S->w3(), hidden, 1.f / std::sqrt((float)hidden), seed * 4 + 2);
  cudaMemsetAsync(S->b1(), 0, hidden * sizeof(float), st);
  cudaMemsetAsync(S->b2(), 0, hidden * sizeof(float), st);
  cudaMemsetAsync(S->b3(), 0, sizeof(float), st);
  cudaMemsetAsync(S->m, 0, S->nparam * sizeof(float), st);
  cudaMemsetAsync(S->v, 0, S->nparam * sizeof(float), st);
  { to_bf16_kernel<<<(unsigned)cdiv(S->nparam, 256), 256, 0, st>>>(S->p, S->pb, S->nparam); count_launch(); }
  pack_weights(S);
  std::vector<float> ones(D, 1.f);
  cudaMemsetAsync(S->mu, 0, D * sizeof(float), st);
  cudaMemcpyAsync(S->sd, ones.data(), D * sizeof(float), cudaMemcpyHostToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(GDML_ERR_CUDA, "scorer init");
  *out = s.release();
  return GDML_OK;
}

// Set the standardisation from the training data (host reduction of B x D is cheap).
gdml_status gdml_scorer_fit_scaling(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B) {
  if (!s || !X_dev || !y_dev || B < 2) return fail(GDML_ERR_ARG, "scorer: bad arguments");
  const int D = s->D;
  std::vector<double> X((size_t)(B * D)), y((size_t)B);
  if (cudaMemcpyAsync(X.data(), X_dev, X.size() * 8, cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaMemcpyAsync(y.data(), y_dev, y.size() * 8, cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "scorer: copy");
  std::vector<float> mu(D), sd(D);
  for (int d = 0; d < D; ++d) {
    double a = 0, b = 0;
    for (int64_t i = 0; i < B; ++i) a += X[i * D + d];
    a /= B;
    for (int64_t i = 0; i < B; ++i) b += (X[i * D + d] - a) * (X[i * D + d] - a);
    mu[d] = (float)a;
    sd[d] = (float)std::max(std::sqrt(b / B), 1e-12);
  }
  double a = 0, b = 0;
  for (double t : y) a += t;
  a /= B;
  for (double t : y) b += (t - a) * (t - a);
  s->ym = (float)a;
  s->ysd = (float)std::max(std::sqrt(b / B), 1e-30);
  cudaMemcpyAsync(s->mu, mu.data(), D * sizeof(float), cudaMemcpyHostToDevice, s->st);
  cudaMemcpyAsync(s->sd, sd.data(), D * sizeof(float), cudaMemcpyHostToDevice, s->st);
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return fail(GDML_ERR_CUDA, "scorer: scaling");
  return GDML_OK;
}

gdml_status gdml_scorer_train(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B, int32_t epochs,
                              int32_t batch, double lr, double* loss_out) {
  clear_msg();
  if (!s || !X_dev || !y_dev || B < 1 || epochs < 1 || batch < 1 || !(lr > 0)) return fail(GDML_ERR_ARG, "scorer: bad arguments");
  const int64_t bs = std::min<int64_t>(batch, B);
  STRY(ensure_batch(s, bs));
  float last = 0.f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t b0 = 0; b0 < B; b0 += bs) {
      const int64_t nb = std::min<int64_t>(bs, B - b0);
      STRY(backward(s, X_dev + b0 * s->D, y_dev + b0, nb));
      ++s->step;
      const float bc1 = 1.f - std::pow(0.9f, (float)s->step), bc2 = 1.f - std::pow(0.999f, (float)s->step);
      { adam_kernel<<<(unsigned)cdiv(s->nparam, 256), 256, 0, s->st>>>(s->p, s->g, s->m, s->v, s->pb, s->nparam, (float)lr, bc1, bc2); count_launch(); }
      pack_weights(s);
    }
  }
  STRY(check_err(s));
  if (cudaMemcpyAsync(&last, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return fail(GDML_ERR_CUDA, "scorer: train");
  if (loss_out) *loss_out = last;
  return GDML_OK;
}

gdml_status gdml_scorer_predict(gdml_scorer* s, const double* X_dev, int64_t B, double* out_dev) {
  clear_msg();
  if (!s || !X_dev || !out_dev || B < 1) return fail(GDML_ERR_ARG, "scorer: bad arguments");
  const int64_t bs = std::min<int64_t>(B, 4096);
  STRY(ensure_batch(s, bs));
  std::vector<float> h((size_t)bs);
  for (int64_t b0 = 0; b0 < B; b0 += bs) {
    const int64_t nb = std::min<int64_t>(bs, B - b0);
    STRY(forward(s, X_dev + b0 * s->D, nb, false));
    launch_destandardize(s->out, nb, s->ym, s->ysd, out_dev + b0, s->st);
  }
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return fail(GDML_ERR_CUDA, "scorer: predict");
  return check_err(s);
}

// Test hook: loss (host) and gradient (device, nparam floats) on one batch.
gdml_status gdml_scorer_grad(gdml_scorer* s, const double* X_dev, const double* y_dev, int64_t B, double* loss_out,
                             float* grad_dev) {
  clear_msg();
  if (!s || !X_dev || !y_dev || B < 1) return fail(GDML_ERR_ARG, "scorer: bad arguments");
  STRY(ensure_batch(s, B));
  STRY(backward(s, X_dev, y_dev, B));
  float l = 0.f;
  if (grad_dev) cudaMemcpyAsync(grad_dev, s->g, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(&l, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->st);
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return fail(GDML_ERR_CUDA, "scorer: grad");
  if (loss_out) *loss_out = l;
  return check_err(s);
}

// Get (set = 0) or set (set = 1) the flat FP32 parameters (device, nparam floats).
gdml_status gdml_scorer_params(gdml_scorer* s, float* params_dev, int32_t set, int64_t* nparam_out) {
  if (!s) return fail(GDML_ERR_ARG, "scorer: null");
  if (nparam_out) *nparam_out = s->nparam;
  if (!params_dev) return GDML_OK;
  if (set) {
    cudaMemcpyAsync(s->p, params_dev, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice, s->st);
    { to_bf16_kernel<<<(unsigned)cdiv(s->nparam, 256), 256, 0, s->st>>>(s->p, s->pb, s->nparam); count_launch(); }
    pack_weights(s);
  } else {
    cudaMemcpyAsync(params_dev, s->p, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice, s->st);
  }
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return fail(GDML_ERR_CUDA, "scorer: params");
  return GDML_OK;
}

void gdml_scorer_destroy(gdml_scorer* s) {
  if (!s) return;
  cudaStreamSynchronize(s->st);
  for (void* q : s->allocs)
    if (q) cudaFree(q);
  delete s;
}

}  // extern "C"
