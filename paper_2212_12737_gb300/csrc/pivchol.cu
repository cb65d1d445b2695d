// Incomplete Cholesky with greedy diagonal pivoting (App. A.2, Algorithm 1),
// matrix-free: only diag(K) and one kernel column per step are needed.
//
// Per step m (all state stays on the device; no host round trip):
//   1. pivot = argmax of the residual diagonal over not-yet-chosen positions
//      (ties -> lowest position, positions kept in a permutation array that is
//      updated by the same swap as the paper's pi); the same pass sums the
//      residual diagonal, which is the trace after step m-1;
//   2. column k_m = K[:, pivot] (kcol kernel);
//   3. for every unchosen row i:  s_i = sum_{j<m} l_{pivot,j} l_{i,j}  (in order j = 0..m-1),
//      l_{i,m} = (k_{m,i} - s_i) / l_{pivot,m},  d_i -= l_{i,m}^2;  l_{pivot,m} = sqrt(d_pivot).
// If the largest residual diagonal is not positive the factorisation stops
// (rank = m) and every later kernel of the loop returns immediately.
#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

constexpr int kArgBlocks = 2 * kNumSMs;
constexpr int kArgThreads = 256;

struct ArgMax {
  double v;
  int64_t pos;
};
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  // larger value wins; ties (or both non-comparable) -> lower position
  if (b.v > a.v) return b;
  if (a.v > b.v) return a;
  if (a.v == b.v) return (b.pos < a.pos) ? b : a;
  return (a.v == a.v) ? a : b;  // NaN loses
}

__global__ void __launch_bounds__(kArgThreads) pc_argmax_kernel(
    int64_t m, int64_t n, int do_select, const double* __restrict__ d, int64_t* __restrict__ perm,
    unsigned char* __restrict__ chosen, int64_t* __restrict__ pivots, double* __restrict__ trace,
    PivState* __restrict__ ps, ArgMaxPart* __restrict__ part, unsigned* __restrict__ ticket) {
  if (ps->stop) return;
  __shared__ double sv[kArgThreads];
  __shared__ int64_t sp[kArgThreads];
  __shared__ double ss[kArgThreads];
  __shared__ bool last;
  const int64_t len = n - m;
  const int64_t chunk = cdiv_dev(len, gridDim.x);
  const int64_t beg = m + blockIdx.x * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  ArgMax best{-1.0 / 0.0, INT64_MAX};
  double sum = 0.0;
  for (int64_t pos = beg + threadIdx.x; pos < end; pos += kArgThreads) {
    const double v = d[perm[pos]];
    sum += v;
    best = better(best, ArgMax{v, pos});
  }
  sv[threadIdx.x] = best.v;
  sp[threadIdx.x] = best.pos;
  ss[threadIdx.x] = sum;
  __syncthreads();
  for (int o = kArgThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ArgMax r = better(ArgMax{sv[threadIdx.x], sp[threadIdx.x]}, ArgMax{sv[threadIdx.x + o], sp[threadIdx.x + o]});
      sv[threadIdx.x] = r.v;
      sp[threadIdx.x] = r.pos;
      ss[threadIdx.x] += ss[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x].v = sv[0];
    part[blockIdx.x].pos = sp[0];
    part[blockIdx.x].sum = ss[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA combines the per-CTA results with all its threads (fixed order)
  {
    ArgMax bt{-1.0 / 0.0, INT64_MAX};
    double st = 0.0;
    volatile ArgMaxPart* vp = part;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += kArgThreads) {
      bt = better(bt, ArgMax{vp[i].v, vp[i].pos});
      st += vp[i].sum;
    }
    sv[threadIdx.x] = bt.v;
    sp[threadIdx.x] = bt.pos;
    ss[threadIdx.x] = st;
  }
  __syncthreads();
  for (int o = kArgThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ArgMax r = better(ArgMax{sv[threadIdx.x], sp[threadIdx.x]}, ArgMax{sv[threadIdx.x + o], sp[threadIdx.x + o]});
      sv[threadIdx.x] = r.v;
      sp[threadIdx.x] = r.pos;
      ss[threadIdx.x] += ss[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const ArgMax b{sv[0], sp[0]};
  const double tot = ss[0];
  *ticket = 0u;
  if (m > 0 && trace) trace[m - 1] = tot;
  if (!do_select) return;
  if (!(b.v > 0.0) || b.pos >= n) {
    ps->stop = 1;
    ps->rank = m;
    return;
  }
  const int64_t piv = perm[b.pos];
  perm[b.pos] = perm[m];
  perm[m] = piv;
  pivots[m] = piv;
  chosen[piv] = 1;
  ps->lmm = sqrt(d[piv]);
  ps->piv = piv;
  ps->rank = m + 1;
}

template <typename TL>
__global__ void __launch_bounds__(256) pc_update_kernel(int64_t m, int64_t n, TL* __restrict__ L,
                                                        const double* __restrict__ col, double* __restrict__ d,
                                                        const unsigned char* __restrict__ chosen,
                                                        const PivState* __restrict__ ps) {
  if (ps->stop) return;
  __shared__ double lp[2048];
  const int64_t piv = ps->piv;
  const double lmm = ps->lmm;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = i < n && !chosen[i];
  double s = 0.0;
  for (int64_t j0 = 0; j0 < m; j0 += 2048) {
    const int64_t jn = (m - j0) < 2048 ? (m - j0) : 2048;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < jn; t += blockDim.x) lp[t] = (double)L[piv + (j0 + t) * n];
    __syncthreads();
    if (active) {
      const TL* Li = L + i + j0 * n;
      for (int64_t j = 0; j < jn; ++j) s = fma(lp[j], (double)Li[j * n], s);
    }
  }
  if (i >= n) return;
  if (active) {
    const double l = (col[i] - s) / lmm;
    const TL lst = (TL)l;
    L[i + m * n] = lst;
    const double lr = (double)lst;  // the stored value defines the factor
    d[i] = __dsub_rn(d[i], __dmul_rn(lr, lr));
  } else if (i == piv) {
    L[i + m * n] = (TL)lmm;
  }
}

// Alg. 1 step with FP32-stored L (DF64 contexts): the Schur correction is a
// double-float sum of exact FP32 products, the new column is formed in FP64
// and stored in FP32, and the residual diagonal is updated with the stored value.
__global__ void __launch_bounds__(256) pc_update_df_kernel(int64_t m, int64_t n, float* __restrict__ L,
                                                           const double* __restrict__ col, double* __restrict__ d,
                                                           const unsigned char* __restrict__ chosen,
                                                           const PivState* __restrict__ ps) {
  if (ps->stop) return;
  __shared__ float lp[4096];
  const int64_t piv = ps->piv;
  const double lmm = ps->lmm;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = i < n && !chosen[i];
  float sh = 0.f, sl = 0.f;
  for (int64_t j0 = 0; j0 < m; j0 += 4096) {
    const int64_t jn = (m - j0) < 4096 ? (m - j0) : 4096;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < jn; t += blockDim.x) lp[t] = L[piv + (j0 + t) * n];
    __syncthreads();
    if (active) {
      const float* Li = L + i + j0 * n;
#pragma unroll 4
      for (int64_t j = 0; j < jn; ++j) df_add_prod(sh, sl, Li[j * n], lp[j], 0.f);
    }
  }
  if (i >= n) return;
  if (active) {
    const double l = (col[i] - ((double)sh + (double)sl)) / lmm;
    const float lst = (float)l;
    L[i + m * n] = lst;
    const double lr = (double)lst;
    d[i] = __dsub_rn(d[i], __dmul_rn(lr, lr));
  } else if (i == piv) {
    L[i + m * n] = (float)lmm;
  }
}

void pivchol_run_df(const PivCholArgs& a, float* L, cudaStream_t st) {
  for (int64_t m = 0; m < a.k; ++m) {
    { pc_argmax_kernel<<<kArgBlocks, kArgThreads, 0, st>>>(m, a.n, 1, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                         a.ps, a.part, a.ticket); count_launch(); }
    a.get_col(a.pivots + m, a.col, &a.ps->stop, st);
    { pc_update_df_kernel<<<(unsigned)cdiv(a.n, 256), 256, 0, st>>>(m, a.n, L, a.col, a.d, a.chosen, a.ps); count_launch(); }
  }
  { pc_argmax_kernel<<<kArgBlocks, kArgThreads, 0, st>>>(a.k, a.n, 0, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                       a.ps, a.part, a.ticket); count_launch(); }
}

// ---------------------------------------------------------------- host driver
template <typename TL>
void pivchol_run(const PivCholArgs& a, TL* L, cudaStream_t st) {
  for (int64_t m = 0; m < a.k; ++m) {
    { pc_argmax_kernel<<<kArgBlocks, kArgThreads, 0, st>>>(m, a.n, 1, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                         a.ps, a.part, a.ticket); count_launch(); }
    a.get_col(a.pivots + m, a.col, &a.ps->stop, st);
    { pc_update_kernel<TL><<<(unsigned)cdiv(a.n, 256), 256, 0, st>>>(m, a.n, L, a.col, a.d, a.chosen, a.ps); count_launch(); }
  }
  // trace after the last step
  { pc_argmax_kernel<<<kArgBlocks, kArgThreads, 0, st>>>(a.k, a.n, 0, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                       a.ps, a.part, a.ticket); count_launch(); }
}

template void pivchol_run<double>(const PivCholArgs&, double*, cudaStream_t);
template void pivchol_run<float>(const PivCholArgs&, float*, cudaStream_t);

int pivchol_part_blocks() { return kArgBlocks; }

}  // namespace gdml
