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
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "ws_stage.cuh"

namespace gdml {

constexpr int kArgMaxBlocks = 1024;  // size of the argmax partial buffer
// two CTAs per SM for the argmax / trace reductions
inline int arg_blocks() { return std::min(2 * num_sms(), kArgMaxBlocks); }
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
    PivState* __restrict__ ps, ArgMaxPart* __restrict__ part, unsigned* __restrict__ ticket,
    int64_t* __restrict__ posof = nullptr) {
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
  const int64_t other = perm[m];
  perm[b.pos] = other;
  perm[m] = piv;
  if (posof) {
    posof[other] = b.pos;
    posof[piv] = m;
  }
  pivots[m] = piv;
  chosen[piv] = 1;
  ps->lmm = sqrt(d[piv]);
  ps->ilmm = 1.0 / ps->lmm;
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

// Alg. 1 step with FP32-stored L (DF64 contexts): the kernel column, then two kernels:
//   schur:   partial Schur sums over column groups, s_g(i) = sum_{j in g} l_{pivot,j} l_{i,j},
//            exact FP32 products summed in double-float; 512 rows per CTA, each warp
//            streams whole 2 KB column segments with the next column's loads in flight
//   finish:  s_i = sum_g s_g(i) (fixed order), l_{i,m} = (k_{m,i} - s_i) / l_{pivot,m} in FP64,
//            stored in FP32; the residual diagonal is updated with the stored value, and
//            the pivot of step m + 1 is selected and its row gathered (prow) in the same pass.
constexpr int kSchurRows = 512;
constexpr int kSchurMaxGroups = 16;

__device__ __forceinline__ void df_add_pair_pc(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float v = s - h;
  float e = (h - (s - v)) + (bh - v);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

template <bool VEC>
__device__ __forceinline__ float4 pc_load4(const float* __restrict__ col, int64_t base, int64_t rem) {
  if (VEC && base + 3 < rem) return __ldg(reinterpret_cast<const float4*>(col + base));
  float4 v;
  v.x = base < rem ? col[base] : 0.f;
  v.y = base + 1 < rem ? col[base + 1] : 0.f;
  v.z = base + 2 < rem ? col[base + 2] : 0.f;
  v.w = base + 3 < rem ? col[base + 3] : 0.f;
  return v;
}

template <bool VEC>
__global__ void __launch_bounds__(256, 2) pc_schur_df_kernel(int64_t m, int64_t n, const float* __restrict__ L,
                                                             const float* __restrict__ prow,
                                                             const PivState* __restrict__ ps,
                                                             float2* __restrict__ schur) {
  if (ps->stop) return;
  __shared__ float2 part[8][kSchurRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * kSchurRows;
  const int64_t rem = n - i0;
  const int64_t g = blockIdx.y;
  const int64_t ja = m * g / gridDim.y, jb = m * (g + 1) / gridDim.y;
  float h[16], l[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) h[e] = l[e] = 0.f;
  int64_t j = ja + warp;
  float4 a[4];
  if (j < jb) {
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = pc_load4<VEC>(L + j * n + i0, 128 * t + 4 * lane, rem);
  }
#pragma unroll 1
  for (; j < jb; j += 8) {
    float4 na[4];
    const bool more = j + 8 < jb;
    if (more) {
#pragma unroll
      for (int t = 0; t < 4; ++t) na[t] = pc_load4<VEC>(L + (j + 8) * n + i0, 128 * t + 4 * lane, rem);
    }
    const float p = prow[j];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      df_add_prod(h[4 * t + 0], l[4 * t + 0], a[t].x, p, 0.f);
      df_add_prod(h[4 * t + 1], l[4 * t + 1], a[t].y, p, 0.f);
      df_add_prod(h[4 * t + 2], l[4 * t + 2], a[t].z, p, 0.f);
      df_add_prod(h[4 * t + 3], l[4 * t + 3], a[t].w, p, 0.f);
    }
    if (more) {
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = na[t];
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) part[warp][128 * t + 4 * lane + e] = make_float2(h[4 * t + e], l[4 * t + e]);
  __syncthreads();
  for (int rr = threadIdx.x; rr < kSchurRows && rr < rem; rr += 256) {
    float hh = part[0][rr].x, ll = part[0][rr].y;
#pragma unroll
    for (int w = 1; w < 8; ++w) df_add_pair_pc(hh, ll, part[w][rr].x, part[w][rr].y);
    schur[g * n + i0 + rr] = make_float2(hh, ll);
  }
}

// Finish step m and select the pivot of step m + 1 in one kernel: every unchosen row i
// forms l_{i,m} = (k_{m,i} - s_i) / l_{pivot,m} (s_i from the Schur partials, FP64
// division, FP32 storage), updates its residual diagonal and offers (d_i, position of i)
// to the argmax of step m + 1 (ties -> lowest position, as pc_argmax_kernel); the
// per-CTA results are combined by the last CTA in a fixed order, which records the
// residual trace after step m, performs the swap of Alg. 1 and gathers the new pivot's
// row of L (columns 0..m) for the next Schur pass.  select = 0 on the last step.
__global__ void __launch_bounds__(kArgThreads) pc_finish_select_df_kernel(
    int64_t m, int64_t n, int groups, int select, float* __restrict__ L, const float2* __restrict__ schur,
    const double* __restrict__ col, double* __restrict__ d, unsigned char* __restrict__ chosen,
    int64_t* __restrict__ perm, int64_t* __restrict__ posof, int64_t* __restrict__ pivots,
    double* __restrict__ trace, PivState* __restrict__ ps, ArgMaxPart* __restrict__ part,
    unsigned* __restrict__ ticket, float* __restrict__ prow) {
  if (ps->stop) return;
  constexpr int kW = kArgThreads / 32;
  __shared__ double sv[kW];
  __shared__ int64_t sp[kW];
  __shared__ double ss[kW];
  __shared__ bool last;
  __shared__ int64_t s_piv;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t piv = ps->piv;
  const double lmm = ps->lmm, ilmm = ps->ilmm;  // one FP64 multiply per row instead of a division
  ArgMax best{-1.0 / 0.0, INT64_MAX};
  double sum = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kArgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kArgThreads) {
    // every operand of the row in one round of loads, before the branch
    const bool ch = chosen[i] != 0;
    const double ci = col[i], di = d[i];
    const int64_t pi = posof[i];
    float sh = 0.f, sl = 0.f;
    for (int g = 0; g < groups; ++g) {
      const float2 v = schur[(int64_t)g * n + i];
      df_add_pair_pc(sh, sl, v.x, v.y);
    }
    if (!ch) {
      const double lv = (ci - ((double)sh + (double)sl)) * ilmm;
      const float lst = (float)lv;
      L[i + m * n] = lst;
      const double lr = (double)lst;
      const double dn = __dsub_rn(di, __dmul_rn(lr, lr));
      d[i] = dn;
      sum += dn;
      best = better(best, ArgMax{dn, pi});
    } else if (i == piv) {
      L[i + m * n] = (float)lmm;
    }
  }
  // CTA reduction: xor butterflies within warps (better() is commutative), then warp 0
  for (int o = 16; o > 0; o >>= 1) {
    const ArgMax ob{__shfl_xor_sync(0xffffffffu, best.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)best.pos, o)};
    best = better(best, ob);
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if (lane == 0) {
    sv[warp] = best.v;
    sp[warp] = best.pos;
    ss[warp] = sum;
  }
  __syncthreads();
  if (warp == 0) {
    ArgMax bw = lane < kW ? ArgMax{sv[lane], sp[lane]} : ArgMax{-1.0 / 0.0, INT64_MAX};
    double sw = lane < kW ? ss[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bw.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bw.pos, o)};
      bw = better(bw, ob);
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    if (lane == 0) {
      part[blockIdx.x].v = bw.v;
      part[blockIdx.x].pos = bw.pos;
      part[blockIdx.x].sum = sw;
      __threadfence();
      last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  {
    ArgMax bt{-1.0 / 0.0, INT64_MAX};
    double st = 0.0;
    volatile ArgMaxPart* vp = part;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += kArgThreads) {
      bt = better(bt, ArgMax{vp[q].v, vp[q].pos});
      st += vp[q].sum;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bt.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bt.pos, o)};
      bt = better(bt, ob);
      st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if (lane == 0) {
      sv[warp] = bt.v;
      sp[warp] = bt.pos;
      ss[warp] = st;
    }
  }
  __syncthreads();
  if (warp == 0) {
    ArgMax bw = lane < kW ? ArgMax{sv[lane], sp[lane]} : ArgMax{-1.0 / 0.0, INT64_MAX};
    double sw = lane < kW ? ss[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bw.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bw.pos, o)};
      bw = better(bw, ob);
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    if (lane == 0) {
      sv[0] = bw.v;
      sp[0] = bw.pos;
      ss[0] = sw;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const ArgMax b{sv[0], sp[0]};
    *ticket = 0u;
    if (trace) trace[m] = ss[0];
    s_piv = -1;
    if (select) {
      const int64_t m1 = m + 1;
      if (!(b.v > 0.0) || b.pos >= n) {
        ps->stop = 1;
        ps->rank = m1;
      } else {
        const int64_t p = perm[b.pos];
        const int64_t other = perm[m1];
        perm[b.pos] = other;
        perm[m1] = p;
        posof[other] = b.pos;
        posof[p] = m1;
        pivots[m1] = p;
        chosen[p] = 1;
        ps->lmm = sqrt(d[p]);
        ps->ilmm = 1.0 / ps->lmm;
        ps->piv = p;
        ps->rank = m1 + 1;
        s_piv = p;
      }
    }
  }
  __syncthreads();
  const int64_t p = s_piv;
  if (p >= 0)  // the next pivot's row of L, columns 0..m (column m written above, fenced);
                // eight independent loads per thread in flight before the stores
    for (int64_t j0 = threadIdx.x; j0 <= m; j0 += 8 * kArgThreads) {
      float pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = j0 + (int64_t)u * kArgThreads;
        pv[u] = j <= m ? L[p + j * n] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = j0 + (int64_t)u * kArgThreads;
        if (j <= m) prow[j] = pv[u];
      }
    }
}

// Algorithm 1 step m in one TMA-staged pass: the Schur sums s_i = sum_{j<m} L[i + j n] prow[j]
// of ws_gemv_n_kernel's SCHUR mode, followed row by row (as each chunk's sums are combined)
// by pc_finish_select_df_kernel's work: l_{i,m}, column m of L, the residual diagonal, the
// argmax and the trace.  The last CTA to finish selects the pivot of step m + 1, performs
// the swap and gathers that pivot's row of L into prow (every CTA has read prow by then).
template <int NT>
__global__ void __launch_bounds__(kWsThreads, 2) pc_schur_finish_ws_kernel(
    const __grid_constant__ CUtensorMap map, int64_t n, int64_t m, int64_t nch, int select, float* __restrict__ L,
    float* __restrict__ prow, const double* __restrict__ col, double* __restrict__ d,
    unsigned char* __restrict__ chosen, int64_t* __restrict__ perm, int64_t* __restrict__ posof,
    int64_t* __restrict__ pivots, double* __restrict__ trace, PivState* __restrict__ ps,
    ArgMaxPart* __restrict__ part, unsigned* __restrict__ ticket, int* __restrict__ err, int evict_first) {
  constexpr int RC = 128 * NT, COLS = 32 / NT, CPW = 4 / NT;
  constexpr int kW = kWsWarps + 1;
  if (ps->stop) return;
  extern __shared__ uint8_t ws_smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws_smem_raw) + kWsAlign - 1) &
                                             ~uintptr_t(kWsAlign - 1));
  float2* cmb = reinterpret_cast<float2*>(ring + kWsStages * kWsTile);  // [warp][RC rows]
  uint64_t* full = reinterpret_cast<uint64_t*>(cmb + kWsWarps * 256);
  uint64_t* empty = full + kWsStages;
  uint64_t* cbar = empty + kWsStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(cbar + 2);
  __shared__ uint32_t issued_s;
  __shared__ double sv[kW];
  __shared__ int64_t sp[kW];
  __shared__ double ss[kW];
  __shared__ bool last;
  __shared__ int64_t s_piv;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (int)((m + COLS - 1) / COLS);
  const int64_t piv = ps->piv;
  const double lmm = ps->lmm, ilmm = ps->ilmm;
  if (threadIdx.x == 0) {
    ws_init(full, empty, cbar, abort_flag);
    issued_s = 0;
  }
  __syncthreads();
  ArgMax best{-1.0 / 0.0, INT64_MAX};
  double sum = 0.0;
  if (warp == kWsWarps) {
    if (lane == 0)
      issued_s = evict_first ? ws_produce<NT, true>(&map, ring, full, empty, abort_flag, nch, ntiles, err)
                             : ws_produce<NT, false>(&map, ring, full, empty, abort_flag, nch, ntiles, err);
  } else {
    WsRing rp;
    uint32_t ci = 0;
    bool go = true;
    for (int64_t ch = blockIdx.x; ch < nch && go; ch += gridDim.x, ++ci) {
      float2 h2[NT][2], l2[NT][2];
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int q = 0; q < 2; ++q) h2[t][q] = l2[t][q] = make_float2(0.f, 0.f);
      for (int s = 0; s < ntiles; ++s) {
        float xv[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const int64_t j = (int64_t)s * COLS + warp * CPW + c;
          xv[c] = j < m ? prow[j] : 0.f;
        }
        if (!ws_consume_wait(&full[rp.slot], rp.phase, abort_flag, err)) {
          go = false;
          break;
        }
        const float* tile = reinterpret_cast<const float*>(ring + rp.slot * kWsTile) + warp * CPW * RC;
        float4 a[CPW][NT];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
          for (int t = 0; t < NT; ++t) a[c][t] = *reinterpret_cast<const float4*>(tile + c * RC + 128 * t + 4 * lane);
        __syncwarp();
        if (lane == 0) ws_arrive(&empty[rp.slot]);
        rp.next();
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const float2 uh = make_float2(xv[c], xv[c]), un = make_float2(-xv[c], -xv[c]);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            df2_add_prod_lazy(h2[t][0], l2[t][0], lo_pair(a[c][t]), uh, un);
            df2_add_prod_lazy(h2[t][1], l2[t][1], hi_pair(a[c][t]), uh, un);
          }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
          for (int q = 0; q < 2; ++q) df2_renorm(h2[t][q], l2[t][q]);
      }
      if (!go) break;
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          cmb[warp * 256 + 128 * t + 4 * lane + 2 * q] = make_float2(h2[t][q].x, l2[t][q].x);
          cmb[warp * 256 + 128 * t + 4 * lane + 2 * q + 1] = make_float2(h2[t][q].y, l2[t][q].y);
        }
      if (!ws_consumer_sync(&cbar[0], ci & 1u, abort_flag, err)) break;
      const int64_t i0 = ch * RC;
      const int rr = threadIdx.x;  // 256 consumer threads, one row each
      if (rr < RC && i0 + rr < n) {
        const int64_t i = i0 + rr;
        const bool chs = chosen[i] != 0;
        const double ci_ = col[i], di = d[i];
        const int64_t pi = posof[i];
        float hh = cmb[rr].x, ll = cmb[rr].y;
#pragma unroll
        for (int w = 1; w < kWsWarps; ++w) df_add_pair_pc(hh, ll, cmb[w * 256 + rr].x, cmb[w * 256 + rr].y);
        if (!chs) {
          const double lv = (ci_ - ((double)hh + (double)ll)) * ilmm;
          const float lst = (float)lv;
          L[i + m * n] = lst;
          const double lr = (double)lst;
          const double dn = __dsub_rn(di, __dmul_rn(lr, lr));
          d[i] = dn;
          sum += dn;
          best = better(best, ArgMax{dn, pi});
        } else if (i == piv) {
          L[i + m * n] = (float)lmm;
        }
      }
      if (!ws_consumer_sync(&cbar[1], ci & 1u, abort_flag, err)) break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) ws_drain(full, issued_s);
  // CTA reduction (the producer warp holds neutral values), then the grid's through part[]
  for (int o = 16; o > 0; o >>= 1) {
    const ArgMax ob{__shfl_xor_sync(0xffffffffu, best.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)best.pos, o)};
    best = better(best, ob);
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if (lane == 0) {
    sv[warp] = best.v;
    sp[warp] = best.pos;
    ss[warp] = sum;
  }
  __syncthreads();
  if (warp == 0) {
    ArgMax bw = lane < kW ? ArgMax{sv[lane], sp[lane]} : ArgMax{-1.0 / 0.0, INT64_MAX};
    double sw = lane < kW ? ss[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bw.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bw.pos, o)};
      bw = better(bw, ob);
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    if (lane == 0) {
      part[blockIdx.x].v = bw.v;
      part[blockIdx.x].pos = bw.pos;
      part[blockIdx.x].sum = sw;
      __threadfence();
      last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  {
    ArgMax bt{-1.0 / 0.0, INT64_MAX};
    double st = 0.0;
    volatile ArgMaxPart* vp = part;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
      bt = better(bt, ArgMax{vp[q].v, vp[q].pos});
      st += vp[q].sum;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bt.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bt.pos, o)};
      bt = better(bt, ob);
      st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if (lane == 0) {
      sv[warp] = bt.v;
      sp[warp] = bt.pos;
      ss[warp] = st;
    }
  }
  __syncthreads();
  if (warp == 0) {
    ArgMax bw = lane < kW ? ArgMax{sv[lane], sp[lane]} : ArgMax{-1.0 / 0.0, INT64_MAX};
    double sw = lane < kW ? ss[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const ArgMax ob{__shfl_xor_sync(0xffffffffu, bw.v, o), (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bw.pos, o)};
      bw = better(bw, ob);
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    if (lane == 0) {
      const ArgMax b = bw;
      *ticket = 0u;
      if (trace) trace[m] = sw;
      s_piv = -1;
      if (select) {
        const int64_t m1 = m + 1;
        if (!(b.v > 0.0) || b.pos >= n) {
          ps->stop = 1;
          ps->rank = m1;
        } else {
          const int64_t p = perm[b.pos];
          const int64_t other = perm[m1];
          perm[b.pos] = other;
          perm[m1] = p;
          posof[other] = b.pos;
          posof[p] = m1;
          pivots[m1] = p;
          chosen[p] = 1;
          ps->lmm = sqrt(d[p]);
          ps->ilmm = 1.0 / ps->lmm;
          ps->piv = p;
          ps->rank = m1 + 1;
          s_piv = p;
        }
      }
    }
  }
  __syncthreads();
  const int64_t p = s_piv;
  if (p >= 0)  // the next pivot's row of L, columns 0..m (column m written above, fenced)
    for (int64_t j0 = threadIdx.x; j0 <= m; j0 += 8 * (int64_t)blockDim.x) {
      float pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = j0 + (int64_t)u * blockDim.x;
        pv[u] = j <= m ? L[p + j * n] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = j0 + (int64_t)u * blockDim.x;
        if (j <= m) prow[j] = pv[u];
      }
    }
}

int pivchol_schur_groups() { return kSchurMaxGroups; }

void pivchol_run_df(const PivCholArgs& a, float* L, cudaStream_t st) {
  const int64_t rblocks = cdiv(a.n, kSchurRows);
  const bool vec = (a.n % 4) == 0;
  const unsigned fblocks = (unsigned)std::min<int64_t>(cdiv(a.n, kArgThreads), arg_blocks());
  // n % 4 == 0: the Schur sums run through the TMA-staged pass (one partial per row)
  WsPlan plan;
  if (a.err) ws_plan(plan, L, a.n, a.k);
  // one argmax partial per CTA: the staged kernel's grid-stride loop takes any grid size
  if (plan.grid > arg_blocks()) plan.grid = arg_blocks();
  // step 0's pivot
  { pc_argmax_kernel<<<arg_blocks(), kArgThreads, 0, st>>>(0, a.n, 1, a.d, a.perm, a.chosen, a.pivots, nullptr,
                                                       a.ps, a.part, a.ticket, a.posof); count_launch(); }
  if (plan.ok) {  // two launches per step: the kernel column, then Schur sums + finish
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(pc_schur_finish_ws_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmemN);
      cudaFuncSetAttribute(pc_schur_finish_ws_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmemN);
      attr = true;
    }
    for (int64_t m = 0; m < a.k; ++m) {
      a.get_col(a.pivots + m, a.col, &a.ps->stop, st);
      const int select = m + 1 < a.k ? 1 : 0;
      // once the first m columns no longer fit in L2 they are streamed evict-first, so the
      // kernel column's operands (X, G as float pairs) and the per-row state stay resident
      const int ef = (double)m * (double)a.n * 4.0 > 96.0 * 1024 * 1024 ? 1 : 0;
      if (plan.rc == 256)
        { pc_schur_finish_ws_kernel<2><<<plan.grid, kWsThreads, kWsSmemN, st>>>(plan.map, a.n, m, plan.nch, select, L, a.prow, a.col, a.d, a.chosen, a.perm, a.posof, a.pivots, a.trace, a.ps, a.part, a.ticket, a.err, ef); count_launch(); }
      else
        { pc_schur_finish_ws_kernel<1><<<plan.grid, kWsThreads, kWsSmemN, st>>>(plan.map, a.n, m, plan.nch, select, L, a.prow, a.col, a.d, a.chosen, a.perm, a.posof, a.pivots, a.trace, a.ps, a.part, a.ticket, a.err, ef); count_launch(); }
    }
    return;
  }
  for (int64_t m = 0; m < a.k; ++m) {
    a.get_col(a.pivots + m, a.col, &a.ps->stop, st);
    // column groups: enough CTAs for ~4 per SM, at least 32 columns per group
    int groups = 0;
    if (m > 0) {
      const int64_t want = cdiv(4 * (int64_t)num_sms(), rblocks);
      groups = (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)kSchurMaxGroups, std::max<int64_t>(1, m / 32)}));
      dim3 g((unsigned)rblocks, (unsigned)groups);
      if (vec)
        { pc_schur_df_kernel<true><<<g, 256, 0, st>>>(m, a.n, L, a.prow, a.ps, a.schur); count_launch(); }
      else
        { pc_schur_df_kernel<false><<<g, 256, 0, st>>>(m, a.n, L, a.prow, a.ps, a.schur); count_launch(); }
    }
    { pc_finish_select_df_kernel<<<fblocks, kArgThreads, 0, st>>>(m, a.n, groups, m + 1 < a.k ? 1 : 0, L, a.schur, a.col, a.d, a.chosen, a.perm, a.posof, a.pivots, a.trace, a.ps, a.part, a.ticket, a.prow); count_launch(); }
  }
}

// ---------------------------------------------------------------- host loop (FP64 and FP32 sums)
template <typename TL>
void pivchol_run(const PivCholArgs& a, TL* L, cudaStream_t st) {
  for (int64_t m = 0; m < a.k; ++m) {
    { pc_argmax_kernel<<<arg_blocks(), kArgThreads, 0, st>>>(m, a.n, 1, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                         a.ps, a.part, a.ticket); count_launch(); }
    a.get_col(a.pivots + m, a.col, &a.ps->stop, st);
    { pc_update_kernel<TL><<<(unsigned)cdiv(a.n, 256), 256, 0, st>>>(m, a.n, L, a.col, a.d, a.chosen, a.ps); count_launch(); }
  }
  // trace after the last step
  { pc_argmax_kernel<<<arg_blocks(), kArgThreads, 0, st>>>(a.k, a.n, 0, a.d, a.perm, a.chosen, a.pivots, a.trace,
                                                       a.ps, a.part, a.ticket); count_launch(); }
}

template void pivchol_run<double>(const PivCholArgs&, double*, cudaStream_t);
template void pivchol_run<float>(const PivCholArgs&, float*, cudaStream_t);

int pivchol_part_blocks() { return kArgMaxBlocks; }

cudaError_t set_wait_limit_pc(uint32_t polls) { return tc::set_wait_limit_here(polls); }

}  // namespace gdml
