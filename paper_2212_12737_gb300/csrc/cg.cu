// CG vector kernels (Sec. 2.1, Eq. 2): deterministic dot products and the
// fused PCG updates.  Scalars stay in device memory; no host round trip is
// needed inside an iteration.
//
// Every reduction uses a fixed grid (dot_blocks() CTAs, each a contiguous
// chunk) and a fixed combination order, so results are bitwise reproducible
// on a given device.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

constexpr int kDotMaxBlocks = 2048;  // the context's partial buffer holds 4096 doubles
// two CTAs per SM; the same grid for every reduction of the loop (bitwise-equal r.r)
inline int dot_blocks() { return std::min(2 * num_sms(), kDotMaxBlocks); }
constexpr int kDotThreads = 256;

// partial[blockIdx.x] = sum over the CTA's chunk of x*y; the last CTA to finish
// sums the partials in index order into *out (and zeroes the ticket).
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const double* __restrict__ x,
                                                          const double* __restrict__ y, int64_t n,
                                                          double* __restrict__ partial,
                                                          unsigned* __restrict__ ticket,
                                                          double* __restrict__ out) {
  __shared__ double red[kDotThreads / 32];
  __shared__ bool last;
  const int64_t chunk = cdiv_dev(n, gridDim.x);
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  double s = 0.0;
  for (int64_t i = beg + threadIdx.x; i < end; i += kDotThreads) s = fma(x[i], y[i], s);
  s = block_sum<kDotThreads>(s, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA combines the partials: thread t sums t, t+256, ... then a fixed tree
  double tot = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kDotThreads) tot += ((volatile double*)partial)[b];
  tot = block_sum<kDotThreads>(tot, red);
  if (threadIdx.x == 0) {
    *out = tot;
    *ticket = 0u;
  }
}

// x += gamma p; r -= gamma q (gamma = sc[RHO] / sc[PQ]), fused with sc[RR] = r.r over the same
// contiguous chunks and combination order as dot_kernel (bitwise the same r.r), and with the
// end-of-iteration test of the graph-captured loop in the last CTA: count the iteration and
// keep the WHILE node running while |r|^2 > tol^2, the residual is finite, no breakdown was
// flagged and the iteration cap is not reached.
// A breakdown (pq not positive and finite) flags status and leaves x, r untouched.
// With hist, the last CTA records gamma of this iteration (the Lanczos matrix of the run).
__global__ void __launch_bounds__(kDotThreads) update_xr_rr_kernel(double* __restrict__ x, double* __restrict__ r,
                                                                   const double* __restrict__ p,
                                                                   const double* __restrict__ q, int64_t n,
                                                                   double* __restrict__ sc, int* __restrict__ status,
                                                                   double* __restrict__ partial,
                                                                   unsigned* __restrict__ ticket, int64_t* ictl,
                                                                   cudaGraphConditionalHandle h, int check,
                                                                   double* __restrict__ hist) {
  __shared__ double red[kDotThreads / 32];
  __shared__ bool last;
  const double pq = sc[SC_PQ];
  const bool ok = pq > 0.0 && isfinite(pq);
  const double gamma = ok ? sc[SC_RHO] / pq : 0.0;
  const int64_t chunk = cdiv_dev(n, gridDim.x);
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  double s = 0.0;
  for (int64_t i = beg + threadIdx.x; i < end; i += kDotThreads) {
    double ri = r[i];
    if (ok) {
      x[i] = fma(gamma, p[i], x[i]);
      ri = fma(-gamma, q[i], ri);
      r[i] = ri;
    }
    s = fma(ri, ri, s);
  }
  s = block_sum<kDotThreads>(s, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kDotThreads) tot += ((volatile double*)partial)[b];
  tot = block_sum<kDotThreads>(tot, red);
  if (threadIdx.x == 0) {
    if (!ok) *status = 1;
    sc[SC_RR] = tot;
    *ticket = 0u;
    if (check) {
      if (hist && ictl[IC_ITER] < ictl[IC_HCAP]) hist[2 * ictl[IC_ITER]] = gamma;
      const int64_t it = ictl[IC_ITER] + 1;
      ictl[IC_ITER] = it;
      const bool go = (tot > sc[SC_TOL2]) && isfinite(tot) && (it < ictl[IC_MAXIT]) && ok && (*status == 0);
      cudaGraphSetConditional(h, go ? 1u : 0u);
    }
  }
}

// p = z + (rho_new / rho) p, then rho <- rho_new in the last CTA (after every CTA has read it);
// with hist it also records the ratio of the iteration just counted by update_xr_rr_kernel
__global__ void __launch_bounds__(256) update_p_rho_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                           int64_t n, double* __restrict__ sc,
                                                           unsigned* __restrict__ ticket,
                                                           const int64_t* __restrict__ ictl,
                                                           double* __restrict__ hist) {
  __shared__ bool last;
  const double beta = sc[SC_RHO_NEW] / sc[SC_RHO];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    if (hist) {
      const int64_t j = ictl[IC_ITER] - 1;
      if (j >= 0 && j < ictl[IC_HCAP]) hist[2 * j + 1] = beta;
    }
    sc[SC_RHO] = sc[SC_RHO_NEW];
    *ticket = 0u;
  }
}

__global__ void axpby_kernel(double* __restrict__ y, const double* __restrict__ x, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

// Entry test of a batched PCG loop: run the WHILE body only if this system
// still has work (|r|^2 > tol^2 and iterations left).
__global__ void pcg_gate_kernel(const double* __restrict__ sc, const int64_t* __restrict__ ictl,
                                cudaGraphConditionalHandle h) {
  const bool go = (sc[SC_RR] > sc[SC_TOL2]) && (ictl[IC_ITER] < ictl[IC_MAXIT]);
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ---------------------------------------------------------------- launchers
cudaError_t add_pcg_gate_node(cudaGraph_t g, cudaGraphNode_t* node, const double* sc, const int64_t* ictl,
                              cudaGraphConditionalHandle h) {
  void* args[] = {(void*)&sc, (void*)&ictl, (void*)&h};
  cudaKernelNodeParams p = {};
  p.func = (void*)pcg_gate_kernel;
  p.gridDim = dim3(1);
  p.blockDim = dim3(1);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, nullptr, 0, &p);
}
void launch_dot(const double* x, const double* y, int64_t n, double* partial, unsigned* ticket, double* out,
                cudaStream_t st) {
  { dot_kernel<<<dot_blocks(), kDotThreads, 0, st>>>(x, y, n, partial, ticket, out); count_launch(); }
}
void launch_update_xr_rr(double* x, double* r, const double* p, const double* q, int64_t n, double* sc, int* status,
                         double* partial, unsigned* ticket, int64_t* ictl, cudaGraphConditionalHandle h, int check,
                         double* hist, cudaStream_t st) {
  { update_xr_rr_kernel<<<dot_blocks(), kDotThreads, 0, st>>>(x, r, p, q, n, sc, status, partial, ticket, ictl, h, check, hist); count_launch(); }
}
void launch_update_p_rho(double* p, const double* z, int64_t n, double* sc, unsigned* ticket, const int64_t* ictl,
                         double* hist, cudaStream_t st) {
  { update_p_rho_kernel<<<4 * num_sms(), 256, 0, st>>>(p, z, n, sc, ticket, ictl, hist); count_launch(); }
}
void launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st) {
  { axpby_kernel<<<4 * num_sms(), 256, 0, st>>>(y, x, a, b, n); count_launch(); }
}

}  // namespace gdml
