// Shared helpers for the libgdml CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/gdml.h"

namespace gdml {

// Streaming multiprocessors of the current device (152 on GB300: 2 dies x 76), queried once per
// device; grids are sized in multiples of it.
int num_sms();

// Host-side error carrier: every internal call returns a gdml_status and
// writes a message into the context.
struct Err {
  gdml_status st = GDML_OK;
  std::string msg;
};

#define GDML_CUDA_TRY(expr)                                                              \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      return ::gdml::fail(GDML_ERR_CUDA, std::string(#expr " -> ") + cudaGetErrorString(_e)); \
    }                                                                                    \
  } while (0)

// thread-local last error (used when no context exists yet)
gdml_status fail(gdml_status st, const std::string& msg);
const std::string& last_msg();
void clear_msg();

// host-side count of kernel launches issued by this library (inside CUDA
// graphs a captured launch counts once per replay; see count_graph_launches)
void count_launch(int64_t n = 1);
int64_t launch_count();

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__device__ __forceinline__ int64_t cdiv_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// (sh, sl) += a * (bh + bl) in double-float: a * bh formed exactly by FMA
// (TwoProduct), the a * bl term folded into the low part, summed by TwoSum.
__device__ __forceinline__ void df_add_prod(float& sh, float& sl, float a, float bh, float bl) {
  const float ph = a * bh;
  float pl = fmaf(a, bh, -ph);
  pl = fmaf(a, bl, pl);
  const float t = sh + ph;
  const float v = t - sh;
  float e = (sh - (t - v)) + (ph - v);
  e += sl + pl;
  sh = t + e;
  sl = e - (sh - t);
}

// Deterministic block reduction of one double (fixed tree order).
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < THREADS / 32 ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// p = i(i-1)/2 + j with i > j  ->  (i, j)
__device__ __forceinline__ void pair_of(int p, int& i, int& j) {
  // FP32 estimate (GB300's FP64 pipe is slow), then exact integer correction
  int ii = (int)((1.f + sqrtf(1.f + 8.f * (float)p)) * 0.5f);
  while (ii * (ii - 1) / 2 > p) --ii;
  while ((ii + 1) * ii / 2 <= p) ++ii;
  i = ii;
  j = p - ii * (ii - 1) / 2;
}
__device__ __forceinline__ int pair_idx(int i, int j) {  // requires i != j
  return i > j ? i * (i - 1) / 2 + j : j * (j - 1) / 2 + i;
}


}  // namespace gdml
