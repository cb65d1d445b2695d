// Inducing-column selection (Sec. 3, "Column selection strategies"):
//   uniform:   the k smallest Philox4x32-10 uniforms (sampling without replacement)
//   weighted:  the k smallest keys -ln(u_i) / tau_i (Efraimidis-Spirakis sampling
//              without replacement proportional to tau, used for ridge leverage scores)
// Keys are sorted together with their index (ties -> lower index) by a bitonic
// sort in global memory; the first k indices are the selection.
//
// Philox4x32-10 (Salmon et al., SC'11): round (c0,c1,c2,c3) ->
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
//   M0 = 0xD2511F53, M1 = 0xCD9E8D57, key bumped by (0x9E3779B9, 0xBB67AE85), 10 rounds.
// Counter (i lo, i hi, stream, 0), key (seed lo, seed hi); the 53-bit integer
// m = ((o0 >> 5) << 26) + (o1 >> 6) gives u = (m + 1) 2^-53.
#include "common.cuh"
#include "kernels.cuh"

namespace gdml {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ uint64_t philox_mant53(uint64_t i, uint32_t stream, uint64_t seed) {
  uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)(c[0] >> 5) << 26) + (uint64_t)(c[1] >> 6);
}

// keys for i < n; padding (n <= i < P) gets UINT64_MAX so it sorts last
__global__ void uniform_keys_kernel(int64_t n, int64_t P, uint64_t seed, uint32_t stream,
                                    uint64_t* __restrict__ key, int64_t* __restrict__ idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P) return;
  key[i] = i < n ? philox_mant53((uint64_t)i, stream, seed) : ~0ull;
  idx[i] = i;
}

__global__ void weighted_keys_kernel(int64_t n, int64_t P, uint64_t seed, uint32_t stream,
                                     const double* __restrict__ tau, uint64_t* __restrict__ key,
                                     int64_t* __restrict__ idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P) return;
  uint64_t kb = ~0ull;
  if (i < n) {
    const double t = tau[i];
    if (t > 0.0) {
      const double u = (double)(philox_mant53((uint64_t)i, stream, seed) + 1ull) * 0x1.0p-53;
      const double e = (0.0 - log(u)) / t;  // >= +0.0, so its bit pattern orders like the value
      kb = (uint64_t)__double_as_longlong(e);
    } else {
      kb = 0x7FF0000000000000ull;  // +inf
    }
  }
  key[i] = kb;
  idx[i] = i;
}

__global__ void bitonic_step_kernel(uint64_t* __restrict__ key, int64_t* __restrict__ idx, int64_t P,
                                    int64_t kk, int64_t jj) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P) return;
  int64_t l = i ^ jj;
  if (l <= i) return;
  const bool up = (i & kk) == 0;
  uint64_t ki = key[i], kl = key[l];
  int64_t ii = idx[i], il = idx[l];
  const bool gt = (ki > kl) || (ki == kl && ii > il);
  if (gt == up) {
    key[i] = kl;
    key[l] = ki;
    idx[i] = il;
    idx[l] = ii;
  }
}

static void bitonic_sort(uint64_t* key, int64_t* idx, int64_t P, cudaStream_t st) {
  const unsigned blocks = (unsigned)cdiv(P, 256);
  for (int64_t kk = 2; kk <= P; kk <<= 1)
    for (int64_t jj = kk >> 1; jj > 0; jj >>= 1) { bitonic_step_kernel<<<blocks, 256, 0, st>>>(key, idx, P, kk, jj); count_launch(); }
}

int64_t select_scratch_len(int64_t n) {
  int64_t P = 1;
  while (P < n) P <<= 1;
  return P;
}

// out[0..k) = indices of the k smallest keys; key/idx scratch of select_scratch_len(n)
void select_uniform(int64_t n, int64_t k, uint64_t seed, uint32_t stream, uint64_t* key, int64_t* idx,
                    int64_t* out, cudaStream_t st) {
  const int64_t P = select_scratch_len(n);
  { uniform_keys_kernel<<<(unsigned)cdiv(P, 256), 256, 0, st>>>(n, P, seed, stream, key, idx); count_launch(); }
  bitonic_sort(key, idx, P, st);
  cudaMemcpyAsync(out, idx, k * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

void select_weighted(int64_t n, int64_t k, uint64_t seed, uint32_t stream, const double* tau, uint64_t* key,
                     int64_t* idx, int64_t* out, cudaStream_t st) {
  const int64_t P = select_scratch_len(n);
  { weighted_keys_kernel<<<(unsigned)cdiv(P, 256), 256, 0, st>>>(n, P, seed, stream, tau, key, idx); count_launch(); }
  bitonic_sort(key, idx, P, st);
  cudaMemcpyAsync(out, idx, k * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

}  // namespace gdml
