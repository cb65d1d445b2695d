// gdml_matvec_noalloc: the FP64 force-kernel matvec without a context and
// without any device allocation, for callers that cannot call cudaMalloc.
//
// All working memory (descriptors, Jacobian factors, distance tables, the
// two contraction results) lives in one file-scope __device__ array sized for
// M <= kNoAllocMaxM geometries of N <= kNoAllocMaxN atoms.  Host code never
// names the array directly: the first call on a device looks up its device
// address with cudaGetSymbolAddress (with that device current) and caches it
// per device; that first call should therefore happen before any stream
// capture.  The cached address belongs to the device's primary context: it
// does not survive cudaDeviceReset, and calls made under another context of
// the same device must not use this entry point.  A stream of another device
// than the current one is rejected.  Every call overwrites the whole region
// it uses before reading it, so nothing has to start at zero; calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race on the array.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace gdml {
namespace {

constexpr int64_t kNoAllocMaxM = 128;
constexpr int kNoAllocMaxN = 24;
constexpr int64_t kNoAllocMaxD = (int64_t)kNoAllocMaxN * (kNoAllocMaxN - 1) / 2;
// X, 3 G, [W ; Xc], U: 7 M D;  S, [A | beta], T: 4 M^2;  t, rowsum: 2 M
constexpr int64_t kNoAllocDoubles =
    7 * kNoAllocMaxM * kNoAllocMaxD + 4 * kNoAllocMaxM * kNoAllocMaxM + 2 * kNoAllocMaxM;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];  // 2.5 MB per device

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

gdml_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(GDML_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(GDML_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return GDML_OK;
}

}  // namespace
}  // namespace gdml

using namespace gdml;

extern "C" gdml_status gdml_matvec_noalloc(const double* R_dev, int64_t M, int32_t N, double sigma, double lambda,
                                           const double* v_dev, double* out_dev, int32_t add_lambda,
                                           void* cuda_stream) {
  clear_msg();
  if (!R_dev || !v_dev || !out_dev || v_dev == out_dev) return fail(GDML_ERR_ARG, "matvec_noalloc: bad pointers");
  if (M < 1 || M > kNoAllocMaxM || N < 2 || N > kNoAllocMaxN)
    return fail(GDML_ERR_ARG, "matvec_noalloc: needs 1 <= M <= " + std::to_string(kNoAllocMaxM) +
                                  " geometries and 2 <= N <= " + std::to_string(kNoAllocMaxN) + " atoms");
  if (!(sigma > 0.0) || !(lambda >= 0.0)) return fail(GDML_ERR_ARG, "matvec_noalloc: need sigma > 0, lambda >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (st) {  // the scratch address is the current device's: the stream must belong to it
    int cur = 0, sdev = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess) e = cudaStreamGetDevice(st, &sdev);
    if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("matvec_noalloc: ") + cudaGetErrorString(e));
    if (sdev != cur)
      return fail(GDML_ERR_ARG, "matvec_noalloc: the stream belongs to device " + std::to_string(sdev) +
                                    " but device " + std::to_string(cur) + " is current");
  }
  double* base = nullptr;
  gdml_status s = scratch_address(&base);
  if (s != GDML_OK) return s;
  const int D = N * (N - 1) / 2;
  const double c = std::sqrt(5.0) / sigma;
  double* X = base;
  double* G = X + M * D;
  double* S = G + 3 * M * D;
  double* P64 = S + M * M;      // M x 2M : [A | beta]
  double* V64 = P64 + 2 * M * M;  // 2M x D : [W ; Xc]
  double* T = V64 + 2 * M * D;
  double* tb = T + M * M;
  double* rowsum = tb + M;
  double* U = rowsum + M;  // M x D
  double* W = V64;
  double* Xc = V64 + M * D;
  launch_desc_jac(R_dev, M, N, D, X, G, st);
  launch_center(X, M, D, Xc, st);
  launch_dist_tab(X, M, D, c, S, P64, 2 * M, st);
  launch_proj(G, Xc, v_dev, M, N, D, W, D, tb, st);
  launch_dgemm<double, double>(true, M, M, D, 1.0, Xc, D, W, D, 0.0, T, M, false, st);
  launch_beta(T, S, tb, M, c, P64 + M, 2 * M, rowsum, st);
  launch_dgemm<double, double>(false, M, D, 2 * M, 1.0, P64, 2 * M, V64, D, 0.0, U, D, false, st);
  launch_backproj<double>(U, D, 1, 0, rowsum, Xc, G, v_dev, M, N, D, lambda, add_lambda ? 1 : 0, out_dev, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GDML_ERR_CUDA, std::string("matvec_noalloc: ") + cudaGetErrorString(e));
  return GDML_OK;
}
