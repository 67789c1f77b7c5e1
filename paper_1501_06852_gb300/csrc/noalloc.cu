// Step combination and error estimate for callers that cannot allocate device memory.
//
// Code that runs where cudaMalloc is not an option - inside a CUDA stream capture
// (an allocation there would break or invalidate the capture), in a loop that
// must not touch the device allocator once it is running, or as a guest in an
// application whose memory manager owns every device byte - cannot create a
// solver context.  It can still combine the stage increments it already holds
// into the new state and get the embedded error estimate of the step through
// pfc_step_combine_static: the caller passes every input and output, and the
// only working memory, the per-block partial sums of the error reduction, is a
// fixed static device array of this file.
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "pfc.h"

namespace {

// Per-block partial sums of the error reduction: one double per block of the
// combination kernel.  Every GPU that loads the library holds these 8 KiB until
// the process exits; every call shares them (see pfc_step_combine_static).
constexpr int kStaticParts = 1024;
__device__ __align__(256) static double g_step_scratch[kStaticParts];

// Largest n: the combination kernel walks 3n entries with a 32-bit int index in
// steps of (its kStaticParts blocks x 256 threads); the last step must not pass
// INT_MAX, so 3n + kStaticParts * 256 <= 2^31 - 1.
constexpr int64_t kStaticStride = (int64_t)kStaticParts * 256;
constexpr int64_t kStaticMaxN = ((int64_t)0x7fffffff - kStaticStride) / 3;
static_assert(kStaticMaxN == 715740501, "limit stated in pfc.h");

// Ros3Pw weights m and mhat (Table 1); the error vector is sum (mhat_j - m_j) y_j.
constexpr double kStaticM[3] = {1.63397459621556, 0.294228634059948, 1.07179676972449};
constexpr double kStaticMhat[3] = {1.99444650053487, 0.654700538379252, 1.07179676972449};

// Device address of g_step_scratch for each device, looked up once per device.
std::mutex g_static_mutex;
void* g_static_ptr[64] = {};

}  // namespace

extern "C" pfc_status pfc_step_combine_static(int64_t n, const double* state, const double* y, double atol,
                                              double rtol, double* state_new, double* err, void* cuda_stream) {
  if (n < 1 || n > kStaticMaxN) return PFC_ERR_INVALID;
  if (!state || !y || !state_new || !err) return PFC_ERR_INVALID;
  if (!(atol >= 0.0) || !(rtol >= 0.0) || atol + rtol <= 0.0) return PFC_ERR_INVALID;
  if (pfc::step_partials() > kStaticParts) return PFC_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PFC_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mutex);
    if (!g_static_ptr[dev]) {
      // In host code g_step_scratch names a host-side stand-in, not device
      // memory: its device address must be looked up (with this device current).
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_step_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PFC_ERR_CUDA;
      }
      g_static_ptr[dev] = p;
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nn = (int)n;
  const size_t n3 = 3 * (size_t)n;
  double e[3];
  for (int j = 0; j < 3; ++j) e[j] = kStaticMhat[j] - kStaticM[j];
  // every block overwrites its own partial and the reduction reads exactly those,
  // so nothing in the shared array needs clearing between calls
  if (pfc::launch_step_combine(nn, state, y, y + n3, y + 2 * n3, kStaticM, e, atol, rtol, state_new,
                               (double*)scratch, pfc::step_partials(), st) != cudaSuccess)
    return PFC_ERR_CUDA;
  if (pfc::launch_reduce_partials(pfc::step_partials(), (const double*)scratch, 1.0 / (double)n, err, st) !=
      cudaSuccess)
    return PFC_ERR_CUDA;
  return PFC_OK;
}
