// lbm_reduce3_noalloc: the compensated three-array reduction behind
// lbm_totals (the same kernels and block partition, so the same sums), for
// callers that cannot allocate device memory (a real-time loop with a fixed
// memory budget, code running inside a memory pool it does not own, or a host
// framework that forbids cudaMalloc after start-up).  Its per-block partial
// sums live in one fixed file-scope device array instead of memory obtained
// per call; nothing is allocated or freed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "launch.cuh"

// Defined in engine.cu (not exported): sets the text lbm_last_error(NULL) returns.
void lbmi_set_error(const char* msg);

namespace {

// Scratch shared by every call on a device: (sum, compensation) x 3 for each
// of the kReduceParts blocks of the reduction lbm_totals runs (48 KiB).
static __device__ __align__(256) double g_partials[lbm::kReduceParts * 6];

// Device address of g_partials, looked up once per device.  In host code the
// name g_partials denotes a host-side shadow, not device memory, so the kernel
// must be given the address that cudaGetSymbolAddress reports.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Error text goes to the engine's context-free error slot, which
// lbm_last_error(NULL) reports.
int report(int code, const char* fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  lbmi_set_error(msg);
  return code;
}

}  // namespace

extern "C" {

int lbm_reduce3_noalloc(const double* d_a, const double* d_b, const double* d_c, int64_t n,
                        double* d_out3, void* cuda_stream) {
  if (!d_out3 || n < 0)
    return report(LBM_EINVAL, "lbm_reduce3_noalloc: null output or negative length");
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return report(LBM_ECUDA, "lbm_reduce3_noalloc: scratch address: %s", cudaGetErrorString(e));
  e = lbm::launch_reduce3(d_a, d_b, d_c, n, scratch, lbm::kReduceParts, d_out3,
                          static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess)
    return report(LBM_ECUDA, "lbm_reduce3_noalloc: launch: %s", cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"
