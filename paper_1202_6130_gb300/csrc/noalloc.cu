// lbm_reduce3_noalloc: the compensated three-array reduction behind
// lbm_totals, for callers that cannot allocate device memory (a real-time
// loop with a fixed memory budget, code running inside a memory pool it does
// not own, or a host framework that forbids cudaMalloc after start-up).  Its
// per-block partial sums live in one fixed file-scope device array instead of
// memory obtained per call; nothing is allocated or freed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"

// Defined in engine.cu (not exported): sets the text lbm_last_error(NULL) returns.
void lbmi_set_error(const char* msg);

namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 65536;  // elements summed by one block
constexpr int kMaxBlocks = 4096;   // => at most kMaxBlocks * kChunk = 2^28 elements

// Scratch shared by every call on a device: (sum, compensation) x 3 per block.
// 4096 * 6 doubles = 192 KiB, held by each GPU that loads the library.
static __device__ __align__(256) double g_partials[kMaxBlocks * 6];

__device__ inline void neum_add(double& s, double& c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

// Block b sums elements [b * kChunk, min(n, (b + 1) * kChunk)).
__global__ void noalloc_block_sums(const double* __restrict__ a, const double* __restrict__ b,
                                   const double* __restrict__ c, int64_t n,
                                   double* __restrict__ partials) {
  __shared__ double sh[3][2][kThreads];
  const double* src[3] = {a, b, c};
  double s[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  const int64_t lo = (int64_t)blockIdx.x * kChunk;
  const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads)
    for (int q = 0; q < 3; ++q)
      if (src[q]) neum_add(s[q], k[q], src[q][i]);
  for (int q = 0; q < 3; ++q) {
    sh[q][0][threadIdx.x] = s[q];
    sh[q][1][threadIdx.x] = k[q];
  }
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int q = 0; q < 3; ++q) {
        double ss = sh[q][0][threadIdx.x], cc = sh[q][1][threadIdx.x];
        neum_add(ss, cc, sh[q][0][threadIdx.x + w]);
        cc += sh[q][1][threadIdx.x + w];
        sh[q][0][threadIdx.x] = ss;
        sh[q][1][threadIdx.x] = cc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) {
      partials[(int64_t)blockIdx.x * 6 + 2 * q] = sh[q][0][0];
      partials[(int64_t)blockIdx.x * 6 + 2 * q + 1] = sh[q][1][0];
    }
}

__global__ void noalloc_final(const double* __restrict__ partials, int nparts,
                              double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 3; ++q) {
    double s = 0.0, c = 0.0;
    for (int p = 0; p < nparts; ++p) {
      neum_add(s, c, partials[6 * p + 2 * q]);
      c += partials[6 * p + 2 * q + 1];
    }
    out[q] = s + c;
  }
}

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
  if (n > (int64_t)kMaxBlocks * kChunk)
    return report(LBM_EINVAL,
                  "lbm_reduce3_noalloc: %lld elements exceed the fixed scratch limit of %lld "
                  "(%d blocks of %lld elements)",
                  (long long)n, (long long)kMaxBlocks * kChunk, kMaxBlocks, (long long)kChunk);
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return report(LBM_ECUDA, "lbm_reduce3_noalloc: scratch address: %s", cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = n == 0 ? 1 : (int)((n + kChunk - 1) / kChunk);
  noalloc_block_sums<<<nblocks, kThreads, 0, st>>>(d_a, d_b, d_c, n, scratch);
  noalloc_final<<<1, 32, 0, st>>>(scratch, nblocks, d_out3);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return report(LBM_ECUDA, "lbm_reduce3_noalloc: launch: %s", cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"
