// Allocation-free entry point: the deterministic multi-vector dot product
// (the reduction FGMRES uses for its Gram-Schmidt coefficients and norms),
// with its partial sums kept in a fixed device array instead of memory the
// library would allocate.
//
// Who needs it: callers that may not call cudaMalloc (or any allocator) at
// the point where they want the result -- code driven by a memory manager
// that owns all device memory and forbids further allocations, or real-time
// loops where an allocation's latency or possible failure is not acceptable.
// They pass their inputs and outputs; the only other memory touched is the
// array below.  The kernels are the solver's own (launch_multidot), so the
// results are bitwise those of the FGMRES reduction.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "msp.h"
#include "msp_kernels.h"

namespace msp {
int fail(int code, const std::string& msg);
}

namespace {

constexpr int kNaBlocks = msp::kDotBlocks;  // stage-1 blocks per vector, as in the solver

// Partial sums of every call: MSP_NOALLOC_MAX_VECTORS x kNaBlocks doubles
// (64 x 296 x 8 B = 151,552 B), resident on every GPU that loads the library
// until the process exits.  Each call writes every entry it later reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU
// share the array and race.
static __device__ __align__(256) double g_noalloc_part[MSP_NOALLOC_MAX_VECTORS * kNaBlocks];

// Device address of g_noalloc_part, looked up once per device with that
// device current (in host code the symbol itself is only a host-side stand-in).
// The cached address belongs to the device's current context: after
// cudaDeviceReset the array may live elsewhere, so a process that resets a
// device must not call this entry point on it again.
constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double* g_na_ptr[kMaxDevices] = {nullptr};

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return msp::fail(MSP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return msp::fail(MSP_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e != cudaSuccess || !p)
      return msp::fail(MSP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return MSP_OK;
}

}  // namespace

extern "C" MSP_API int msp_multidot_noalloc(const double* V, int64_t ld, int nv, const double* w,
                                            int64_t n, double* out, void* stream) {
  if (nv < 1 || nv > MSP_NOALLOC_MAX_VECTORS)
    return msp::fail(MSP_ERR_INVALID, "msp_multidot_noalloc: nv must be in 1.." +
                                          std::to_string(MSP_NOALLOC_MAX_VECTORS));
  if (n < 0 || (nv > 1 && ld < n)) return msp::fail(MSP_ERR_INVALID, "msp_multidot_noalloc: bad n or ld");
  if (!V || !w || !out) return msp::fail(MSP_ERR_INVALID, "msp_multidot_noalloc: NULL pointer");
  double* part = nullptr;
  int rc = scratch_for_current_device(&part);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  msp::launch_multidot(V, ld, nv, w, n, part, out, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return msp::fail(MSP_ERR_CUDA, std::string("msp_multidot_noalloc: ") + cudaGetErrorString(e));
  return MSP_OK;
}
