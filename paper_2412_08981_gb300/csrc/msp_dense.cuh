// Definitions shared by the dense-factor kernels (k_dense.cu) and the
// triangular-solve kernels (k_ras.cu): the factor tile, the arithmetic type
// of each storage type, and the device limits the launchers size against.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace msp {
namespace {

constexpr int T64 = 64;
constexpr int TE = T64 * T64;

template <typename T> struct Acc { using type = double; };
template <> struct Acc<float> { using type = float; };
template <> struct Acc<__nv_bfloat16> { using type = float; };  // BF16 storage, FP32 arithmetic

struct DevLimits {
  int nsm = 0, smem = 0;
};
DevLimits& limits() {
  static DevLimits L = [] {
    DevLimits d;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    d.smem -= 1024;  // static shared memory and slack
    return d;
  }();
  return L;
}

}  // namespace
}  // namespace msp
