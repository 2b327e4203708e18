// 5th-generation tensor-core (tcgen05) building blocks for sm_103a, and a
// self-check of them.
//
// The BF16 trailing updates of the subdomain factorisation are dense
// 128 x N x 64 products, C -= (L_ik D_k) L_jk^T (Section 2.2, Eq. 6, with the
// factors in symmetric form).  They run as tcgen05.mma of kind::f16 with BF16
// operands staged in shared memory (canonical K-major layout, no swizzle) and
// FP32 accumulators in tensor memory (TMEM), read back with tcgen05.ld.
//
// Canonical K-major layout without swizzle: the operand is cut into "core
// matrices" of 8 rows x 16 bytes (8 BF16 values of K), each stored as 128
// contiguous bytes (row r of the core matrix at byte 16 r).  Here core matrix
// (row group g, K chunk c) of a 64-wide K slab sits at byte g * 1024 + c * 128:
// the K-adjacent core matrices are 128 bytes apart (the descriptor's leading
// byte offset) and the row-adjacent ones 1024 bytes apart (its stride byte
// offset).  One MMA consumes K = 16, i.e. two K chunks, so step s starts at
// byte 256 s of the slab.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "msp.h"
#include "msp_tc.cuh"

namespace msp {
int fail(int code, const std::string& msg);

namespace {

constexpr int kM = 128, kN = 128, kK = 64;
constexpr uint32_t kSlack = 32768;  // operand buffer stride: room for any misread layout

// D (128 x 128, FP32, row-major) = A (128 x 64) B^T (B: 128 x 64), BF16 inputs.
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const __nv_bfloat16* __restrict__ A,
                                                        const __nv_bfloat16* __restrict__ B,
                                                        float* __restrict__ D, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sa = sm;
  unsigned char* sb = sm + kSlack;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kSlack);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * kSlack + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < kM * kK; e += blockDim.x) {
    const int r = e / kK, k = e % kK;
    const uint32_t off = tc::kmajor_offset(r, k);
    *reinterpret_cast<__nv_bfloat16*>(sa + off) = A[e];
    *reinterpret_cast<__nv_bfloat16*>(sb + off) = B[e];
  }
  tc::fence_async_smem();
  if (warp == 0) {
    tc::tmem_alloc(tslot, kN);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(kM, kN);
    for (int s = 0; s < kK / 16; ++s)
      tc::mma_bf16(taddr, tc::sdesc(sa + 256 * s), tc::sdesc(sb + 256 * s), idesc, s > 0);
    tc::commit(bar);
  }
  __syncwarp();
  int ok = tc::mbar_wait_bounded(bar, 0);
  if (!ok && lane == 0) atomicOr(status, 1);
  tc::fence_after();
  // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), all 128 columns
  for (int c0 = 0; c0 < kN; c0 += 16) {
    float v[16];
    tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    const int row = 32 * warp + lane;
#pragma unroll
    for (int i = 0; i < 16; ++i) D[row * kN + c0 + i] = v[i];
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kN);
}

}  // namespace
}  // namespace msp

extern "C" MSP_API int msp_tensor_selftest(int* mismatches) {
  using namespace msp;
  // integer-valued inputs: every product and partial sum is exact in FP32, so
  // the tensor-core result must equal the host's integer product bit for bit
  std::vector<__nv_bfloat16> ha(kM * kK), hb(kN * kK);
  std::vector<int> ia(kM * kK), ib(kN * kK);
  uint32_t x = 12345u;
  auto next = [&]() {
    x = x * 1664525u + 1013904223u;
    return (int)((x >> 24) % 17) - 8;
  };
  for (int e = 0; e < kM * kK; ++e) {
    ia[e] = next();
    ha[e] = __float2bfloat16((float)ia[e]);
  }
  for (int e = 0; e < kN * kK; ++e) {
    ib[e] = next();
    hb[e] = __float2bfloat16((float)ib[e]);
  }
  __nv_bfloat16 *da = nullptr, *db = nullptr;
  float* dd = nullptr;
  int* dst = nullptr;
  auto cleanup = [&]() {
    cudaFree(da);
    cudaFree(db);
    cudaFree(dd);
    cudaFree(dst);
  };
  if (cudaMalloc(&da, ha.size() * 2) != cudaSuccess || cudaMalloc(&db, hb.size() * 2) != cudaSuccess ||
      cudaMalloc(&dd, (size_t)kM * kN * 4) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(MSP_ERR_OOM, "msp_tensor_selftest: device allocation failed");
  }
  cudaMemcpy(da, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(db, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice);
  cudaMemset(dd, 0xFF, (size_t)kM * kN * 4);
  cudaMemset(dst, 0, sizeof(int));
  const int smem = 2 * kSlack + 64;
  cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_tc_selftest<<<1, 128, smem>>>(da, db, dd, dst);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cleanup();
    return fail(MSP_ERR_CUDA, std::string("msp_tensor_selftest: ") + cudaGetErrorString(e));
  }
  std::vector<float> hd((size_t)kM * kN);
  int hst = 0;
  cudaMemcpy(hd.data(), dd, hd.size() * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hst, dst, sizeof(int), cudaMemcpyDeviceToHost);
  cleanup();
  if (hst) return fail(MSP_ERR_TIMEOUT, "msp_tensor_selftest: the MMA completion wait expired");
  int bad = 0, first = -1;
  for (int i = 0; i < kM; ++i)
    for (int j = 0; j < kN; ++j) {
      int s = 0;
      for (int k = 0; k < kK; ++k) s += ia[i * kK + k] * ib[j * kK + k];
      if (hd[(size_t)i * kN + j] != (float)s) {
        if (first < 0) first = i * kN + j;
        ++bad;
      }
    }
  if (mismatches) *mismatches = bad;
  if (bad)
    return fail(MSP_ERR_INTERNAL, "msp_tensor_selftest: " + std::to_string(bad) +
                                      " of 16384 products differ (first at row " +
                                      std::to_string(first / kN) + ", column " +
                                      std::to_string(first % kN) + ")");
  return MSP_OK;
}
