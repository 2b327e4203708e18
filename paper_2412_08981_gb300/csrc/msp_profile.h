// Per-kernel-class launch accounting and CUDA-event timing.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "msp.h"

namespace msp {

enum {
  PK_ASSEMBLE = MSP_PK_ASSEMBLE, PK_EXTRACT = MSP_PK_EXTRACT, PK_LDLT_DIAG = MSP_PK_LDLT_DIAG,
  PK_LDLT_PANEL = MSP_PK_LDLT_PANEL, PK_LDLT_TRAIL = MSP_PK_LDLT_TRAIL, PK_RAS = MSP_PK_RAS,
  PK_RAS_COARSER = MSP_PK_RAS_COARSER, PK_COARSE = MSP_PK_COARSE, PK_SPMV = MSP_PK_SPMV,
  PK_TRANSFER = MSP_PK_TRANSFER, PK_VEC = MSP_PK_VEC, PK_LDLT_BLOCKS = MSP_PK_LDLT_BLOCKS,
  PK_COUNT = MSP_PK_COUNT
};

struct Profile {
  msp_kernel_profile c[PK_COUNT];
  uint32_t mask = 0;
  struct Pending {
    int k;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;

  Profile() { reset(); }
  void init(cudaStream_t) { reset(); }
  void reset() { std::memset(c, 0, sizeof(c)); }
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  // Folds the durations of completed timed launches into the counters.
  void harvest() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        c[p.k].ms += ms;
        c[p.k].timed += 1;
      } else {
        cudaGetLastError();
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void destroy() {
    harvest();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// Counts `nk` kernels of class k launched inside its lifetime; records
// events around them when the class is being timed.
struct ProfScope {
  Profile& P;
  int k, nk;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  double bytes = 0, flops = 0;
  ProfScope(Profile& p, int kk, cudaStream_t st, int nkern = 1) : P(p), k(kk), nk(nkern), s(st) {
    if (P.mask & (1u << k)) {
      a = P.get();
      if (a) cudaEventRecord(a, s);
    }
  }
  void account(double by, double fl) {
    bytes = by;
    flops = fl;
  }
  ~ProfScope() {
    P.c[k].launches += nk;
    P.c[k].bytes += bytes;
    P.c[k].flops += flops;
    if (a) {
      cudaEvent_t b = P.get();
      if (b) {
        cudaEventRecord(b, s);
        P.pending.push_back({k, a, b});
      } else {
        P.pool.push_back(a);
      }
    }
  }
};

}  // namespace msp
