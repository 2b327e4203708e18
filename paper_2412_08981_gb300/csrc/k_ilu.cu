// ILU(p) subdomain solver kernels (the incomplete factorisation of Section
// 4.4 in place of the exact block LU), in FP64 or FP32 (T: factor storage
// and arithmetic of the factorisation and of the sweeps; the vectors the
// sweeps read and write stay FP64).
//
// The factor of block p is kept in symmetric form, L (unit lower, sparse) and
// D, with U = D L^T; its pattern is the level-of-fill pattern of ILU(p) (host
// set-up).  Both the factorisation and the triangular sweeps run one CTA per
// block and walk its rows by dependency level (set-up): the rows of a level
// depend only on rows of earlier levels, so each level is one parallel step
// (one warp per row) followed by a CTA barrier.  A block's vectors live in
// shared memory; the factor streams from global memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "msp_kernels.h"

namespace msp {
namespace {

constexpr int kIluWarps = 4;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// zero or non-finite pivot
template <typename T>
__device__ __forceinline__ bool bad_pivot(T d) {
  const double dd = (double)d;
  return dd == 0.0 || !(fabs(dd) < 1e300);
}

// Up-looking incomplete L D L^T of block p (Section 4.4), rows of at most 32
// strictly-lower entries: lane j of the row's warp owns entry (i, k_j).  With
// u_j = l_{i k_j} d_{k_j} (the not yet divided entry), the row satisfies
//   u_j = a_{i k_j} - sum_{j' < j} u_{j'} l_{k_j k_j'}    over the pattern,
// so entry j is final once the earlier ones are, and step j broadcasts u_j and
// every lane j'' > j with (k_j'', k_j) in the pattern subtracts u_j times that
// entry of L (a register update: no reduction per step).  Then
// l_{i k_j} = u_j / d_{k_j} and d_i = a_ii - sum_j l_{i k_j} u_j.  The L
// entries a lane needs are gathered once per row into S[j][lane] through
// pos (column -> lane of this row, -1 elsewhere).  Same fac layout as the
// warp-per-dot form below.  smem per warp: 32 x 32 T + max_n int16.
template <typename T>
__global__ void __launch_bounds__(32 * kIluWarps) k_ilu_factor_lanes(
    T* __restrict__ fac, int64_t nnz, int64_t rows, const int32_t* __restrict__ sub_ptr,
    const int64_t* __restrict__ lptr, const int32_t* __restrict__ lcol,
    const int32_t* __restrict__ fwd_rows, const int32_t* __restrict__ fwd_lvl,
    const int32_t* __restrict__ fwd_loff, int max_n, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char sm_ilu_raw[];
  T* sm_ilu = reinterpret_cast<T*>(sm_ilu_raw);
  const int p = blockIdx.x;
  const int R0 = sub_ptr[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pos_stride = (max_n + 3) & ~3;
  T* S = sm_ilu + warp * 1024;
  int16_t* pos_all = reinterpret_cast<int16_t*>(sm_ilu + kIluWarps * 1024);
  int16_t* pos = pos_all + warp * pos_stride;
  T* L = fac;
  T* D = fac + nnz;
  T* Dinv = D + rows;
  for (int e = threadIdx.x; e < kIluWarps * pos_stride; e += blockDim.x) pos_all[e] = -1;
  __syncthreads();
  for (int q = fwd_loff[p]; q + 1 < fwd_loff[p + 1]; ++q) {
    const int r0 = fwd_lvl[q], r1 = fwd_lvl[q + 1];
    for (int rr = r0 + warp; rr < r1; rr += kIluWarps) {
      const int i = fwd_rows[rr];
      const int64_t b = lptr[R0 + i];
      const int len = (int)(lptr[R0 + i + 1] - b);  // <= 32 (host check)
      int k = 0;
      T u = T(0), dinv = T(0);
      if (lane < len) {
        k = lcol[b + lane];
        u = L[b + lane];
        dinv = Dinv[R0 + k];
        pos[k] = (int16_t)lane;
      }
      __syncwarp();
      uint32_t mask = 0;
      if (lane < len) {
        const int64_t kb = lptr[R0 + k], ke = lptr[R0 + k + 1];
        for (int64_t t = kb; t < ke; ++t) {
          const int jj = pos[lcol[t]];
          if (jj >= 0) {
            S[jj * 32 + lane] = L[t];
            mask |= 1u << jj;
          }
        }
      }
      __syncwarp();
      for (int j = 0; j < len; ++j) {
        const T uj = __shfl_sync(0xffffffffu, u, j);
        if ((mask >> j) & 1u) u = fma_t(-uj, S[j * 32 + lane], u);
      }
      const T l = u * dinv;
      const T s = warp_sum<T>(lane < len ? l * u : T(0));
      if (lane < len) {
        L[b + lane] = l;
        pos[k] = -1;
      }
      if (lane == 0) {
        const T di = D[R0 + i] - s;
        D[R0 + i] = di;
        Dinv[R0 + i] = T(1) / di;
        if (bad_pivot(di)) atomicOr(info, 1);
      }
      __syncwarp();
    }
    __syncthreads();  // the level's rows (L, D, 1/D) are final for the next levels
  }
}

// Up-looking incomplete L D L^T of block p, any row length: for row i, in
// ascending k over its pattern, l_ik = (a_ik - sum_{m in P(k)} l_km d_m l_im) / d_k (entries of row
// i outside its pattern are zero, which drops the fill of level > p), then
// d_i = a_ii - sum_m l_im^2 d_m.  fac = [L (nnz) | D (rows) | 1/D (rows)],
// holding A_p's lower triangle on entry (extraction).  Each warp keeps its
// row dense in shared memory.  smem: (kIluWarps + 1) * max_n T.
template <typename T>
__global__ void __launch_bounds__(32 * kIluWarps) k_ilu_factor(
    T* __restrict__ fac, int64_t nnz, int64_t rows, const int32_t* __restrict__ sub_ptr,
    const int64_t* __restrict__ lptr, const int32_t* __restrict__ lcol,
    const int32_t* __restrict__ fwd_rows, const int32_t* __restrict__ fwd_lvl,
    const int32_t* __restrict__ fwd_loff, int max_n, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char sm_ilu_raw[];
  T* sm_ilu = reinterpret_cast<T*>(sm_ilu_raw);
  const int p = blockIdx.x;
  const int R0 = sub_ptr[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* d_s = sm_ilu;                    // [max_n] d of finished rows
  T* w = d_s + max_n + warp * max_n;  // [max_n] this warp's current row
  T* L = fac;
  T* D = fac + nnz;
  T* Dinv = D + rows;
  for (int e = threadIdx.x; e < kIluWarps * max_n; e += blockDim.x) sm_ilu[max_n + e] = T(0);
  __syncthreads();
  for (int q = fwd_loff[p]; q + 1 < fwd_loff[p + 1]; ++q) {  // level q: rows fwd_lvl[q] .. fwd_lvl[q+1]
    const int r0 = fwd_lvl[q], r1 = fwd_lvl[q + 1];
    for (int rr = r0 + warp; rr < r1; rr += kIluWarps) {
      const int i = fwd_rows[rr];
      const int64_t b = lptr[R0 + i], e = lptr[R0 + i + 1];
      for (int64_t t = b + lane; t < e; t += 32) w[lcol[t]] = L[t];
      __syncwarp();
      for (int64_t t = b; t < e; ++t) {
        const int k = lcol[t];
        const int64_t kb = lptr[R0 + k], ke = lptr[R0 + k + 1];
        T s = T(0);
        for (int64_t u = kb + lane; u < ke; u += 32) {
          const int m = lcol[u];
          s = fma_t(L[u] * d_s[m], w[m], s);
        }
        s = warp_sum<T>(s);
        const T lik = (w[k] - s) * Dinv[R0 + k];
        __syncwarp();
        if (lane == 0) w[k] = lik;
        __syncwarp();
      }
      T s = T(0);
      for (int64_t t = b + lane; t < e; t += 32) {
        const int m = lcol[t];
        s = fma_t(w[m] * w[m], d_s[m], s);
      }
      s = warp_sum<T>(s);
      const T di = D[R0 + i] - s;
      for (int64_t t = b + lane; t < e; t += 32) {
        const int m = lcol[t];
        L[t] = w[m];
        w[m] = T(0);
      }
      if (lane == 0) {
        D[R0 + i] = di;
        Dinv[R0 + i] = T(1) / di;
        d_s[i] = di;
        if (bad_pivot(di)) atomicOr(info, 1);
      }
      __syncwarp();
    }
    __syncthreads();  // the level's rows (L, D, d_s) are final for the next levels
  }
}

// One triangular sweep of a block, level by level: y_i -= sum_e Lx[e] y[src[e]]
// over the entries e of row i (the rows of a level are independent).  A
// group of kGroup lanes takes one row: lane g forms the products of entries
// g, g + kGroup, ... with FMAs and the group adds its partial sums by a fixed
// shuffle tree (deterministic), so a level costs a few dependent
// floating-point operations instead of one per entry.  A level's entries are contiguous
// (level-major lists): they are copied into a ring of kRing shared-memory
// slots with cp.async kRing - 1 levels ahead, so the global-memory latency is
// off the level-to-level critical path (entries past a slot's kRingEnt come
// straight from global memory).  One barrier per level.
constexpr int kSweepThreads = 256, kGroup = 8, kGroups = kSweepThreads / kGroup;
constexpr int kRing = 4, kRingEnt = 384, kEntUnroll = 4;

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_val(double* dst, const double* src) { cp_async8(dst, src); }
__device__ __forceinline__ void cp_async_val(float* dst, const float* src) { cp_async4(dst, src); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
  for (int o = 1; o < kGroup; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Issues (and commits, possibly empty) the copies of level q into its slot.
template <typename T>
__device__ __forceinline__ void sweep_fetch(int q, int nlev, const int* lvl_s, const int* eptr_s,
                                            const T* __restrict__ Lx, const int32_t* __restrict__ src,
                                            T* ring_v, int* ring_s) {
  if (q < nlev) {
    const int e0 = eptr_s[lvl_s[q]], ne = min(eptr_s[lvl_s[q + 1]] - e0, kRingEnt);
    T* sv = ring_v + (q % kRing) * kRingEnt;
    int* ss = ring_s + (q % kRing) * kRingEnt;
    for (int j = threadIdx.x; j < ne; j += kSweepThreads) {
      cp_async_val(sv + j, Lx + e0 + j);
      cp_async4(ss + j, src + e0 + j);
    }
  }
  cp_async_commit();
}

// Sweep over levels [0, nlev) of the block; Lx and src start at the block's
// first entry, lvl_s / rows_s / eptr_s are relative to the block.
template <typename T>
__device__ void ilu_sweep(T* __restrict__ y, const T* __restrict__ Lx, const int32_t* __restrict__ src,
                          const int* lvl_s, const int* rows_s, const int* eptr_s, int nlev, T* ring_v,
                          int* ring_s) {
  const int lane = threadIdx.x & 31, gl = threadIdx.x % kGroup;
  // the row groups of a pass start at a block-dependent warp, so that the
  // FP64 work of the blocks sharing an SM spreads over its four schedulers
  const int quad = ((threadIdx.x >> 5) - (int)blockIdx.x) & (kSweepThreads / 32 - 1);
#pragma unroll
  for (int q = 0; q < kRing - 1; ++q) sweep_fetch(q, nlev, lvl_s, eptr_s, Lx, src, ring_v, ring_s);
  for (int q = 0; q < nlev; ++q) {
    cp_async_wait<kRing - 2>();  // this thread's copies of level q have landed
    __syncthreads();             // everyone's, and the y of the previous levels
    const int r0 = lvl_s[q], r1 = lvl_s[q + 1], e0 = eptr_s[r0];
    const T* sv = ring_v + (q % kRing) * kRingEnt;
    const int* ss = ring_s + (q % kRing) * kRingEnt;
    for (int base = r0; base < r1; base += kGroups) {
      if (base + quad * (32 / kGroup) >= r1) break;  // no row for this warp (warp-uniform)
      const int rr = base + quad * (32 / kGroup) + (lane / kGroup);
      T acc = T(0);
      int row = 0;
      if (rr < r1) {
        row = rows_s[rr];
        const int jb = eptr_s[rr] - e0 + gl, je = eptr_s[rr + 1] - e0;
        if (je <= kRingEnt) {
          // the first kEntUnroll entries of the lane at once (loads issued together)
          T v[kEntUnroll];
          int c[kEntUnroll];
#pragma unroll
          for (int k = 0; k < kEntUnroll; ++k) {
            const int j = jb + k * kGroup;
            v[k] = T(0);
            c[k] = 0;
            if (j < je) {
              v[k] = sv[j];
              c[k] = ss[j];
            }
          }
#pragma unroll
          for (int k = 0; k < kEntUnroll; ++k) acc = fma_t(v[k], y[c[k]], acc);
          for (int j = jb + kEntUnroll * kGroup; j < je; j += kGroup) acc = fma_t(sv[j], y[ss[j]], acc);
        } else {
          for (int j = jb; j < je; j += kGroup)
            acc = j < kRingEnt ? fma_t(sv[j], y[ss[j]], acc) : fma_t(Lx[e0 + j], y[src[e0 + j]], acc);
        }
      }
      acc = group_sum<T>(acc);
      if (gl == 0 && rr < r1) y[row] -= acc;
    }
    sweep_fetch(q + kRing - 1, nlev, lvl_s, eptr_s, Lx, src, ring_v, ring_s);  // into the slot of q - 1
  }
  cp_async_wait<0>();
  __syncthreads();
}

// Copies the sweep's schedule of block p into shared memory (relative to the
// block): level bounds, rows in level order, entry offsets.  Returns the
// level count and the block's first entry.
__device__ int sweep_schedule(int p, const int32_t* __restrict__ loff, const int32_t* __restrict__ lvl,
                              const int32_t* __restrict__ rows, const int64_t* __restrict__ eptr, int* lvl_s,
                              int* rows_s, int* eptr_s, int64_t* e_base) {
  const int q0 = loff[p], nlev = loff[p + 1] - 1 - q0;
  const int rb = lvl[q0], nr = lvl[q0 + nlev] - rb;
  const int64_t eb = eptr[rb];
  for (int q = threadIdx.x; q <= nlev; q += blockDim.x) lvl_s[q] = lvl[q0 + q] - rb;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) rows_s[r] = rows[rb + r];
  for (int r = threadIdx.x; r <= nr; r += blockDim.x) eptr_s[r] = (int)(eptr[rb + r] - eb);
  *e_base = eb;
  return nlev;
}

// y = (L D L^T)^{-1} t[dofs] of block p and the owned scatter into z (RAS,
// Eq. 7): the forward sweep over the rows of L, y /= D, the backward sweep
// over the columns of L (L^T), in T.  smem: max_n T + 3 max_n + 2 ints, and
// the ring of kRing x kRingEnt entries.
template <typename T>
__global__ void __launch_bounds__(kSweepThreads) k_ilu_solve(
    const T* __restrict__ fac, int64_t nnz, int64_t rows, const int32_t* __restrict__ sub_ptr,
    const int32_t* __restrict__ dofs, const uint8_t* __restrict__ own,
    const int64_t* __restrict__ fe_ptr, const int32_t* __restrict__ fe_src,
    const int64_t* __restrict__ be_ptr, const int32_t* __restrict__ be_src,
    const int32_t* __restrict__ fwd_rows, const int32_t* __restrict__ fwd_lvl,
    const int32_t* __restrict__ fwd_loff, const int32_t* __restrict__ bwd_rows,
    const int32_t* __restrict__ bwd_lvl, const int32_t* __restrict__ bwd_loff, int max_n,
    const int32_t* __restrict__ dir_list, int ndir, const double* __restrict__ t,
    double* __restrict__ z, int add) {
  extern __shared__ __align__(16) unsigned char sm_ilu_raw[];
  const int p = blockIdx.x;
  const int R0 = sub_ptr[p], n = sub_ptr[p + 1] - R0;
  const T* Dinv = fac + nnz + rows;
  const T* Lf = fac + nnz + 2 * rows;  // forward entries, level-major
  const T* Lb = Lf + nnz;              // backward entries, level-major
  T* y = reinterpret_cast<T*>(sm_ilu_raw);
  int* rows_s = reinterpret_cast<int*>(y + ((max_n + 1) & ~1));  // 8-byte aligned
  int* eptr_s = rows_s + max_n;
  int* lvl_s = eptr_s + max_n + 1;
  T* ring_v = reinterpret_cast<T*>(rows_s + ((3 * max_n + 3) & ~1));  // 8-byte aligned
  int* ring_s = reinterpret_cast<int*>(ring_v + kRing * kRingEnt);
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndir; d += gridDim.x * blockDim.x) {
    const int g = dir_list[d];
    z[g] = add ? z[g] + t[g] : t[g];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (T)t[dofs[R0 + i]];
  int64_t eb = 0;
  int nlev = sweep_schedule(p, fwd_loff, fwd_lvl, fwd_rows, fe_ptr, lvl_s, rows_s, eptr_s, &eb);
  __syncthreads();
  ilu_sweep(y, Lf + eb, fe_src + eb, lvl_s, rows_s, eptr_s, nlev, ring_v, ring_s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= Dinv[R0 + i];
  nlev = sweep_schedule(p, bwd_loff, bwd_lvl, bwd_rows, be_ptr, lvl_s, rows_s, eptr_s, &eb);
  __syncthreads();
  ilu_sweep(y, Lb + eb, be_src + eb, lvl_s, rows_s, eptr_s, nlev, ring_v, ring_s);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (own[R0 + i]) {
      const int g = dofs[R0 + i];
      z[g] = add ? z[g] + (double)y[i] : (double)y[i];
    }
}

// Level-major copies of the factor for the sweeps: Lf[e] = L[fe_slot[e]],
// Lb[e] = L[be_slot[e]].
template <typename T>
__global__ void k_ilu_gather(T* __restrict__ fac, int64_t nnz, int64_t rows,
                             const int64_t* __restrict__ fe_slot, const int64_t* __restrict__ be_slot) {
  const T* L = fac;
  T* Lf = fac + nnz + 2 * rows;
  T* Lb = Lf + nnz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    Lf[e] = L[fe_slot[e]];
    Lb[e] = L[be_slot[e]];
  }
}

template <typename T>
__global__ void k_ilu_zero(T* __restrict__ p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = T(0);
}

// A's values (FP64) into the factor storage, rounded to nearest when T is FP32
template <typename T>
__global__ void k_ilu_scatter(const int64_t* __restrict__ pos, const int32_t* __restrict__ nz,
                              const double* __restrict__ val, int64_t nent, T* __restrict__ fac) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nent) fac[pos[e]] = (T)val[nz[e]];
}

int nblocks(int64_t n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

size_t ilu_factor_smem(int max_n, int max_row, size_t es) {
  if (max_row <= 32) return (size_t)kIluWarps * (1024 * es + ((max_n + 3) & ~3) * sizeof(int16_t));
  return (size_t)(kIluWarps + 1) * max_n * es;
}
size_t ilu_solve_smem(int max_n, size_t es) {
  // y (padded to 8 bytes); rows, entry offsets and level bounds (3 max_n + 2
  // ints, padded to 8 bytes); ring values and columns
  return (size_t)((max_n + 1) & ~1) * es + (size_t)((3 * max_n + 3) & ~1) * sizeof(int) +
         (size_t)kRing * kRingEnt * (es + sizeof(int));
}

template <typename T>
void launch_ilu_extract(const int64_t* pos, const int32_t* nz, int64_t nent, const double* val, int64_t total,
                        T* fac, cudaStream_t s) {
  if (total > 0) k_ilu_zero<T><<<std::min<int64_t>(nblocks(total, 256), 1 << 16), 256, 0, s>>>(fac, total);
  if (nent > 0) k_ilu_scatter<T><<<nblocks(nent, 256), 256, 0, s>>>(pos, nz, val, nent, fac);
}

template <typename T>
void launch_ilu_factor(T* fac, int64_t nnz, int64_t rows, int nsub, const int32_t* sub_ptr,
                       const int64_t* lptr, const int32_t* lcol, const int32_t* fwd_rows,
                       const int32_t* fwd_lvl, const int32_t* fwd_loff, int max_n, int max_row, int* info,
                       cudaStream_t s) {
  if (nsub <= 0) return;
  const size_t smem = ilu_factor_smem(max_n, max_row, sizeof(T));
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_ilu_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ilu_factor_lanes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (max_row <= 32)
    k_ilu_factor_lanes<T><<<nsub, 32 * kIluWarps, smem, s>>>(fac, nnz, rows, sub_ptr, lptr, lcol, fwd_rows,
                                                            fwd_lvl, fwd_loff, max_n, info);
  else
    k_ilu_factor<T><<<nsub, 32 * kIluWarps, smem, s>>>(fac, nnz, rows, sub_ptr, lptr, lcol, fwd_rows, fwd_lvl,
                                                        fwd_loff, max_n, info);
}

template <typename T>
void launch_ilu_gather(T* fac, int64_t nnz, int64_t rows, const int64_t* fe_slot, const int64_t* be_slot,
                       cudaStream_t s) {
  if (nnz > 0)
    k_ilu_gather<T><<<std::min<int64_t>(nblocks(nnz, 256), 1 << 16), 256, 0, s>>>(fac, nnz, rows, fe_slot, be_slot);
}

template <typename T>
void launch_ilu_solve(const T* fac, int64_t nnz, int64_t rows, int nsub, const int32_t* sub_ptr,
                      const int32_t* dofs, const uint8_t* own, const int64_t* fe_ptr, const int32_t* fe_src,
                      const int64_t* be_ptr, const int32_t* be_src, const int32_t* fwd_rows,
                      const int32_t* fwd_lvl, const int32_t* fwd_loff, const int32_t* bwd_rows,
                      const int32_t* bwd_lvl, const int32_t* bwd_loff, int max_n,
                      const int32_t* dir_list, int ndir, const double* t, double* z, int add, cudaStream_t s) {
  if (nsub <= 0) return;
  const size_t smem = ilu_solve_smem(max_n, sizeof(T));
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_ilu_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  k_ilu_solve<T><<<nsub, kSweepThreads, smem, s>>>(fac, nnz, rows, sub_ptr, dofs, own, fe_ptr, fe_src, be_ptr,
                                                    be_src, fwd_rows, fwd_lvl, fwd_loff, bwd_rows, bwd_lvl, bwd_loff,
                                                    max_n, dir_list, ndir, t, z, add);
}

#define MSP_ILU_INST(T)                                                                                          \
  template void launch_ilu_extract<T>(const int64_t*, const int32_t*, int64_t, const double*, int64_t, T*,      \
                                      cudaStream_t);                                                             \
  template void launch_ilu_factor<T>(T*, int64_t, int64_t, int, const int32_t*, const int64_t*, const int32_t*, \
                                     const int32_t*, const int32_t*, const int32_t*, int, int, int*,             \
                                     cudaStream_t);                                                              \
  template void launch_ilu_gather<T>(T*, int64_t, int64_t, const int64_t*, const int64_t*, cudaStream_t);       \
  template void launch_ilu_solve<T>(const T*, int64_t, int64_t, int, const int32_t*, const int32_t*,            \
                                    const uint8_t*, const int64_t*, const int32_t*, const int64_t*,              \
                                    const int32_t*, const int32_t*, const int32_t*, const int32_t*,              \
                                    const int32_t*, const int32_t*, const int32_t*, int, const int32_t*, int,    \
                                    const double*, double*, int, cudaStream_t);
MSP_ILU_INST(double)
MSP_ILU_INST(float)
#undef MSP_ILU_INST

}  // namespace msp
