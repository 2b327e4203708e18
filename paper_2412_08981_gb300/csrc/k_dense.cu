// Dense subdomain kernels of the msp library (Section 2.2, Eq. 6-7):
//   * extraction of the blocks J^delta_p = R J R^T into tiled storage,
//   * batched, blocked, right-looking unpivoted LU of every block in its
//     symmetric form J_p = L D L^T (U = D L^T; the blocks are SPD, so no
//     pivoting is needed and half of the LU work is skipped),
//   (the RAS application that uses these factors is in k_ras.cu).
//
// Tile layout (see msp.h): 64 x 64 row-major tiles over the tile envelope of
// each block; tile row I holds the tiles (I, F_I) .. (I, I) contiguously.  The
// blocks are banded (DoFs in ascending global order), fill stays inside the
// envelope, so the tiles left of F_I are never stored, read or updated: the
// arithmetic on every stored entry is that of the full dense factorisation.
// Diagonal tiles hold L below the diagonal, D on it and X^T above it, X =
// inverse of the unit lower diagonal block of L; the triangular solves use X,
// so every step is a dense product and the only sequential dependency is
// between tile rows.
//
// On GB300 FP64 runs on the SIMT pipe at ~1/64 of the FP32 rate (there is no
// fast FP64 tensor path), so the FP64 kernels are ALU-bound: their design
// keeps the FMA pipe fed from shared memory and avoids idle lanes.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "msp_dense.cuh"
#include "msp_kernels.h"
#include "msp_tc.cuh"

namespace msp {
namespace {


// 1/d of a pivot, correctly rounded.  Every reciprocal sits on the
// sequential pivot chain of a factorisation.  On GB300 the dependent latency
// of __drcp_rn (about 440 cycles for one warp, against 63 for one FP64 FMA)
// is shorter than that of Newton steps from a single-precision seed, whose
// conversions cost more than the steps (about 640 cycles), and it is exact
// over the whole double range (a test on meshes scaled by 2^+-133 puts
// pivots near 1e40 and 1e-40).
__device__ inline double pivot_rcp(double d) { return __drcp_rn(d); }
__device__ inline float pivot_rcp(float d) { return 1.0f / d; }

// element offset of tile (I, J), J >= F_I, of subdomain p
__device__ inline int64_t tile_at(const EnvDev& E, int p, int I, int J) {
  const int rb = E.trow[p] + I;
  return E.fac_off[p] + (int64_t)(E.toff[rb] + (J - E.first[rb])) * TE;
}

// ------------------------------------------------------------ extraction
template <typename T>
__global__ void k_scatter(const int64_t* __restrict__ pos, const int32_t* __restrict__ nz,
                          const double* __restrict__ val, int64_t nent, T* __restrict__ fac) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  int q = nz[e];
  fac[pos[e]] = (T)(q >= 0 ? val[q] : 1.0);
}

// Reads N elements of T (N a multiple of 16 bytes' worth; src 16-byte
// aligned) with 16-byte loads, up to four of a thread's loads in flight
// together, and hands each element to f(e, value), e = 0 .. N-1.  The tile
// loops of the factorisation otherwise wait out one L2 round trip per
// element in turn.  Every thread of the 256-thread block takes part.  Plain
// (coherent) loads: the factors are rewritten within the same launch.
template <typename T, int N, typename F>
__device__ __forceinline__ void read_elems(const T* src, F&& f) {
  constexpr int V = 16 / sizeof(T);
  constexpr int NVEC = N / V;
  constexpr int PER = (NVEC + 255) / 256;
  constexpr int R = PER < 4 ? PER : 4;
  static_assert(N % V == 0, "whole 16-byte vectors");
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const Vec* sv = reinterpret_cast<const Vec*>(src);
#pragma unroll
  for (int r0 = 0; r0 < PER; r0 += R) {
    Vec v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = threadIdx.x + 256 * (r0 + q);
      if (NVEC % 256 == 0 || i < NVEC) v[q] = sv[i];
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = threadIdx.x + 256 * (r0 + q);
      if (NVEC % 256 == 0 || i < NVEC) {
        const T* x = reinterpret_cast<const T*>(&v[q]);
#pragma unroll
        for (int k = 0; k < V; ++k) f(i * V + k, x[k]);
      }
    }
  }
}

// Programmatic dependent launch between the tile-step kernels of a chain
// (launched with the programmatic-serialisation attribute on one stream):
// a kernel lets its successor launch at once (step_release) and waits for
// its predecessor's completion and memory before its first read
// (step_acquire; a no-op without such a predecessor), so that a launch's
// set-up overlaps the previous step instead of following it.
__device__ __forceinline__ void step_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void step_acquire() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------- diagonal tile LDL^T
// Factors one diagonal tile in shared memory, computing in the factor's
// precision: unblocked right-looking elimination of the lower triangle with
// the inverse of the unit lower factor built in the same sweep.  Step c
// (one barrier pair):
//   * l_r = A_rc / d_c for the rows r > c;
//   * A_rs -= l_r A_sc for c < s <= r (the Schur complement, W = L D), and
//   * X_rj -= l_r X_cj for r > c, j <= c (X_cc = 1): the elimination that
//     turns L into I turns I into X = L^{-1} (X_c is final at step c, since
//     later steps only change rows below c).
// All entries of both updates are spread evenly over the threads, one FMA
// each; on GB300 FP64 issues one warp instruction per 16 SM cycles, so the
// work must fill every lane of every warp.  Then L = W D^{-1}.  Layout on
// exit: L strictly below the diagonal, D on it, X^T strictly above it
// (X_ij at A[j][i]).  smem: (64*65 + 128) elements of AT.
constexpr int kDiagThreads = 256;  // every kernel that factors a diagonal tile

template <typename T, typename AT>
__device__ void diag_tile(T* __restrict__ tile, AT* __restrict__ A, int* __restrict__ info) {
  AT* lcol = A + 64 * 65;  // [64] the scaled column of the current step
  AT* dinv = lcol + 64;    // [64] 1/d_c, formed once each, by the thread finishing d_c
  const int tid = threadIdx.x;
  __syncthreads();  // the shared buffer may still be read by a previous phase
  read_elems<T, TE>(tile, [&](int e, T v) {
    const int r = e >> 6, c = e & 63;
    A[r * 65 + c] = (c <= r) ? (AT)v : AT(0);  // X starts as the identity (zeros above)
  });
  __syncthreads();
  if (tid == 0) dinv[0] = pivot_rcp(A[0]);
  __syncthreads();
  for (int c = 0; c < T64 - 1; ++c) {
    if (tid > c && tid < T64) lcol[tid] = A[tid * 65 + c] * dinv[c];
    __syncthreads();
    const int m = T64 - 1 - c;            // trailing size
    const int nA = m * (m + 1) / 2;       // Schur complement entries
    const int nX = m * (c + 1);           // inverse entries X_rj, r > c, j <= c
    const float inv_w = 1.0f / (float)(c + 1);
    for (int e = tid; e < nA + nX; e += blockDim.x) {
      if (e < nA) {
        int rr = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
        rr += ((rr + 1) * (rr + 2) / 2 <= e);
        rr -= (rr * (rr + 1) / 2 > e);
        const int r = c + 1 + rr, s2 = c + 1 + (e - rr * (rr + 1) / 2);
        const AT v = fma(-lcol[r], A[s2 * 65 + c], A[r * 65 + s2]);
        A[r * 65 + s2] = v;
        if (e == 0) dinv[c + 1] = pivot_rcp(v);  // entry (c+1, c+1): the next pivot is final
      } else {
        const int x = e - nA;  // x = rr (c+1) + j
        int rr = (int)((float)x * inv_w);
        rr += ((rr + 1) * (c + 1) <= x);
        rr -= (rr * (c + 1) > x);
        const int j = x - rr * (c + 1), r = c + 1 + rr;
        const AT xcj = (j == c) ? AT(1) : A[j * 65 + c];
        A[j * 65 + r] = fma(-lcol[r], xcj, A[j * 65 + r]);
      }
    }
    __syncthreads();
  }
  if (tid < T64) {
    const AT d = A[tid * 65 + tid];
    if (!(d > AT(0)) || !(d < AT(1e300))) atomicOr(info, 1);
  }
  for (int e = tid; e < TE; e += blockDim.x) {  // L = W D^{-1}
    int r = e >> 6, c = e & 63;
    if (c < r) A[r * 65 + c] *= dinv[c];
  }
  __syncthreads();
  for (int e = tid; e < TE; e += blockDim.x) tile[e] = (T)A[(e >> 6) * 65 + (e & 63)];
}

// The off-diagonal 16 x 16 blocks of X = L^{-1} of a 64 x 64 diagonal tile in
// shared memory (L strictly below the diagonal, the diagonal blocks X_KK^T
// above it), block row by block row: X_IJ = -X_II sum_{J <= K < I} L_IK X_KJ,
// as T_ij = L_ij + sum_{j < m < i0} L_im X_mj, then
// X_ij = -(T_ij + sum_{i0 <= m < i} X_im T_mj).  X_ij is stored at A[j][i].
// Tb: [16][49] elements.  Every thread of the block takes part.
template <typename AT>
__device__ void x_offdiag_blocks(AT* __restrict__ A, AT* __restrict__ Tb) {
  constexpr int NB = 16;
  const int tid = threadIdx.x;
  for (int I = 1; I < 4; ++I) {
    const int i0 = I * NB;
    for (int e = tid; e < NB * i0; e += blockDim.x) {
      const int i = i0 + e / i0, j = e % i0;
      AT v = A[i * 65 + j], v2 = 0;
      int mm = j + 1;
      for (; mm + 1 < i0; mm += 2) {
        v = fma(A[i * 65 + mm], A[j * 65 + mm], v);
        v2 = fma(A[i * 65 + mm + 1], A[j * 65 + mm + 1], v2);
      }
      if (mm < i0) v = fma(A[i * 65 + mm], A[j * 65 + mm], v);
      Tb[(i - i0) * 49 + j] = v + v2;
    }
    __syncthreads();
    for (int e = tid; e < NB * i0; e += blockDim.x) {
      const int i = i0 + e / i0, j = e % i0;
      AT v = Tb[(i - i0) * 49 + j];
      for (int mm = i0; mm < i; ++mm) v = fma(A[mm * 65 + i], Tb[(mm - i0) * 49 + j], v);
      A[j * 65 + i] = -v;
    }
    __syncthreads();
  }
}

// Blocked form for a lone CTA (the tile steps of the coarsest block, whose
// diagonal tiles form the critical path): four 16-column blocks K, each
//   (a) its 16 x 16 diagonal block as above (one entry per thread per step),
//       with the inverse X_KK built in the same sweep.  A step reads column
//       c and writes only columns > c, so one barrier per column suffices:
//       every thread forms its own l_rc = A_rc / d_c (the same bits as a
//       shared scaled column).  The step's critical path is the next pivot
//       and its reciprocal; on GB300 an FP64 warp instruction holds its SM
//       sub-partition's FP64 unit for ~64 cycles, so the pivot has a warp to
//       itself (warp 7, whose sub-partition no other entry of (a) uses:
//       the entries go to warps 0-2 and 4-5);
//   (b) the panel W_rK = A_rK X_KK^T below it (W = L D), and L_rK = W_rK D_K^{-1};
//   (c) the trailing update A_rs -= W_rK L_sK^T, c1 <= s <= r (16-long dot
//       products in registers, one output entry each);
// then L = W D^{-1}, and (kXFull) the off-diagonal blocks of X = L^{-1}.
// Without them the tile holds X's diagonal blocks only, which is all that
// the blocked panel solve of the tile steps needs; k_ldlt_xfill adds the
// rest once the level is factored, off the chain of diagonal tiles.  Per
// column only the short steps of (a) are sequential; everything else is a
// few wide phases.
// smem: (64*65 + 64 + 48*17 + 16*49) elements of AT.
constexpr int kDiagBlockedElems = 64 * 65 + 64 + 48 * 17 + 16 * 49;

template <typename T, typename AT, bool kXFull = true>
__device__ void diag_tile_blocked(T* __restrict__ tile, AT* __restrict__ A, int* __restrict__ info) {
  constexpr int NB = 16;
  static_assert(kDiagThreads == 256, "the entry-to-thread map of (a) assumes 8 warps");
  AT* dinv = A + 64 * 65;  // [64] 1/d_c
  AT* Lp = dinv + 64;      // [48][17] L of the current panel
  AT* Tb = Lp + 48 * 17;   // [16][49] sum_K L_IK X_KJ of the current X block row
  const int tid = threadIdx.x;
  __syncthreads();
  read_elems<T, TE>(tile, [&](int e, T v) {
    const int r = e >> 6, c = e & 63;
    A[r * 65 + c] = (c <= r) ? (AT)v : AT(0);
  });
  __syncthreads();
  if (tid == 0) dinv[0] = pivot_rcp(A[0]);
  __syncthreads();
  // (a)'s entry of this thread: 0 (the next pivot) on warp 7, 1..96 on
  // warps 0-2, 97..136 on warps 4-5 (a step has at most 120 + 15 entries).
  // A triangle entry e of step c is (c + 1 + rr, c + 1 + off) with (rr, off)
  // a function of e alone, so it is decoded once; likewise (c)'s entries
  // e = tid + 256 k (at most 1176 of them: five per thread), packed rr << 8 | off.
  const int ea = tid == 224 ? 0 : (tid < 96 ? tid + 1 : (tid >= 128 && tid < 168 ? tid - 31 : -1));
  auto tri = [](int e) {
    int rr = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    rr += ((rr + 1) * (rr + 2) / 2 <= e);
    rr -= (rr * (rr + 1) / 2 > e);
    return (rr << 8) | (e - rr * (rr + 1) / 2);
  };
  const int ea_tri = ea >= 0 ? tri(ea) : 0;
  constexpr int kTrailPer = (48 * 49 / 2 + kDiagThreads - 1) / kDiagThreads;
  int tc_tri[kTrailPer];
#pragma unroll
  for (int k = 0; k < kTrailPer; ++k) tc_tri[k] = tri(tid + kDiagThreads * k);
  for (int K = 0; K < 4; ++K) {
    const int c0 = K * NB, c1 = c0 + NB;
    // (a) diagonal block: Schur complement inside the block and X_KK
    for (int c = c0; c < c1; ++c) {
      const int m = c1 - 1 - c, w = c - c0 + 1;
      const int nA = m * (m + 1) / 2, nX = m * w;
      const int e = ea;
      int r = 0, s2 = 0, j = 0;
      if (e >= 0 && e < nA) {
        r = c + 1 + (ea_tri >> 8);
        s2 = c + 1 + (ea_tri & 255);
      } else if (e >= nA && e < nA + nX) {
        const int x = e - nA, rr = x / w;
        j = c0 + (x - rr * w);
        r = c + 1 + rr;
      }
      __syncthreads();  // column c and d_c are final
      if (e >= 0 && e < nA) {
        const AT l = A[r * 65 + c] * dinv[c];
        const AT v = fma(-l, A[s2 * 65 + c], A[r * 65 + s2]);
        A[r * 65 + s2] = v;
        if (e == 0) dinv[c + 1] = pivot_rcp(v);  // entry (c+1, c+1): the next pivot is final
      } else if (e >= nA && e < nA + nX) {
        const AT l = A[r * 65 + c] * dinv[c];
        const AT xcj = (j == c) ? AT(1) : A[j * 65 + c];
        A[j * 65 + r] = fma(-l, xcj, A[j * 65 + r]);
      }
    }
    __syncthreads();
    if (K == 3) break;
    // (b) panel below the block: W_rc = A_rc + sum_{c0 <= m < c} A_rm X_cm
    const int nr = 64 - c1;
    {
      AT wv[3];
      int at[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {  // nr * 16 <= 768 entries
        const int e = tid + q * kDiagThreads;
        at[q] = -1;
        if (e < nr * NB) {
          const int r = c1 + e / NB, c = c0 + e % NB;
          AT v = A[r * 65 + c], v2 = 0;
          int mm = c0;
          for (; mm + 1 < c; mm += 2) {
            v = fma(A[r * 65 + mm], A[mm * 65 + c], v);
            v2 = fma(A[r * 65 + mm + 1], A[(mm + 1) * 65 + c], v2);
          }
          if (mm < c) v = fma(A[r * 65 + mm], A[mm * 65 + c], v);
          wv[q] = v + v2;
          at[q] = e;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (at[q] >= 0) {
          const int r = c1 + at[q] / NB, cc = at[q] % NB;
          A[r * 65 + c0 + cc] = wv[q];
          Lp[(r - c1) * 17 + cc] = wv[q] * dinv[c0 + cc];
        }
    }
    __syncthreads();
    // (c) trailing update of the rows and columns >= c1
    {
      const int n2 = nr * (nr + 1) / 2;  // at most 1176 entries
#pragma unroll
      for (int kk = 0; kk < kTrailPer; ++kk) {
        const int e = tid + kDiagThreads * kk;
        if (e >= n2) break;
        const int r = c1 + (tc_tri[kk] >> 8), s2 = c1 + (tc_tri[kk] & 255);
        const AT* wr = A + r * 65 + c0;
        const AT* ls = Lp + (s2 - c1) * 17;
        AT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
        for (int cc = 0; cc < NB; cc += 4) {
          a0 = fma(wr[cc], ls[cc], a0);
          a1 = fma(wr[cc + 1], ls[cc + 1], a1);
          a2 = fma(wr[cc + 2], ls[cc + 2], a2);
          a3 = fma(wr[cc + 3], ls[cc + 3], a3);
        }
        const AT v = A[r * 65 + s2] - ((a0 + a1) + (a2 + a3));
        A[r * 65 + s2] = v;
        if (e == 0) dinv[c1] = pivot_rcp(v);  // the next block's first pivot
      }
    }
    __syncthreads();
  }
  if (tid < T64) {
    const AT d = A[tid * 65 + tid];
    if (!(d > AT(0)) || !(d < AT(1e300))) atomicOr(info, 1);
  }
  for (int e = tid; e < TE; e += blockDim.x) {  // L = W D^{-1}
    int r = e >> 6, c = e & 63;
    if (c < r) A[r * 65 + c] *= dinv[c];
  }
  __syncthreads();
  if (kXFull) x_offdiag_blocks(A, Tb);
  for (int e = tid; e < TE; e += blockDim.x) tile[e] = (T)A[(e >> 6) * 65 + (e & 63)];
}

template <typename T>
__global__ void __launch_bounds__(256) k_ldlt_diag(T* __restrict__ fac, EnvDev E,
                                                   const int32_t* __restrict__ order, int k,
                                                   int* __restrict__ info) {
  using AT = typename Acc<T>::type;
  extern __shared__ unsigned char smraw[];
  step_release();
  step_acquire();
  const int p = order[blockIdx.x];
  diag_tile_blocked<T, AT, false>(fac + tile_at(E, p, k, k), reinterpret_cast<AT*>(smraw), info);
}

// The off-diagonal blocks of X in every diagonal tile (block order[y], tile
// x) of a level factored by the tile steps; only those entries are written.
template <typename T>
__global__ void __launch_bounds__(256) k_ldlt_xfill(T* __restrict__ fac, EnvDev E,
                                                    const int32_t* __restrict__ order) {
  using AT = typename Acc<T>::type;
  const int p = order[blockIdx.y], k = blockIdx.x;
  if (k >= E.nt[p]) return;
  extern __shared__ unsigned char smraw[];
  AT* A = reinterpret_cast<AT*>(smraw);  // [64][65]
  AT* Tb = A + 64 * 65;                   // [16][49]
  T* tile = fac + tile_at(E, p, k, k);
  read_elems<T, TE>(tile, [&](int e, T v) { A[(e >> 6) * 65 + (e & 63)] = (AT)v; });
  __syncthreads();
  x_offdiag_blocks(A, Tb);
  for (int e = threadIdx.x; e < TE; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    if ((r >> 4) < (c >> 4)) tile[e] = (T)A[r * 65 + c];
  }
}

// ------------------------------------------ coupling tiles of a block solve
// For a level solved as one block (p = 0) on a cluster: per tile row I the
// tiles that carry one tile row's solution into the next row's sums, so that
// each row of a sweep needs only the previous row's right-hand side acc
// (y_J = X_J acc_J forward, x_J = X_J^T acc_J backward, X_J = L_JJ^{-1}):
//   M_I = L_{I,I-1} X_{I-1}   (L_{I,I-1} y_{I-1} = M_I acc_{I-1}),
//   N_I = X_{I+1} L_{I+1,I}   (L_{I+1,I}^T x_{I+1} = N_I^T acc_{I+1}),
// and the reciprocals 1/d of D.  They follow the block's envelope: M_I at
// tile I, N_I^T at tile NT + I, then NT * 64 reciprocals.  CTA (I, 0) forms
// M_I and row I's reciprocals, CTA (I, 1) N_I^T; a tile outside the envelope
// (no L_{I,I-1} / L_{I+1,I}) is not formed, and the solve never reads it.
// The diagonal tile holds X above its diagonal: X[a][c] at dt[c][a], a > c.
template <typename T>
__global__ void __launch_bounds__(256) k_ldlt_mnfill(T* __restrict__ fac, EnvDev E) {
  using AT = typename Acc<T>::type;
  const int NT = E.nt[0], I = blockIdx.x, kind = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T* mn = fac + E.fac_off[1];
  if (kind == 0 && tid < 64) {
    const T* dt = fac + tile_at(E, 0, I, I);
    mn[(int64_t)2 * NT * TE + I * 64 + tid] = (T)(AT(1) / (AT)dt[tid * 65]);
  }
  const int Ir = kind == 0 ? I : I + 1;  // the tile row of L_{I,I-1} / L_{I+1,I}
  const int Jd = kind == 0 ? I - 1 : I + 1;  // the diagonal tile whose X is applied
  if (Ir >= NT || Ir - 1 < E.first[E.trow[0] + Ir] || Ir < 1) return;
  extern __shared__ unsigned char smraw[];
  AT* Ls = reinterpret_cast<AT*>(smraw);  // [64][65] L_{Ir,Ir-1}, then the result
  AT* Xs = Ls + 64 * 65;                  // [64][65] the diagonal tile of Jd
  read_elems<T, TE>(fac + tile_at(E, 0, Ir, Ir - 1), [&](int e, T v) { Ls[(e >> 6) * 65 + (e & 63)] = (AT)v; });
  read_elems<T, TE>(fac + tile_at(E, 0, Jd, Jd), [&](int e, T v) { Xs[(e >> 6) * 65 + (e & 63)] = (AT)v; });
  __syncthreads();
  AT o[2][8];
  if (kind == 0) {
    // M[r][c] = L[r][c] + sum_{a>c} L[r][a] X[a][c]; lane: rows lane, lane + 32; warp: columns warp + 8 j
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = warp + 8 * j;
      AT v0 = Ls[lane * 65 + c], v1 = Ls[(lane + 32) * 65 + c];
      for (int a = c + 1; a < 64; ++a) {
        const AT x = Xs[c * 65 + a];
        v0 = fma(Ls[lane * 65 + a], x, v0);
        v1 = fma(Ls[(lane + 32) * 65 + a], x, v1);
      }
      o[0][j] = v0;
      o[1][j] = v1;
    }
  } else {
    // N[a][c] = L[a][c] + sum_{b<a} X[a][b] L[b][c]; lane: columns lane, lane + 32; warp: rows warp + 8 j
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int a = warp + 8 * j;
      AT v0 = Ls[a * 65 + lane], v1 = Ls[a * 65 + lane + 32];
      for (int b = 0; b < a; ++b) {
        const AT x = Xs[b * 65 + a];
        v0 = fma(x, Ls[b * 65 + lane], v0);
        v1 = fma(x, Ls[b * 65 + lane + 32], v1);
      }
      o[0][j] = v0;
      o[1][j] = v1;
    }
  }
  __syncthreads();
  // the result in [row of the stored tile][column] order: M_I as is, N_I transposed
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int u = warp + 8 * j, w = lane + 32 * k;  // M: column u, row w; N: row u, column w
      Ls[w * 65 + u] = o[k][j];
    }
  __syncthreads();
  T* dst = mn + (int64_t)(kind == 0 ? I : NT + I) * TE;
  for (int e = tid; e < TE; e += blockDim.x) dst[e] = (T)Ls[(e >> 6) * 65 + (e & 63)];
}

// ----------------------------------------------------------- panel solve
// L_ik = A_ik X^T D^{-1} for a tile below the diagonal tile of step k.
// Column c needs the products over m <= c (X^T is upper triangular), so warp
// w takes the 4 columns 4w..4w+3 and the 4 columns 60-4w..63-4w: every warp
// does the same work.  Each lane owns 2 rows.  smem: (64*65 + 64*64 + 64) AT.
template <typename T, typename AT>
__device__ void panel_tile(const T* __restrict__ dtile, T* __restrict__ ptile, AT* __restrict__ A) {
  AT* Xt = A + 64 * 65;     // [64][64] X^T (upper, unit diagonal)
  AT* Dinv = Xt + 64 * 64;  // [64]
  const int tid = threadIdx.x;
  __syncthreads();
  read_elems<T, TE>(ptile, [&](int e, T v) { A[(e >> 6) * 65 + (e & 63)] = (AT)v; });
  read_elems<T, TE>(dtile, [&](int e, T v) {
    const int r = e >> 6, c = e & 63;
    Xt[e] = (r < c) ? (AT)v : (r == c ? AT(1) : AT(0));
    if (r == c) Dinv[r] = AT(1) / (AT)v;
  });
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int r0 = lane, r1 = lane + 32;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int c0 = half == 0 ? warp * 4 : 60 - warp * 4;
    AT w0[4], w1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { w0[q] = 0; w1[q] = 0; }
    const int mend = c0 + 4;
    for (int m = 0; m < mend; ++m) {
      AT a0 = A[r0 * 65 + m], a1 = A[r1 * 65 + m];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        AT x = Xt[m * 64 + c0 + q];
        w0[q] = fma(a0, x, w0[q]);
        w1[q] = fma(a1, x, w1[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ptile[r0 * 64 + c0 + q] = (T)(w0[q] * Dinv[c0 + q]);
      ptile[r1 * 64 + c0 + q] = (T)(w1[q] * Dinv[c0 + q]);
    }
  }
}

// Multi-launch form (levels with few, large blocks, the coarsest chain):
// every panel tile is split into kStepSplit CTAs of kStepRows rows, so that
// a step spreads over more SMs.  The diagonal tile holds X's diagonal
// blocks only (its off-diagonal blocks come after the level is factored), so
// W = A X^T is formed as the blocked solve W L^T = A, block column by block
// column: W_J = (A_J - sum_{K<J} W_K L_JK^T) X_JJ^T.  A thread pair shares
// one output (r, c) of block column J: each sums half of the products (the
// two halves of n < 16J, then the even and odd m of X_JJ) and the pair adds
// its halves with a shuffle.  Then L_ik = W D^{-1}.
constexpr int kStepSplit = 8, kStepRows = 64 / kStepSplit;
constexpr int kPanelElems = kStepRows * 65 + 64 * 65 + 64 + kStepRows * 17 + kStepRows * 65;

template <typename T>
__global__ void __launch_bounds__(256) k_ldlt_panel(T* __restrict__ fac, EnvDev E,
                                                    const int32_t* __restrict__ order, int k, int off) {
  using AT = typename Acc<T>::type;
  static_assert(kStepRows * 16 * 2 == 256, "a thread pair per output of a block column");
  step_release();
  step_acquire();
  const int p = order[blockIdx.y];
  const int i = k + 1 + off + blockIdx.x / kStepSplit, q = blockIdx.x % kStepSplit;
  if (i > E.last[E.trow[p] + k]) return;
  extern __shared__ unsigned char smraw[];
  AT* A = reinterpret_cast<AT*>(smraw);  // [kStepRows][65] rows of the panel tile
  AT* Lk = A + kStepRows * 65;           // [64][65] diagonal tile k: L below, X_JJ^T in the blocks above
  AT* Dinv = Lk + 64 * 65;               // [64]
  AT* Tt = Dinv + 64;                    // [kStepRows][17] T of the current block column
  AT* Wb = Tt + kStepRows * 17;          // [kStepRows][65] W, block column by block column
  const T* dtile = fac + tile_at(E, p, k, k);
  T* ptile = fac + tile_at(E, p, i, k) + q * kStepRows * 64;
  const int tid = threadIdx.x;
  read_elems<T, TE>(dtile, [&](int e, T v) {
    const int r = e >> 6, c = e & 63;
    Lk[r * 65 + c] = (AT)v;
    if (r == c) Dinv[r] = AT(1) / (AT)v;
  });
  read_elems<T, kStepRows * 64>(ptile, [&](int e, T v) { A[(e >> 6) * 65 + (e & 63)] = (AT)v; });
  __syncthreads();
  const int o = tid >> 1, h = tid & 1;  // output o of the block column, half h of its sums
  const int r = o >> 4, cc = o & 15;
  for (int J = 0; J < 4; ++J) {
    const int c = 16 * J + cc;
    AT t = 0;  // sum_{n < 16J} W_rn L_cn, half h
    for (int n = 8 * J * h; n < 8 * J * (h + 1); ++n) t = fma(Wb[r * 65 + n], Lk[c * 65 + n], t);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    if (h == 0) Tt[r * 17 + cc] = A[r * 65 + c] - t;
    __syncthreads();
    AT w = 0;  // sum_{16J <= m <= c} T_rm X_cm (X_cc = 1, X_cm at Lk[m][c]), the m of parity h
    for (int mm = h; mm <= cc; mm += 2)
      w = fma(Tt[r * 17 + mm], mm == cc ? AT(1) : Lk[(16 * J + mm) * 65 + c], w);
    w += __shfl_xor_sync(0xffffffffu, w, 1);
    if (h == 0) Wb[r * 65 + c] = w;
    __syncthreads();
  }
  for (int e = tid; e < kStepRows * 64; e += blockDim.x) {
    const int rr = e >> 6, c = e & 63;
    ptile[e] = (T)(Wb[rr * 65 + c] * Dinv[c]);
  }
}

// -------------------------------------------------------- trailing update
// A_ij -= (L_ik D_k) L_jk^T for one pair k < j <= i; each thread accumulates a
// 4x4 register block from k-major tiles.  smem: 2*64*65 AT.
__device__ inline void pair_of(int t, int& a, int& b) {  // t -> (a, b), b <= a
  int x = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((x + 1) * (x + 2) / 2 <= t) ++x;
  while (x * (x + 1) / 2 > t) --x;
  a = x;
  b = t - x * (x + 1) / 2;
}

template <typename T, typename AT>
__device__ void trail_pair(const T* __restrict__ dt, const T* __restrict__ li,
                           const T* __restrict__ lj, T* __restrict__ out, bool diagonal,
                           AT* __restrict__ smem) {
  constexpr int LD = 65;  // odd stride: the transposed stores spread over the banks
  AT* Wt = smem;         // [64 m][LD] = L_ik[r][m] * d_m
  AT* Lt = Wt + 64 * LD; // [64 m][LD] = L_jk[c][m]
  const int tid = threadIdx.x;
  __syncthreads();
  read_elems<T, TE>(li, [&](int e, T v) {
    const int r = e >> 6, m = e & 63;
    Wt[m * LD + r] = (AT)v * (AT)dt[m * 65];
  });
  read_elems<T, TE>(lj, [&](int e, T v) { Lt[(e & 63) * LD + (e >> 6)] = (AT)v; });
  __syncthreads();
  // 4x4 output blocks: all 256 of a general pair.  A diagonal pair needs the
  // 2080 entries on or below the diagonal (an idle lane costs as much FP64
  // issue time as a busy one): its 120 blocks strictly below the diagonal go
  // to warps 0-3, one block a thread, and the 160 entries of the 16 diagonal
  // blocks to warps 4-7, one entry a thread (a second pass for the last 32);
  // 69 warp instructions a step of m where 4x4 blocks for all 136 took 80.
  // (FP32 arithmetic keeps the 136 blocks: its issue is cheap, and the split
  // would cost the FP32 kernels registers)
  int rb, cb;
  if (!diagonal) {
    rb = tid >> 4;
    cb = tid & 15;
  } else if (sizeof(AT) == 4) {
    if (tid >= 136) return;
    pair_of(tid, rb, cb);  // rb >= cb
  } else if (tid < 128) {
    if (tid >= 120) return;
    pair_of(tid, rb, cb);  // cb <= rb < 15
    ++rb;
  } else {
#pragma unroll 1
    for (int u = tid - 128; u < 160; u += 128) {
      int x, y;
      pair_of(u % 10, x, y);  // y <= x < 4
      const int r = (u / 10) * 4 + x, c = (u / 10) * 4 + y;
      AT a0 = 0, a1 = 0;
#pragma unroll 8
      for (int m = 0; m < T64; m += 2) {
        a0 = fma(Wt[m * LD + r], Lt[m * LD + c], a0);
        a1 = fma(Wt[(m + 1) * LD + r], Lt[(m + 1) * LD + c], a1);
      }
      T* o = out + r * 64 + c;
      *o = (T)((AT)*o - (a0 + a1));
    }
    return;
  }
  const int r0 = rb * 4, c0 = cb * 4;
  AT acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0;
#pragma unroll 4
  for (int m = 0; m < T64; ++m) {
    AT av[4], bv[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      av[x] = Wt[m * LD + r0 + x];
      bv[x] = Lt[m * LD + c0 + x];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int r = r0 + x, c = c0 + y;
      if (!diagonal || c <= r) {
        T* o = out + r * 64 + c;
        *o = (T)((AT)*o - acc[x][y]);
      }
    }
}

// Multi-launch form: every pair is split into kStepSplit CTAs of kStepRows
// output rows; warp w owns row kStepRows*q + w and lane l the columns 2l and
// 2l + 1 (on a diagonal pair only those on or below the diagonal).
template <typename T>
__global__ void __launch_bounds__(256) k_ldlt_trail(T* __restrict__ fac, EnvDev E,
                                                    const int32_t* __restrict__ order, int k, int pair0) {
  using AT = typename Acc<T>::type;
  static_assert(kStepRows * 32 == 256, "one warp per output row");
  step_release();
  step_acquire();
  const int p = order[blockIdx.y];
  const int rem = E.last[E.trow[p] + k] - k;
  const int pair = pair0 + blockIdx.x / kStepSplit, q = blockIdx.x % kStepSplit;
  if (pair >= rem * (rem + 1) / 2) return;
  int a, b;
  pair_of(pair, a, b);
  const int i = k + 1 + a, j = k + 1 + b;
  const bool diagonal = (i == j);
  extern __shared__ unsigned char smraw[];
  constexpr int LD = 65;  // odd stride: the transposed stores spread over the banks
  AT* Wt = reinterpret_cast<AT*>(smraw);  // [64 m][kStepRows] = L_ik[kStepRows q + r][m] * d_m
  AT* Lt = Wt + 64 * kStepRows;           // [64 m][LD] = L_jk[c][m]
  const T* dt = fac + tile_at(E, p, k, k);
  const T* li = fac + tile_at(E, p, i, k) + q * kStepRows * 64;
  const T* lj = fac + tile_at(E, p, j, k);
  T* out = fac + tile_at(E, p, i, j) + q * kStepRows * 64;
  const int tid = threadIdx.x;
  read_elems<T, TE>(lj, [&](int e, T v) { Lt[(e & 63) * LD + (e >> 6)] = (AT)v; });
  read_elems<T, kStepRows * 64>(li, [&](int e, T v) {
    const int r = e >> 6, m = e & 63;
    Wt[m * kStepRows + r] = (AT)v * (AT)dt[m * 65];
  });
  __syncthreads();
  const int r = tid >> 5, c0 = (tid & 31) * 2;
  const int rg = kStepRows * q + r;  // row inside the tile
  if (diagonal && c0 > rg) return;
  AT acc0 = 0, acc1 = 0;
#pragma unroll 8
  for (int m = 0; m < T64; ++m) {
    const AT av = Wt[m * kStepRows + r];
    acc0 = fma(av, Lt[m * LD + c0], acc0);
    acc1 = fma(av, Lt[m * LD + c0 + 1], acc1);
  }
  T* o = out + r * 64 + c0;
  o[0] = (T)((AT)o[0] - acc0);
  if (!diagonal || c0 + 1 <= rg) o[1] = (T)((AT)o[1] - acc1);
}

// ------------------------------------------------- whole-block factorisation
// Persistent: CTA b factors the blocks cta_list[cta_ptr[b] .. cta_ptr[b+1])
// (a longest-first balanced assignment built on the host), every tile step
// in turn -- diagonal tile, its panel, the trailing pairs -- with the phases
// separated by block barriers (global writes of one phase are visible to the
// whole block in the next).  Used on levels with many blocks, where one launch
// replaces three launches per tile step.
// One whole block p of a level: every tile step in turn.
template <typename T, typename AT>
__device__ void factor_block(T* __restrict__ fac, const EnvDev& E, int p, AT* sm, int* info) {
  const int NT = E.nt[p];
  for (int k = 0; k < NT; ++k) {
    const int R = E.last[E.trow[p] + k];
    T* dt = fac + tile_at(E, p, k, k);
    // FP32 arithmetic: the blocked form (few index decodes, short sequential
    // steps); FP64: the unblocked one, whose every step fills all the lanes
    if constexpr (std::is_same<AT, float>::value) diag_tile_blocked<T, AT>(dt, sm, info);
    else diag_tile<T, AT>(dt, sm, info);
    for (int i = k + 1; i <= R; ++i) panel_tile<T, AT>(dt, fac + tile_at(E, p, i, k), sm);
    for (int i = k + 1; i <= R; ++i)
      for (int j = k + 1; j <= i; ++j)
        trail_pair<T, AT>(dt, fac + tile_at(E, p, i, k), fac + tile_at(E, p, j, k), fac + tile_at(E, p, i, j),
                          i == j, sm);
  }
}

// CTAs per SM the whole-block kernels are built for (their registers are
// capped to fit): FP32 arithmetic four, FP64 three.
template <typename T>
struct LevelCtas {
  static constexpr int value = sizeof(T) == 4 ? 4 : 3;
};

template <typename T>
__global__ void __launch_bounds__(256, LevelCtas<T>::value) k_ldlt_blocks(T* __restrict__ fac, EnvDev E,
                                                     const int32_t* __restrict__ cta_ptr,
                                                     const int32_t* __restrict__ cta_list,
                                                     int* __restrict__ info) {
  using AT = typename Acc<T>::type;
  extern __shared__ unsigned char smraw[];
  AT* sm = reinterpret_cast<AT*>(smraw);
  for (int q = cta_ptr[blockIdx.x]; q < cta_ptr[blockIdx.x + 1]; ++q) factor_block<T, AT>(fac, E, cta_list[q], sm, info);
}

// The same over blocks of several levels and instances (uneven sizes): item
// cta_list[q] names the factor storage, the level's envelope, the block and
// the instance's status word.  Each block's arithmetic is exactly that of
// k_ldlt_blocks.
template <typename T>
__global__ void __launch_bounds__(256, LevelCtas<T>::value) k_ldlt_blocks_batch(const BlockItem* __restrict__ items,
                                                           const int32_t* __restrict__ cta_ptr,
                                                           const int32_t* __restrict__ cta_list,
                                                           int* __restrict__ ctr, int nbins) {
  using AT = typename Acc<T>::type;
  extern __shared__ unsigned char smraw[];
  AT* sm = reinterpret_cast<AT*>(smraw);
  __shared__ BlockItem it;  // the current item, read from shared memory where it is used
  if (ctr == nullptr) {  // one static list per CTA
    for (int q = cta_ptr[blockIdx.x]; q < cta_ptr[blockIdx.x + 1]; ++q) {
      __syncthreads();  // the previous item is finished with
      if (threadIdx.x == 0) it = items[cta_list[q]];
      __syncthreads();
      factor_block<T, AT>(static_cast<T*>(it.fac), it.E, it.p, sm, it.info);
    }
    return;
  }
  // One list per SM (the CTAs resident on an SM share its FP64 pipe, so it is
  // the SMs' loads that are balanced): a CTA takes the next item of its own
  // SM's list.  Once that is exhausted it takes items only from lists that no
  // CTA of their own SM works on (an SM this launch did not reach, or left),
  // and leaves when there are none: a CTA that took another SM's items would
  // keep sharing its own SM's pipe with the block still running there, which
  // is often the list's largest.  ctr[b] counts the items taken from list b,
  // ctr[nbins + b] the CTAs of SM b still on it (both zeroed before the launch).
  __shared__ int got;
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  const int home = (int)(smid % (unsigned)nbins);
  int* active = ctr + nbins;
  int bin = home, tried = 0;
  bool own = true;
  if (threadIdx.x == 0) atomicAdd(&active[home], 1);
  for (;;) {
    __syncthreads();  // the previous item is finished with
    if (threadIdx.x == 0) {
      int g = -1;
      while (tried < nbins) {
        if (own || atomicAdd(&active[bin], 0) == 0) {
          const int q = atomicAdd(&ctr[bin], 1);
          if (q < cta_ptr[bin + 1] - cta_ptr[bin]) {
            g = cta_list[cta_ptr[bin] + q];
            break;
          }
          if (own) {  // the home list is exhausted
            atomicSub(&active[home], 1);
            own = false;
          }
        }
        bin = bin + 1 == nbins ? 0 : bin + 1;
        ++tried;
      }
      if (g >= 0) it = items[g];
      got = g;
    }
    __syncthreads();
    if (got < 0) break;
    factor_block<T, AT>(static_cast<T*>(it.fac), it.E, it.p, sm, it.info);
  }
}

// ------------------------------- whole-block factorisation, BF16 tensor cores
// The persistent factorisation for BF16 factors: diagonal tile and panel as
// in k_ldlt_blocks (FP32), the trailing update C_ij -= (L_ik D_k) L_jk^T on
// the tensor cores.  Tile rows k+1..R of the step are taken two at a time
// (M = 128) against two tile columns at a time (N = 128): the operands are
// rounded to BF16 into shared memory (K-major, no swizzle; a missing second
// tile is zero-filled), four K = 16 MMAs accumulate in FP32 in tensor memory
// (128 lanes x 128 columns per CTA), and the epilogue subtracts the
// accumulator from the FP32 working tiles: warp w reads lanes 32 (w % 4) ..
// of column half w / 4, one thread per row of one 64 x 64 output tile.  Only
// tiles with j <= i are written, and on the diagonal only c <= r.
constexpr int kTcCols = 128;                  // tensor-memory columns per CTA
constexpr int kTcSmem = 48 * 1024;           // >= every phase; keeps <= 4 CTAs per SM
constexpr int kTcSlab = 128 * 64 * 2;         // one 128 x 64 BF16 operand
constexpr int kTcBarOff = kTcSmem - 64;       // mbarrier + TMEM base address slot

// rows row0..row0+63 of a K-major BF16 slab = bf16(tile[r][k] * scale[k])
// (scale may be null); tile == null writes zeros.
// Each warp writes one 8-row x 8-column core matrix per pass (lane -> row
// lane / 4, column pair lane % 4): 32 distinct banks.
__device__ void stage_bf16(unsigned char* slab, int row0, const float* __restrict__ tile,
                           const float* __restrict__ scale) {
  constexpr int kIt = 64 * 32 / 256;  // 256 threads; all of a thread's loads in flight together
  float2 v[kIt];
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int e = threadIdx.x + 256 * it, lane = e & 31, blk = e >> 5;
    const int r = (blk >> 3) * 8 + (lane >> 2), k = (blk & 7) * 8 + (lane & 3) * 2;
    v[it] = tile ? *reinterpret_cast<const float2*>(tile + r * 64 + k) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int e = threadIdx.x + 256 * it, lane = e & 31, blk = e >> 5;
    const int r = (blk >> 3) * 8 + (lane >> 2), k = (blk & 7) * 8 + (lane & 3) * 2;
    if (tile && scale) {
      v[it].x *= scale[k];
      v[it].y *= scale[k + 1];
    }
    *reinterpret_cast<__nv_bfloat162*>(slab + tc::kmajor_offset(row0 + r, k)) =
        __floats2bfloat162_rn(v[it].x, v[it].y);
  }
}

__global__ void __launch_bounds__(256, 4) k_ldlt_blocks_tc(float* __restrict__ fac, EnvDev E,
                                                           const int32_t* __restrict__ cta_ptr,
                                                           const int32_t* __restrict__ cta_list,
                                                           int* __restrict__ info) {
  extern __shared__ __align__(1024) unsigned char smtc[];
  float* sm = reinterpret_cast<float*>(smtc);
  unsigned char* sA = smtc;                // W rows of the two output tile rows
  unsigned char* sB = smtc + kTcSlab;      // L rows of the two output tile columns
  float* dk = reinterpret_cast<float*>(smtc + 2 * kTcSlab);  // D of the step
  uint64_t* bar = reinterpret_cast<uint64_t*>(smtc + kTcBarOff);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smtc + kTcBarOff + 16);
  const int q0 = cta_ptr[blockIdx.x], q1 = cta_ptr[blockIdx.x + 1];
  if (q0 >= q1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(tslot, kTcCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const uint32_t idesc = tc::idesc_bf16_f32(128, 128);
  uint32_t phase = 0;
  bool failed = false;
  for (int q = q0; q < q1; ++q) {
    const int p = cta_list[q];
    const int NT = E.nt[p];
    for (int k = 0; k < NT; ++k) {
      const int R = E.last[E.trow[p] + k];
      float* dt = fac + tile_at(E, p, k, k);
      diag_tile_blocked<float, float>(dt, sm, info);
      for (int i = k + 1; i <= R; ++i) panel_tile<float, float>(dt, fac + tile_at(E, p, i, k), sm);
      if (R == k) continue;
      __syncthreads();
      if (tid < 64) dk[tid] = dt[tid * 65];
      __syncthreads();
      for (int i0 = k + 1; i0 <= R; i0 += 2) {
        const int i1 = i0 + 1;
        stage_bf16(sA, 0, fac + tile_at(E, p, i0, k), dk);
        stage_bf16(sA, 64, i1 <= R ? fac + tile_at(E, p, i1, k) : nullptr, dk);
        for (int j0 = k + 1; j0 <= i0; j0 += 2) {
          const int j1 = j0 + 1;
          stage_bf16(sB, 0, fac + tile_at(E, p, j0, k), nullptr);
          stage_bf16(sB, 64, j1 <= R ? fac + tile_at(E, p, j1, k) : nullptr, nullptr);
          tc::fence_async_smem();
          tc::fence_before();
          __syncthreads();
          tc::fence_after();
          if (tid == 0) {
#pragma unroll
            for (int st = 0; st < 4; ++st)
              tc::mma_bf16(taddr, tc::sdesc(sA + 256 * st), tc::sdesc(sB + 256 * st), idesc, st > 0);
            tc::commit(bar);
          }
          if (!tc::mbar_wait_bounded(bar, phase, failed ? 64 : (1L << 22))) {
            failed = true;
            if (lane == 0) atomicOr(info, 2);
          }
          phase ^= 1;
          tc::fence_after();
          // epilogue: this thread's row r of the 128 accumulator rows, column half h
          const int qd = warp & 3, h = warp >> 2;
          const int r = 32 * qd + lane;
          const int ti = r < 64 ? i0 : i1, tj = h ? j1 : j0, ri = r & 63;
          const bool valid = ti <= R && tj <= R && tj <= ti;
          float* crow = valid ? fac + tile_at(E, p, ti, tj) + ri * 64 : nullptr;
#pragma unroll
          for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * h + c0), v);
            if (valid) {
#pragma unroll
              for (int u = 0; u < 16; u += 4) {
                float4 cv = *reinterpret_cast<float4*>(crow + c0 + u);
                const int c = c0 + u;
                const bool diag = (ti == tj);
                if (!diag || c <= ri) cv.x -= v[u];
                if (!diag || c + 1 <= ri) cv.y -= v[u + 1];
                if (!diag || c + 2 <= ri) cv.z -= v[u + 2];
                if (!diag || c + 3 <= ri) cv.w -= v[u + 3];
                *reinterpret_cast<float4*>(crow + c0 + u) = cv;
              }
            }
          }
          tc::fence_before();
          __syncthreads();
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kTcCols);
}

// Diagonal tiles for the sliced kernel, one or two at a time (t1 may be
// null): the arithmetic of diag_tile, entry by entry and in the same order (so
// the same bits), two columns per pass:
//   P: for the rows r > c, the scaled column l0 = A_rc / d_c, the entries
//      (r, c+1) after step c and, from them, l1 = A'_r,c+1 / d_c+1 (every
//      thread forms d_c+1 = A'_c+1,c+1 and its reciprocal itself); row c+1 of
//      X after step c;
//   U: the two updates of every other entry of the trailing triangle and of
//      X, fused (fma(-l1, .., fma(-l0, .., a))), a thread's entries loaded,
//      updated and stored as a batch.
// Half the barriers of one column per pass, and two tiles share them: the
// pivots of a tile form a dependent chain of FP64 operations, which the other
// tile's work overlaps.  Scratch per tile: (64*65 + 3*64) doubles; at least
// 256 threads (128 per tile in P).
constexpr int kPairBatch = 4;
constexpr int kDiagScratch = 64 * 65 + 3 * 64;

__device__ void diag_tiles2(double* __restrict__ t0, double* __restrict__ t1, double* __restrict__ S0,
                            double* __restrict__ S1, int* __restrict__ info) {
  const int tid = threadIdx.x, nthr = blockDim.x, half = nthr / 2;
  const int ntile = t1 ? 2 : 1;
  __syncthreads();  // the shared buffers may still be read by a previous phase
  for (int e = tid; e < ntile * TE; e += nthr) {
    const int t = e >= TE, ee = e - t * TE;
    double* A = t ? S1 : S0;
    const double* tile = t ? t1 : t0;
    const int r = ee >> 6, c = ee & 63;
    A[r * 65 + c] = (c <= r) ? tile[ee] : 0.0;  // X starts as the identity (zeros above)
  }
  __syncthreads();
  if (tid < ntile) {
    double* A = tid ? S1 : S0;
    A[64 * 65 + 128] = pivot_rcp(A[0]);  // dinv[0]
  }
  __syncthreads();
  for (int c = 0; c < T64; c += 2) {
    const int c1 = c + 1;
    // ---- P: threads [half t, half t + 128) for tile t
    {
      const int t = tid / half, lt = tid - t * half;
      if (t < ntile && lt < 128) {
        double* A = t ? S1 : S0;
        double* l0 = A + 64 * 65;
        double* l1 = l0 + 64;
        double* dinv = l1 + 64;
        if (lt < T64) {
          const int r = lt;
          if (r > c) {
            const double lc = A[r * 65 + c] * dinv[c];
            l0[r] = lc;
            // pivot d_c+1 after step c, formed by every thread the same way
            const double lp = A[c1 * 65 + c] * dinv[c];
            const double d1 = fma(-lp, A[c1 * 65 + c], A[c1 * 65 + c1]);
            const double di1 = pivot_rcp(d1);
            if (r > c1) {
              const double a1 = fma(-lc, A[c1 * 65 + c], A[r * 65 + c1]);
              A[r * 65 + c1] = a1;
              l1[r] = a1 * di1;
            } else {  // r == c + 1: the pivot's own row
              dinv[c1] = di1;
              l1[c1] = d1;  // handed to U, which stores it on the diagonal
            }
          }
        } else if (lt - T64 <= c) {  // row c+1 of X after step c: X_c+1,j (at A[j][c+1]), j <= c
          const int j = lt - T64;
          const double lp = A[c1 * 65 + c] * dinv[c];
          const double xcj = (j == c) ? 1.0 : A[j * 65 + c];
          A[j * 65 + c1] = fma(-lp, xcj, A[j * 65 + c1]);
        }
      }
    }
    __syncthreads();
    // ---- U: the entries of both tiles in one range
    const int m = T64 - 2 - c;        // rows c+2 .. 63
    const int nA = m * (m + 1) / 2;   // trailing entries (r, s), c+2 <= s <= r
    const int w = c + 2;              // X columns j <= c+1
    const int nU = nA + m * w;
    if (tid < ntile) {
      double* A = tid ? S1 : S0;
      A[c1 * 65 + c1] = A[64 * 65 + 64 + c1];  // d_c+1 onto the diagonal
    }
    for (int base = 0; base < ntile * nU; base += nthr * kPairBatch) {
      int idx[kPairBatch];
      unsigned tsel = 0;  // bit q: entry q is in the second tile
      double av[kPairBatch], b0[kPairBatch], b1[kPairBatch], f0[kPairBatch], f1[kPairBatch];
#pragma unroll
      for (int q = 0; q < kPairBatch; ++q) {
        int e = base + tid + q * nthr;
        idx[q] = -1;
        if (e >= ntile * nU) continue;
        const int t = e >= nU;
        e -= t * nU;
        double* A = t ? S1 : S0;
        const double* l0 = A + 64 * 65;
        const double* l1 = l0 + 64;
        tsel |= (unsigned)t << q;
        int r, s;
        if (e < nA) {
          int rr = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
          rr += ((rr + 1) * (rr + 2) / 2 <= e);
          rr -= (rr * (rr + 1) / 2 > e);
          r = c + 2 + rr;
          s = c + 2 + (e - rr * (rr + 1) / 2);
          idx[q] = r * 65 + s;
          f0[q] = l0[r];
          f1[q] = l1[r];
          b0[q] = A[s * 65 + c];
          b1[q] = A[s * 65 + c1];
        } else {
          const int x = e - nA, rr = x / w, j = x - rr * w;
          r = c + 2 + rr;
          idx[q] = j * 65 + r;  // X_rj at A[j][r]
          f0[q] = (j <= c) ? l0[r] : 0.0;
          f1[q] = l1[r];
          b0[q] = (j == c) ? 1.0 : (j < c ? A[j * 65 + c] : 0.0);
          b1[q] = (j == c1) ? 1.0 : A[j * 65 + c1];
        }
        av[q] = A[idx[q]];
      }
#pragma unroll
      for (int q = 0; q < kPairBatch; ++q) {
        if (idx[q] < 0) continue;
        const double v = fma(-f1[q], b1[q], fma(-f0[q], b0[q], av[q]));
        double* A = ((tsel >> q) & 1u) ? S1 : S0;
        A[idx[q]] = v;
        if (idx[q] == (c + 2) * 65 + (c + 2)) A[64 * 65 + 128 + c + 2] = pivot_rcp(v);  // next first pivot
      }
    }
    __syncthreads();
  }
  if (tid < ntile * T64) {
    const double* A = tid >= T64 ? S1 : S0;
    const int r = tid & 63;
    const double d = A[r * 65 + r];
    if (!(d > 0.0) || !(d < 1e300)) atomicOr(info, 1);
  }
  for (int e = tid; e < ntile * TE; e += nthr) {  // L = W D^{-1}
    const int t = e >= TE, ee = e - t * TE;
    double* A = t ? S1 : S0;
    const int r = ee >> 6, c = ee & 63;
    if (c < r) A[r * 65 + c] *= A[64 * 65 + 128 + c];
  }
  __syncthreads();
  for (int e = tid; e < ntile * TE; e += nthr) {
    const int t = e >= TE, ee = e - t * TE;
    (t ? t1 : t0)[ee] = (t ? S1 : S0)[(ee >> 6) * 65 + (ee & 63)];
  }
}

// ------------------------- whole-block factorisation, FP64 by exact BF16 slices
// FP64 factors whose GEMM-shaped products -- the panel W_ik = A_ik X^T and the
// trailing update C_ij -= W_ik L_jk^T of every tile step -- run on the BF16
// tensor cores without rounding error, by splitting the operands into digits
// (the Ozaki scheme):
//   * every row of an operand (K = 64 entries) gets the exponent e of its
//     largest entry, |x| < 2^e, and becomes the integer m = round(x 2^(54-e)),
//     |m| < 2^54;
//   * m is written as eight balanced base-128 digits, m = sum_s d_s 128^(7-s),
//     |d_0| <= 33, |d_s| <= 64 for s > 0: every digit is exact in BF16;
//   * for one output block (128 rows x 64 columns) the digit products with
//     s + t = g are summed by the tensor cores in FP32, group g in its own 64
//     tensor-memory columns (8 groups: all 512).  Each product is below 2^12,
//     a K = 64 sum below 2^18 and a group of at most 8 sums below 2^21, so every
//     FP32 accumulation is exact;
//   * the groups g = 0..7 are combined in 64-bit integers in units of
//     2^(e_r + e_c - 56) (group g weighs 2^(46 - 7g); the last one is rounded
//     to the unit) and converted to FP64 once.  The digit pairs with s + t > 7
//     are left out: with every digit at its bound they add up to about
//     2^-49.2 K max|a_r| max|b_c|; the rounding of the operands to 54 bits is
//     below 2^-53 of it.
// So each product entry is within 2^-48 K max|a_r| max|b_c| of the exact sum
// (random digits land far inside): below the worst case of an FP64 dot product
// of the same length, K 2^-53 sum|a||b|, which reaches 2^-47 of that bound.  The diagonal tile
// (its L D L^T and X = L^-1, a sequential sweep: diag_tile_pair) stays on the
// FP64 pipe.  One CTA of 512 threads per SM: 192 KB of digit slabs and all
// 512 tensor-memory columns.
constexpr int kOzDigits = 8;                               // digits per entry
constexpr int kOzASlab = 128 * 64 * 2;                     // one 128 x 64 BF16 digit slab (A)
constexpr int kOzBSlab = 64 * 64 * 2;                      // one 64 x 64 BF16 digit slab (B)
constexpr int kOzBOff = kOzDigits * kOzASlab;              // 128 KB
constexpr int kOzMetaOff = kOzBOff + kOzDigits * kOzBSlab; // 192 KB
constexpr int kOzEA = kOzMetaOff;                          // int32 [128] row exponents of A
constexpr int kOzEB = kOzEA + 128 * 4;                     // int32 [64] row exponents of B
constexpr int kOzDk = kOzEB + 64 * 4;                      // double [64] D of the step
constexpr int kOzDinv = kOzDk + 64 * 8;                    // double [64] 1 / D
constexpr int kOzBar = kOzDinv + 64 * 8;                   // mbarrier, then the TMEM base slot
constexpr int kOzSmem = kOzBar + 64;
constexpr int kOzS1 = 36 * 1024;                          // the second diagonal tile's scratch
static_assert(kOzS1 + kDiagScratch * 8 <= kOzBOff, "two diagonal tiles' scratch fits in the A slabs");
static_assert(kDiagScratch * 8 <= kOzS1, "the first scratch ends before the second");

// biased exponent field of x (0 for zero and subnormal numbers)
__device__ __forceinline__ int oz_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// |m| = round(|x| 2^(54 - e)) < 2^54 for the row exponent e = emax - 1022
// (emax: the largest biased exponent of the row); subnormal entries count as
// zero.
__device__ __forceinline__ unsigned long long oz_fixed_abs(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;  // 53 bits
  const int sh = e - emax + 1;                                                     // <= 1
  if (sh >= 0) return mant << sh;
  if (sh > -56) return (mant + (1ull << (-sh - 1))) >> (-sh);
  return 0;
}

// One balanced base-128 digit of an FP32-exact integer v >= 0 (v < 2^22):
// q = rint(v / 128) through the 1.5 * 2^23 offset, d = v - 128 q in [-64, 64].
__device__ __forceinline__ float oz_peel(float& v) {
  const float q = __fadd_rn(__fmaf_rn(v, 0.0078125f, 12582912.0f), -12582912.0f);
  const float d = __fmaf_rn(-128.0f, q, v);
  v = q;
  return d;
}

// The eight balanced base-128 digits of |m| < 2^54, most significant first,
// |d_0| <= 33, |d_s| <= 64: |m| is cut into three FP32-exact pieces (bits
// 0..13, 14..34, 35..55, each read into FP32 through the 2^23 offset), whose
// digits are peeled in FP32 with the carries going upward.  The digits are
// small integers in FP32, so their BF16 form is the upper half of their bits.
__device__ __forceinline__ void oz_digits(unsigned long long m, float (&d)[kOzDigits]) {
  float v = __uint_as_float(0x4B000000u | ((uint32_t)m & 0x3FFFu)) - 8388608.0f;
  d[7] = oz_peel(v);
  d[6] = oz_peel(v);
  v += __uint_as_float(0x4B000000u | ((uint32_t)(m >> 14) & 0x1FFFFFu)) - 8388608.0f;
  d[5] = oz_peel(v);
  d[4] = oz_peel(v);
  d[3] = oz_peel(v);
  v += __uint_as_float(0x4B000000u | (uint32_t)(m >> 35)) - 8388608.0f;
  d[2] = oz_peel(v);
  d[1] = oz_peel(v);
  d[0] = v;
}

// Writes the digits of 8 consecutive K entries of one row into the 8 slabs
// (the sign of an entry is the sign bit of each of its BF16 digits).
__device__ __forceinline__ void oz_store8(unsigned char* slab0, int slab_bytes, int row, int k0,
                                          const double (&x)[8], int emax) {
  uint32_t w[kOzDigits][4];
#pragma unroll
  for (int u = 0; u < 8; u += 2) {
    float d0[kOzDigits], d1[kOzDigits];
    oz_digits(oz_fixed_abs(x[u], emax), d0);
    oz_digits(oz_fixed_abs(x[u + 1], emax), d1);
    const uint32_t sg = (x[u] < 0.0 ? 0x8000u : 0u) | (x[u + 1] < 0.0 ? 0x80000000u : 0u);
#pragma unroll
    for (int s = 0; s < kOzDigits; ++s)
      w[s][u >> 1] = __byte_perm(__float_as_uint(d0[s]), __float_as_uint(d1[s]), 0x7632) ^ sg;
  }
#pragma unroll
  for (int s = 0; s < kOzDigits; ++s)
    *reinterpret_cast<uint4*>(slab0 + s * slab_bytes + tc::kmajor_offset(row, k0)) =
        make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// A operand: rows 0..63 from tile t0, 64..127 from t1 (null: zeros), each
// entry times dk[m] when dk is given (W = L D).  Four threads per row, 16 K
// entries each (512 threads).
__device__ void oz_split_a(unsigned char* sA, int* eA, const double* __restrict__ t0,
                           const double* __restrict__ t1, const double* dk) {
  const int tid = threadIdx.x, r = tid >> 2, kq = tid & 3;
  const double* src = r < 64 ? t0 : t1;
  double x[16];
  int emax = 0;
  if (src) {
    const double* row = src + (r & 63) * 64 + kq * 16;
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      const double2 v = *reinterpret_cast<const double2*>(row + u);
      x[u] = v.x;
      x[u + 1] = v.y;
    }
    if (dk) {
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] *= dk[kq * 16 + u];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) emax = max(emax, oz_exp(x[u]));
  } else {
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = 0.0;
  }
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
  if (kq == 0) eA[r] = emax;
#pragma unroll
  for (int c8 = 0; c8 < 2; ++c8) {
    double y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) y[u] = x[c8 * 8 + u];
    oz_store8(sA, kOzASlab, r, kq * 16 + c8 * 8, y, emax);
  }
}

// B operand (64 rows c, K = m): the tile t itself (B[c][m] = t[c][m]), or with
// xmat the unit lower X of a factored diagonal tile, X[c][m] = t[m][c] for
// m < c.  Eight threads per row, 8 K entries each (512 threads).
__device__ void oz_split_b(unsigned char* sB, int* eB, const double* __restrict__ t, bool xmat) {
  const int tid = threadIdx.x, c = tid >> 3, k8 = tid & 7;
  double x[8];
  int emax = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int m = k8 * 8 + u;
    if (xmat) x[u] = m < c ? t[m * 64 + c] : (m == c ? 1.0 : 0.0);
    else x[u] = t[c * 64 + m];
    emax = max(emax, oz_exp(x[u]));
  }
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 4));
  if (k8 == 0) eB[c] = emax;
  oz_store8(sB, kOzBSlab, c, k8 * 8, x, emax);
}

// V 2^(er + ec - 2100) in FP64, rounded to nearest even, for the biased row
// exponents er, ec of the two operands: the integer sum in units of
// 2^(e_r + e_c - 56), e = biased exponent - 1022.  Built from the bits: the
// leading one of |V| gives the exponent, the next 52 bits (rounded) the
// significand.  Results outside the normal range go through FP64 products.
__device__ __forceinline__ double oz_to_double(long long V, int er, int ec) {
  if (V == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)V & 0x8000000000000000ull;
  unsigned long long a = V < 0 ? 0ull - (unsigned long long)V : (unsigned long long)V;
  const int lz = __clzll((long long)a);
  a <<= lz;  // leading one at bit 63
  unsigned long long mant = a >> 11;  // 53 bits, hidden one included
  const unsigned long long rest = a & 0x7FFull;
  mant += (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  const int e = 63 - lz + er + ec - 2100 + 1023;  // biased exponent of the leading one
  if (e < 1 || e > 2046) {  // 2^(er - 1050) 2^(ec - 1050); rows below 2^-994 count as zero
    if (er <= 28 || ec <= 28) return 0.0;
    return ((double)V * __longlong_as_double((long long)(er - 27) << 52)) *
           __longlong_as_double((long long)(ec - 27) << 52);
  }
  // the hidden one carries into the exponent field (twice after a rounding carry)
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(e - 1) << 52) + mant)));
}

// Issues the 36 digit-pair products of one output block (s + t <= 7, group
// s + t in tensor-memory columns 64 (s + t) ..) and commits them to `bar`.
// One thread.  The first product of every group overwrites its columns.
__device__ __forceinline__ void oz_issue(uint32_t taddr, const unsigned char* sA, const unsigned char* sB,
                                         uint64_t* bar) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
  // the descriptors of every slab step differ only in the start address
  // field (address / 16, 14 bits; the slabs lie below 256 KB): one add each
  const uint64_t a0 = tc::sdesc(sA), b0 = tc::sdesc(sB);
#pragma unroll 1
  for (int s = 0; s < kOzDigits; ++s) {
    const uint64_t as = a0 + (uint64_t)((s * kOzASlab) >> 4);
#pragma unroll 1
    for (int t = 0; s + t < kOzDigits; ++t) {
      const uint32_t d = taddr + (uint32_t)((s + t) * 64);
      const uint64_t bt = b0 + (uint64_t)((t * kOzBSlab) >> 4);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_bf16(d, as + (uint64_t)(16 * kk), bt + (uint64_t)(16 * kk), idesc, (s > 0 || kk > 0) ? 1 : 0);
    }
  }
  tc::commit(bar);
}

// The product of the slabs in shared memory for one output block: MMAs by
// thread 0; while they run, pre(r, q, C) may load this thread's 16 outputs
// (row r = 32 (warp % 4) + lane, columns 16 (warp / 4) ..); a bounded wait;
// then the 64-bit integer sums V of those entries, handed to epi(r, q, V, C)
// before the block barrier that frees the slabs, the row exponents and the
// tensor memory.  Returns the updated `failed`.
template <typename Pre, typename Epi>
__device__ __forceinline__ bool oz_product(uint32_t taddr, unsigned char* sm, uint64_t* bar, uint32_t& phase,
                                           bool failed, int* info, Pre pre, Epi epi) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid == 0) oz_issue(taddr, sm, sm + kOzBOff, bar);
  double C[16];
  pre(32 * (warp & 3) + lane, warp >> 2, C);
  if (!tc::mbar_wait_bounded(bar, phase, failed ? 64 : (1L << 22))) {
    failed = true;
    if (lane == 0) atomicOr(info, 2);
  }
  phase ^= 1;
  tc::fence_after();
  const int qd = warp & 3, q = warp >> 2;
  long long V[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) V[c] = 0;
#pragma unroll
  for (int g = 0; g < kOzDigits; g += 2) {
    float v0[16], v1[16];
    const uint32_t ta = taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(g * 64 + 16 * q);
    tc::tmem_ld16(ta, v0);
    tc::tmem_ld16(ta + 64, v1);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      // the exact integer group sums (|v| < 2^22) through the 1.5 * 2^23
      // offset; groups g and g + 1 joined in 32 bits (< 2^29), weight 2^(39 - 7g)
      const int i0 = __float_as_int(v0[u] + 12582912.0f) - 0x4B400000;
      const int i1 = __float_as_int(v1[u] + 12582912.0f) - 0x4B400000;
      const int qv = i0 * 128 + i1;
      if (g < kOzDigits - 2) V[u] += (long long)qv << (39 - 7 * g);
      else V[u] += (long long)((qv + 4) >> 3);
    }
  }
  epi(32 * qd + lane, q, V, C);
  tc::fence_before();
  __syncthreads();
  return failed;
}

// One tile step k of block p after its diagonal tile dt is factored (R > k):
// the panel L_ik = (A_ik X^T) D^-1 and the trailing update, every product on
// the tensor cores by digit slices.
__device__ __noinline__ bool oz_step(double* __restrict__ fac, const EnvDev& E, int p, int k, int R,
                                        const double* __restrict__ dt, unsigned char* smoz, uint32_t taddr,
                                        uint64_t* bar, uint32_t& phase, bool failed, int* info) {
  int* eA = reinterpret_cast<int*>(smoz + kOzEA);
  int* eB = reinterpret_cast<int*>(smoz + kOzEB);
  double* dk = reinterpret_cast<double*>(smoz + kOzDk);
  double* dinv = reinterpret_cast<double*>(smoz + kOzDinv);
  const int tid = threadIdx.x;
  __syncthreads();  // the factored diagonal tile is in global memory
  if (tid < 64) {
    const double d = dt[tid * 65];
    dk[tid] = d;
    dinv[tid] = 1.0 / d;
  }
  // panel: L_ik = (A_ik X^T) D^-1, tile rows two at a time
  oz_split_b(smoz + kOzBOff, eB, dt, true);
  for (int i0 = k + 1; i0 <= R; i0 += 2) {
    oz_split_a(smoz, eA, fac + tile_at(E, p, i0, k), i0 + 1 <= R ? fac + tile_at(E, p, i0 + 1, k) : nullptr,
               nullptr);
    failed = oz_product(
        taddr, smoz, bar, phase, failed, info, [](int, int, double(&)[16]) {},
        [&](int r, int h, long long(&V)[16], double(&)[16]) {
      const int ti = r < 64 ? i0 : i0 + 1;
      if (ti > R) return;
      const int er = eA[r];
      double* out = fac + tile_at(E, p, ti, k) + (r & 63) * 64 + 16 * h;
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const int cc = 16 * h + c;
        double2 o;
        o.x = oz_to_double(V[c], er, eB[cc]) * dinv[cc];
        o.y = oz_to_double(V[c + 1], er, eB[cc + 1]) * dinv[cc + 1];
        *reinterpret_cast<double2*>(out + c) = o;
      }
    });
  }
  // trailing update: C_ij -= (L_ik D_k) L_jk^T, k < j <= i <= R; the
  // digits of two rows of W = L D at a time, against every column tile j
  // up to the second row (the rows i < j of a block are not written)
  for (int i0 = k + 1; i0 <= R; i0 += 2) {
    const int i1 = i0 + 1 <= R ? i0 + 1 : i0;
    oz_split_a(smoz, eA, fac + tile_at(E, p, i0, k), i0 + 1 <= R ? fac + tile_at(E, p, i0 + 1, k) : nullptr,
               dk);
    for (int j = k + 1; j <= i1; ++j) {
      oz_split_b(smoz + kOzBOff, eB, fac + tile_at(E, p, j, k), false);
      // this thread's 16 entries of C_ij, loaded while the tensor cores run
      auto pre = [&](int r, int h, double(&C)[16]) {
        const int ti = r < 64 ? i0 : i0 + 1;
        if (ti > R || ti < j) return;
        const double2* src = reinterpret_cast<const double2*>(fac + tile_at(E, p, ti, j) + (r & 63) * 64 + 16 * h);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const double2 v = src[c];
          C[2 * c] = v.x;
          C[2 * c + 1] = v.y;
        }
      };
      failed = oz_product(taddr, smoz, bar, phase, failed, info, pre,
                          [&](int r, int h, long long(&V)[16], double(&C)[16]) {
        const int ti = r < 64 ? i0 : i0 + 1;
        if (ti > R || ti < j) return;
        const int rr = r & 63, er = eA[r];
        double2* out = reinterpret_cast<double2*>(fac + tile_at(E, p, ti, j) + rr * 64 + 16 * h);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int cc = 16 * h + c;
          // a diagonal tile keeps its upper part (X^T later): written back unchanged
          if (ti != j || cc <= rr) C[c] -= oz_to_double(V[c], er, eB[cc]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) out[c] = make_double2(C[2 * c], C[2 * c + 1]);
      });
    }
  }
  return failed;
}

// Persistent: CTA b takes the blocks cta_list[cta_ptr[b] .. cta_ptr[b+1]) two
// at a time, step by step: their diagonal tiles together (diag_tiles2), then
// the tensor-core products of each.
__global__ void __launch_bounds__(512, 1) k_ldlt_blocks_oz(double* __restrict__ fac, EnvDev E,
                                                           const int32_t* __restrict__ cta_ptr,
                                                           const int32_t* __restrict__ cta_list,
                                                           int* __restrict__ info) {
  extern __shared__ __align__(1024) unsigned char smoz[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smoz + kOzBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smoz + kOzBar + 16);
  double* S0 = reinterpret_cast<double*>(smoz);
  double* S1 = reinterpret_cast<double*>(smoz + kOzS1);
  const int q0 = cta_ptr[blockIdx.x], q1 = cta_ptr[blockIdx.x + 1];
  if (q0 >= q1) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(tslot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  uint32_t phase = 0;
  bool failed = false;
  for (int q = q0; q < q1; q += 2) {
    const int pa = cta_list[q], pb = q + 1 < q1 ? cta_list[q + 1] : -1;
    const int nta = E.nt[pa], ntb = pb >= 0 ? E.nt[pb] : 0;
    for (int k = 0; k < max(nta, ntb); ++k) {
      double* da = k < nta ? fac + tile_at(E, pa, k, k) : nullptr;
      double* db = k < ntb ? fac + tile_at(E, pb, k, k) : nullptr;
      diag_tiles2(da ? da : db, da ? db : nullptr, S0, S1, info);
      if (da) {
        const int R = E.last[E.trow[pa] + k];
        if (R > k) failed = oz_step(fac, E, pa, k, R, da, smoz, taddr, bar, phase, failed, info);
      }
      if (db) {
        const int R = E.last[E.trow[pb] + k];
        if (R > k) failed = oz_step(fac, E, pb, k, R, db, smoz, taddr, bar, phase, failed, info);
      }
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
void launch_extract(const int64_t* ext_pos, const int32_t* ext_nz, int64_t nent,
                    const double* val, int64_t fac_elems, T* fac, cudaStream_t s) {
  // the envelope's zeros (0.0 is all-zero bits in every factor type): a
  // memset, which runs at the copy rate where a store loop of 4- or 8-byte
  // elements is instruction-bound
  if (fac_elems > 0) cudaMemsetAsync(fac, 0, (size_t)fac_elems * sizeof(T), s);
  if (nent > 0) k_scatter<T><<<nblk(nent, 256), 256, 0, s>>>(ext_pos, ext_nz, val, nent, fac);
}

// Launch with programmatic stream serialisation (the kernels order their
// reads behind their predecessor with step_acquire).
template <typename... KArgs, typename... Args>
void launch_step(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
void launch_ldlt_diag(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                      int* info, cudaStream_t s) {
  if (nactive <= 0) return;
  using AT = typename Acc<T>::type;
  size_t smem = (size_t)kDiagBlockedElems * sizeof(AT);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_ldlt_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  launch_step(k_ldlt_diag<T>, dim3(nactive), smem, s, fac, E, order, k, info);
}

template <typename T>
void launch_ldlt_panel(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                       int off, int max_rows, cudaStream_t s) {
  if (nactive <= 0 || max_rows <= 0) return;
  using AT = typename Acc<T>::type;
  size_t smem = (size_t)kPanelElems * sizeof(AT);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_ldlt_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  launch_step(k_ldlt_panel<T>, dim3(kStepSplit * max_rows, nactive), smem, s, fac, E, order, k, off);
}

template <typename T>
void launch_ldlt_trail(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                       int pair0, int max_pairs, cudaStream_t s) {
  if (nactive <= 0 || max_pairs <= 0) return;
  using AT = typename Acc<T>::type;
  size_t smem = (64 * kStepRows + 64 * 65) * sizeof(AT);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_ldlt_trail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  launch_step(k_ldlt_trail<T>, dim3(kStepSplit * max_pairs, nactive), smem, s, fac, E, order, k, pair0);
}


template <typename T>
void launch_ldlt_xfill(T* fac, const EnvDev& E, const int32_t* order, int nblocks, int max_nt, cudaStream_t s) {
  if (nblocks <= 0 || max_nt <= 0) return;
  using AT = typename Acc<T>::type;
  size_t smem = (size_t)(64 * 65 + 16 * 49) * sizeof(AT);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_ldlt_xfill<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_ldlt_xfill<T><<<dim3(max_nt, nblocks), 256, smem, s>>>(fac, E, order);
}

template <typename T>
void launch_ldlt_mnfill(T* fac, const EnvDev& E, int nt, cudaStream_t s) {
  if (nt <= 0) return;
  using AT = typename Acc<T>::type;
  const size_t smem = (size_t)2 * 64 * 65 * sizeof(AT);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_ldlt_mnfill<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_ldlt_mnfill<T><<<dim3(nt, 2), 256, smem, s>>>(fac, E);
}

// CTAs of a 256-thread persistent kernel resident per SM at once: limited by
// its shared memory (with the carveout set to the maximum) and its registers.
int resident_per_sm(const void* fn, size_t smem) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  int dev = 0, per_sm_smem = 0, per_sm_regs = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&per_sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, fn);
  const size_t per_cta_smem = smem + fa.sharedSizeBytes + 1024;  // + the per-CTA reservation
  const int regs = std::max(1, ((fa.numRegs + 7) / 8) * 8) * 256;
  int n = (int)std::min<size_t>(per_sm_smem / per_cta_smem, (size_t)(per_sm_regs / regs));
  n = std::min(n, 2048 / 256);
  cudaGetLastError();
  return std::max(1, n);
}

template <typename T>
void launch_ldlt_blocks(T* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                        int grid, int* info, cudaStream_t s) {
  using AT = typename Acc<T>::type;
  if (grid < 1) return;
  const size_t smem = (size_t)(2 * 64 * 65) * sizeof(AT);  // the largest phase (trailing pair)
  static std::once_flag attr;
  std::call_once(attr, [&] { resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks<T>), smem); });
  k_ldlt_blocks<T><<<grid, 256, smem, s>>>(fac, E, cta_ptr, cta_list, info);
}

template <typename T>
void launch_ldlt_blocks_batch(const BlockItem* items, const int32_t* cta_ptr, const int32_t* cta_list, int grid,
                              cudaStream_t s, int* sm_ctr, int nbins) {
  using AT = typename Acc<T>::type;
  if (grid < 1) return;
  const size_t smem = (size_t)(2 * 64 * 65) * sizeof(AT);  // the largest phase (trailing pair)
  static std::once_flag attr;
  std::call_once(attr, [&] { resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks_batch<T>), smem); });
  k_ldlt_blocks_batch<T><<<grid, 256, smem, s>>>(items, cta_ptr, cta_list, sm_ctr, nbins);
}

template <typename T>
int ldlt_blocks_batch_per_sm() {
  using AT = typename Acc<T>::type;
  const size_t smem = (size_t)(2 * 64 * 65) * sizeof(AT);
  static int n = resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks_batch<T>), smem);
  return n;
}

// CTAs of k_ldlt_blocks per SM, so that the persistent grid is exactly one wave.
template <typename T>
int ldlt_blocks_per_sm() {
  using AT = typename Acc<T>::type;
  const size_t smem = (size_t)(2 * 64 * 65) * sizeof(AT);  // the largest phase (trailing pair)
  static int n = resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks<T>), smem);
  return n;
}

void launch_ldlt_blocks_tc(float* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                           int grid, int* info, cudaStream_t s) {
  if (grid < 1) return;
  static std::once_flag attr;
  std::call_once(attr, [] { resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks_tc), kTcSmem); });
  k_ldlt_blocks_tc<<<grid, 256, kTcSmem, s>>>(fac, E, cta_ptr, cta_list, info);
}

void launch_ldlt_blocks_oz(double* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                           int grid, int* info, cudaStream_t s) {
  if (grid < 1) return;
  static std::once_flag attr;
  std::call_once(attr, [] { resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks_oz), kOzSmem); });
  k_ldlt_blocks_oz<<<grid, 512, kOzSmem, s>>>(fac, E, cta_ptr, cta_list, info);
}

// k_ldlt_blocks_oz: one CTA per SM (its shared memory and all the tensor memory).
int ldlt_blocks_oz_per_sm() { return 1; }

// CTAs of k_ldlt_blocks_tc per SM: resident at once, and at most 512 / 128
// (the tensor memory of an SM), so that no allocation ever waits.
int ldlt_blocks_tc_per_sm() {
  static int n = resident_per_sm(reinterpret_cast<const void*>(k_ldlt_blocks_tc), kTcSmem);
  return std::min(512 / kTcCols, n);
}

#define MSP_INST(T)                                                                              \
  template void launch_extract<T>(const int64_t*, const int32_t*, int64_t, const double*,        \
                                  int64_t, T*, cudaStream_t);                                    \
  template void launch_ldlt_diag<T>(T*, const EnvDev&, const int32_t*, int, int, int*,           \
                                    cudaStream_t);                                               \
  template void launch_ldlt_panel<T>(T*, const EnvDev&, const int32_t*, int, int, int, int,      \
                                     cudaStream_t);                                              \
  template void launch_ldlt_trail<T>(T*, const EnvDev&, const int32_t*, int, int, int, int,      \
                                     cudaStream_t);                                              \
  template void launch_ldlt_xfill<T>(T*, const EnvDev&, const int32_t*, int, int, cudaStream_t); \
  template void launch_ldlt_mnfill<T>(T*, const EnvDev&, int, cudaStream_t);                      \
  template void launch_ldlt_blocks_batch<T>(const BlockItem*, const int32_t*, const int32_t*, int,    \
                                            cudaStream_t, int*, int);                             \
  template int ldlt_blocks_batch_per_sm<T>();                                                     \
  template void launch_ldlt_blocks<T>(T*, const EnvDev&, const int32_t*, const int32_t*, int,     \
                                      int*, cudaStream_t);                                       \
  template int ldlt_blocks_per_sm<T>();
MSP_INST(double)
MSP_INST(float)

// ------------------------------------------------- BF16 storage of factors
// dst = bf16(src), round to nearest even; n a multiple of 4 (whole tiles).
__global__ void k_round_bf16(const float4* __restrict__ src, __nv_bfloat162* __restrict__ dst,
                             int64_t n4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = src[i];
    dst[2 * i] = __floats2bfloat162_rn(v.x, v.y);
    dst[2 * i + 1] = __floats2bfloat162_rn(v.z, v.w);
  }
}

void launch_round_bf16(const float* src, __nv_bfloat16* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t n4 = n / 4;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + 255) / 256, (int64_t)limits().nsm * 8));
  k_round_bf16<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(src),
                                    reinterpret_cast<__nv_bfloat162*>(dst), n4);
}

}  // namespace msp
