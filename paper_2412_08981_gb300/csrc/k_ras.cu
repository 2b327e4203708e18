// Triangular-solve kernels of the msp library (Section 2.2, Eq. 7): the
// restricted additive Schwarz application z = sum_p R0_p^T (L D L^T)^{-1} R_p t
// over the subdomain factors of a smoothed level (the staged, persistent
// k_ras_solve), and the direct solve of the coarsest level's single block on
// a thread-block cluster (k_block_solve_cluster).  The factors are the tiled
// envelopes written by k_dense.cu (layout in msp.h): 64 x 64 row-major
// tiles, diagonal tiles holding L below the diagonal, D on it and the
// transpose of X = L_II^{-1} above it, so that both sweeps are dense tile
// products.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "msp_dense.cuh"
#include "msp_kernels.h"

namespace msp {
namespace {

// -------------------------------------------------------------- RAS solve
// Persistent and warp-specialised.  Each CTA (one per SM) takes the
// subdomains order[b], order[b + G], ... (largest first).  Warp 8 is the
// producer: one lane streams the factor tiles of every subdomain, in the
// order the sweeps consume them, into a ring of shared-memory slots with
// cp.async.bulk, each slot guarded by a "full" mbarrier (transaction count)
// and an "empty" mbarrier (one arrival per consumer warp).  Warps 0-7 are the
// consumers: gather t[dofs] -> y; forward sweep over tile rows
// (y_I = X_II (y_I - sum_{F_I <= J < I} L_IJ y_J)); backward sweep over the column
// tiles, then the diagonal tile (x_I = X_II^T (y_I / D_I - sum_{I < J <= R_I} L_JI^T x_J));
// scatter the owned entries.  Every mbarrier wait is bounded: on expiry it
// records an error bit and goes on (the results are then garbage and the
// host reports MSP_ERR_TIMEOUT); the producer finally waits, bounded, for its
// own copies, so none is in flight when the CTA exits.
// Consumer warps per CTA and CTAs per SM.  FP64 sweeps are ALU-bound: two
// CTAs of 8 consumers, so that one CTA's row sums and barriers overlap the
// other's FMAs on the SM's FP64 pipe.  FP32 and BF16 sweeps are bound by
// latency and HBM: four CTAs of 8 consumers, so that a level's blocks (512 at
// 64^3) take one CTA each rather than leaving CTAs with two to set the time
// (FP32 then runs two ring slots a CTA, enough with four CTAs streaming).
// Levels whose tile band needs more ring slots than that leaves per CTA use
// the wide form (one CTA of 16 consumers per SM) in every precision.
template <typename T, bool Wide> struct RasCfg { static constexpr int NCW = 16, CTAS = 1; };
template <> struct RasCfg<double, false> { static constexpr int NCW = 8, CTAS = 2; };
template <> struct RasCfg<float, false> { static constexpr int NCW = 8, CTAS = 4; };
template <> struct RasCfg<__nv_bfloat16, false> { static constexpr int NCW = 8, CTAS = 4; };
constexpr long kWaitLimit = 1L << 20;

__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of `parity` to complete.  After a first expiry
// (flag set) later waits give up almost at once.
__device__ inline void mbar_wait(uint64_t* bar, uint32_t parity, volatile int* sflag, int* err, long limit0) {
  const long limit = *sflag ? 64 : limit0;
  for (long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return;
  *sflag = 1;
  atomicOr(err, 4);
}
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
template <int NCW>
__device__ inline void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NCW * 32) : "memory"); }

// FP32 / BF16 tiles: a lane takes contiguous entries of a tile row, so that
// one shared-memory load brings several (16 bytes: 8 BF16 or 4 FP32 entries),
// where one entry per load left these sweeps bound by load instructions.
__device__ __forceinline__ void load8(const float* p, float (&e)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w; e[4] = b.x; e[5] = b.y; e[6] = b.z; e[7] = b.w;
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ void load8(const __nv_bfloat16* p, float (&e)[8]) {
  const uint4 w = *reinterpret_cast<const uint4*>(p);
  e[0] = bf16_lo(w.x); e[1] = bf16_hi(w.x); e[2] = bf16_lo(w.y); e[3] = bf16_hi(w.y);
  e[4] = bf16_lo(w.z); e[5] = bf16_hi(w.z); e[6] = bf16_lo(w.w); e[7] = bf16_hi(w.w);
}
__device__ __forceinline__ float2 load2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 load2(const __nv_bfloat16* p) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
  return make_float2(bf16_lo(w), bf16_hi(w));
}

// Per-subdomain envelope metadata staged in shared memory (one copy for the
// producer, which runs ahead, one for the consumers): F_I, R_I and the tile
// index of (I, F_I), so that no tile address needs a global-memory lookup.
struct MetaSm {
  int32_t* first;
  int32_t* last;
  int32_t* toff;
};

// All 32 lanes of the calling warp load the metadata of subdomain p.
__device__ inline void load_meta(const EnvDev& E, int p, int NT, MetaSm m, int lane) {
  const int rb = E.trow[p];
  for (int I = lane; I < NT; I += 32) {
    m.first[I] = E.first[rb + I];
    m.last[I] = E.last[rb + I];
    m.toff[I] = E.toff[rb + I];
  }
}

// One launch may serve the same level of several instances (a batch): every
// work item is (view v, block p), encoded (v << kViewShift) | p in the CTA
// lists; view v gives the level's factors, envelope, subdomains, Dirichlet
// nodes and error word, and vecs.t[v] / vecs.z[v] its input and output
// (vecs.z[v] == NULL: the view sits this launch out -- its items are skipped
// by producer and consumers alike).  A block's arithmetic does not depend on
// the launch it is part of.
template <typename T, int NCW, int CTAS>
__global__ void __launch_bounds__(32 * (NCW + 1), CTAS) k_ras_solve(
    const RasView* __restrict__ views, int nviews, const __grid_constant__ RasVecs vecs,
    const int32_t* __restrict__ cta_ptr, const int32_t* __restrict__ cta_list, int add, int max_nt,
    int nslot, int inject, int* __restrict__ claim, int nbins) {
  using AT = typename Acc<T>::type;
  constexpr int kConsumers = NCW;
  // inject != 0 (failure-injection tests only): the producer issues no copies,
  // so every wait on a full slot runs out after a short limit; no copy is
  // ever in flight, the output is meaningless and bit 4 of *err is set
  const long wlim = inject ? 4096 : kWaitLimit;
  constexpr uint32_t kTileBytes = TE * sizeof(T);
  constexpr int NC = kConsumers * 32;       // consumer threads
  constexpr int RW = 64 / kConsumers;       // tile rows per consumer warp
  constexpr int NPASS = RW / 4;             // 4-row passes of a warp (8 lanes per row)
  constexpr int CH = kConsumers / 8;        // column halves of the column-wise products (1 or 2)
  constexpr int NB = 2 / CH;                // 32-column sets per lane in those products
  static_assert(RW % 4 == 0 && (CH == 1 || CH == 2), "8 or 16 consumer warps");
  extern __shared__ __align__(128) unsigned char smraw[];
  T* ring = reinterpret_cast<T*>(smraw);                                        // [nslot][TE]
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + (size_t)nslot * kTileBytes);  // [nslot]
  uint64_t* empty = full + nslot;                                               // [nslot]
  AT* y = reinterpret_cast<AT*>(empty + nslot);                                 // [max_nt*64]
  AT* acc = y + max_nt * 64;                                                    // [64]
  AT* part = acc + 64;                                                          // [kConsumers][64]
  AT* red = part + kConsumers * 64;                                             // [64][9] row partials (8 a row)
  int32_t* meta = reinterpret_cast<int32_t*>(red + 64 * 9);                     // [2][3][max_nt]
  const MetaSm pm{meta, meta + max_nt, meta + 2 * max_nt};                      // producer's
  const MetaSm cm{meta + 3 * max_nt, meta + 4 * max_nt, meta + 5 * max_nt};    // consumers'
  __shared__ int sflag;
  __shared__ int slist;  // the work list this CTA takes
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int rl = lane >> 3, g = lane & 7;            // row within a 4-row pass, lane within the row
  const int hh = warp % CH, rb = warp / CH;          // column half and 8-row block of the column-wise products
  const int G = gridDim.x;
  if (tid == 0) {
    sflag = 0;
    for (int s = 0; s < nslot; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // claim == nullptr: list blockIdx.x.  Else the lists come per_sm to an SM
    // (the host balanced the SMs' sums, then split each over its CTAs): a
    // CTA takes list (its SM, its arrival rank there); one whose list is
    // taken, or whose SM holds more CTAs than that, takes the first list no
    // one has.  There are as many lists as CTAs, so each is taken once.
    // claim[0, nbins): arrivals per SM, claim[nbins, nbins + G): list taken.
    int lid = blockIdx.x;
    if (claim != nullptr) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      const int b = (int)(smid % (unsigned)nbins), per = gridDim.x / nbins;
      const int rank = atomicAdd(&claim[b], 1);
      lid = -1;
      if (rank < per && atomicExch(&claim[nbins + b * per + rank], 1) == 0) lid = b * per + rank;
      for (int i = 0; lid < 0 && i < (int)gridDim.x; ++i)
        if (atomicExch(&claim[nbins + i], 1) == 0) lid = i;
    }
    slist = lid;
  }
  __syncthreads();
  const int mylist = slist;

  int* err = views[0].err;  // the error word of the item in hand
  if (warp == kConsumers) {  // ------------------------------------ producer
    long seq = 0;
    auto issue = [&](const T* src) {
      const int slot = (int)(seq % nslot);
      if (seq >= nslot) mbar_wait(&empty[slot], (uint32_t)(((seq / nslot) - 1) & 1), &sflag, err, wlim);
      if (!inject) {
        mbar_expect_tx(&full[slot], kTileBytes);
        bulk_g2s(ring + (size_t)slot * TE, src, kTileBytes, &full[slot]);
      }
      ++seq;
    };
    for (int q = cta_ptr[mylist]; q < cta_ptr[mylist + 1]; ++q) {
      const int vw = cta_list[q] >> kViewShift, p = cta_list[q] & ((1 << kViewShift) - 1);
      if (vecs.z[vw] == nullptr) continue;
      const EnvDev& E = views[vw].E;
      err = views[vw].err;
      const int NT = E.nt[p];
      load_meta(E, p, NT, pm, lane);
      __syncwarp();
      if (lane == 0) {
        const T* base = static_cast<const T*>(views[vw].fac) + E.fac_off[p];
        for (int I = 0; I < NT; ++I) {
          const T* row = base + (int64_t)pm.toff[I] * TE;
          for (int J = pm.first[I]; J <= I; ++J) issue(row + (int64_t)(J - pm.first[I]) * TE);
        }
        for (int I = NT - 1; I >= 0; --I) {
          for (int J = I + 1; J <= pm.last[I]; ++J)
            issue(base + (int64_t)(pm.toff[J] + (I - pm.first[J])) * TE);
          issue(base + (int64_t)(pm.toff[I] + (I - pm.first[I])) * TE);
        }
      }
      __syncwarp();
    }
    // drain: the last copy of every slot has landed before the CTA may exit
    if (lane == 0)
      for (long k = (seq > nslot ? seq - nslot : 0); k < seq; ++k)
        mbar_wait(&full[k % nslot], (uint32_t)((k / nslot) & 1), &sflag, err, wlim);
    return;
  }

  // ------------------------------------------------------------ consumers
  for (int vw = 0; vw < nviews; ++vw) {
    const double* t = vecs.t[vw];
    double* z = vecs.z[vw];
    if (z == nullptr) continue;
    const int32_t* dir_list = views[vw].dir_list;
    for (int d = blockIdx.x * NC + tid; d < views[vw].ndir; d += G * NC) {
      const int g = dir_list[d];
      z[g] = add ? z[g] + t[g] : t[g];
    }
  }
  long seq = 0;
  auto acquire = [&]() -> const T* {
    const int slot = (int)(seq % nslot);
    mbar_wait(&full[slot], (uint32_t)((seq / nslot) & 1), &sflag, err, wlim);
    return ring + (size_t)slot * TE;
  };
  auto release = [&]() {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[seq % nslot]);
    ++seq;
  };
  for (int q = cta_ptr[mylist]; q < cta_ptr[mylist + 1]; ++q) {
    const int vw = cta_list[q] >> kViewShift, p = cta_list[q] & ((1 << kViewShift) - 1);
    const double* __restrict__ t = vecs.t[vw];
    double* __restrict__ z = vecs.z[vw];
    if (z == nullptr) continue;
    const EnvDev& E = views[vw].E;
    const int32_t* __restrict__ sub_ptr = views[vw].sub_ptr;
    const int32_t* __restrict__ dofs = views[vw].dofs;
    const uint8_t* __restrict__ own = views[vw].own;
    err = views[vw].err;
    const int NT = E.nt[p];
    const int off = sub_ptr[p];
    const int np_ = sub_ptr[p + 1] - off;
    if (warp == 0) load_meta(E, p, NT, cm, lane);
    for (int li = tid; li < NT * 64; li += NC) y[li] = (li < np_) ? (AT)t[dofs[off + li]] : AT(0);
    consumers_sync<kConsumers>();
    // forward sweep
    for (int I = 0; I < NT; ++I) {
      // off-diagonal tiles: lane (rl, g) of a warp takes row warp*RW + 4*ps + rl
      // of pass ps and the columns 8*((c + rl) & 7) + g, c = 0..7 (the four
      // rows of an access read four different 8-column chunks, so the loads
      // spread over all banks); two FMA chains per row, 8 partials per row
      AT se[NPASS], so[NPASS];
#pragma unroll
      for (int k = 0; k < NPASS; ++k) se[k] = so[k] = 0;
      for (int J = cm.first[I]; J < I; ++J) {
        const T* tl = acquire();
        const AT* yJ = y + J * 64;
#pragma unroll
        for (int ps = 0; ps < NPASS; ++ps) {
          const T* trow = tl + (warp * RW + 4 * ps + rl) * 64;
          if constexpr (sizeof(T) < sizeof(double)) {  // columns 8g .. 8g + 7
            AT e[8];
            load8(trow + 8 * g, e);
            const float4 ya = *reinterpret_cast<const float4*>(yJ + 8 * g);
            const float4 yb = *reinterpret_cast<const float4*>(yJ + 8 * g + 4);
            se[ps] = fma(e[0], ya.x, se[ps]);
            so[ps] = fma(e[1], ya.y, so[ps]);
            se[ps] = fma(e[2], ya.z, se[ps]);
            so[ps] = fma(e[3], ya.w, so[ps]);
            se[ps] = fma(e[4], yb.x, se[ps]);
            so[ps] = fma(e[5], yb.y, so[ps]);
            se[ps] = fma(e[6], yb.z, se[ps]);
            so[ps] = fma(e[7], yb.w, so[ps]);
          } else {
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
              const int c0 = 8 * ((c + rl) & 7) + g, c1 = 8 * ((c + 1 + rl) & 7) + g;
              se[ps] = fma((AT)trow[c0], yJ[c0], se[ps]);
              so[ps] = fma((AT)trow[c1], yJ[c1], so[ps]);
            }
          }
        }
        release();
      }
      // row sums: one thread per row adds the 8 lane partials (a shared-memory
      // transpose costs far fewer FP64 instructions than warp shuffles)
#pragma unroll
      for (int ps = 0; ps < NPASS; ++ps) red[(warp * RW + 4 * ps + rl) * 9 + g] = se[ps] + so[ps];
      consumers_sync<kConsumers>();
      if (tid < 64) {
        const AT* rr = red + tid * 9;
        const AT v0 = (rr[0] + rr[2]) + (rr[4] + rr[6]), v1 = (rr[1] + rr[3]) + (rr[5] + rr[7]);
        acc[tid] = y[I * 64 + tid] - (v0 + v1);
      }
      consumers_sync<kConsumers>();
      {  // y_I = X acc, X[b][a] = tile[a][b] for a < b: warp (rb, h) takes rows
         // a = 8 rb .. 8 rb + 7 and its columns b; (row, column set) pairs with
         // no a < b are skipped by the whole warp
        const T* dt = acquire();
        if constexpr (sizeof(T) < sizeof(double) && CH == 1) {  // columns 2 lane, 2 lane + 1
          const int b = 2 * lane;
          AT v0 = 0, v1 = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int a = rb * 8 + k;
            if (a < b + 1) {
              const float2 x = load2(dt + a * 64 + b);
              if (a < b) v0 = fma(x.x, acc[a], v0);
              v1 = fma(x.y, acc[a], v1);
            }
          }
          *reinterpret_cast<float2*>(part + rb * 64 + b) = make_float2(v0, v1);
        } else if constexpr (CH == 1) {
          // FP64, 8 warps: the 2016 products of the strict triangle in 64 warp
          // instructions with every lane busy (an FP64 warp instruction costs
          // the same with idle lanes).  Column halves 0..31 and 32..63:
          //  * rows a < 32 of the right half are full: lane l, column 32 + l;
          //  * the triangles (rows 0..30 of the left half, 32..62 of the right)
          //    pair row p with row 30 - p of the same half: lane l takes column
          //    l of row p when l > p, else column 31 - l of row 30 - p, which
          //    are exactly the columns above the diagonal; row 15 (47) goes alone.
          // Warp w: left pairs 2w, 2w + 1 (15: the single row), right full rows
          // 4w .. 4w + 3, right pairs 2w, 2w + 1.  A lane keeps its own column's
          // sums (d) and its mirror column's (m); the mirror sums reach their
          // column's lane by a shuffle.
          AT d0 = 0, m0 = 0, d1 = 0, m1 = 0;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int pr = 2 * rb + k;  // pair index 0..15
            const bool dir = lane > pr, on = dir || pr < 15;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              // one FMA for the whole warp: the operands and the accumulator are
              // selected per lane, not branched on
              const int c = 32 * half;
              const int row = dir ? c + pr : c + 30 - pr;
              const int col = dir ? c + lane : c + 31 - lane;
              const AT x = on ? (AT)dt[row * 64 + col] : AT(0);
              AT& dh = half == 0 ? d0 : d1;
              AT& mh = half == 0 ? m0 : m1;
              const AT t = fma(x, acc[row], dir ? dh : mh);
              dh = dir ? t : dh;
              mh = dir ? mh : t;
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int a = 4 * rb + k;
            d1 = fma((AT)dt[a * 64 + 32 + lane], acc[a], d1);
          }
          part[rb * 64 + lane] = d0 + __shfl_sync(0xffffffffu, m0, 31 - lane);
          part[rb * 64 + 32 + lane] = d1 + __shfl_sync(0xffffffffu, m1, 31 - lane);
        } else {
          AT v[NB];
#pragma unroll
          for (int q = 0; q < NB; ++q) v[q] = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int a = rb * 8 + k;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
              const int b0 = (CH == 2 ? 32 * hh : 32 * q);
              if (a < b0 + 31) {
                const int b = b0 + lane;
                if (a < b) v[q] = fma((AT)dt[a * 64 + b], acc[a], v[q]);
              }
            }
          }
#pragma unroll
          for (int q = 0; q < NB; ++q) part[rb * 64 + (CH == 2 ? 32 * hh : 32 * q) + lane] = v[q];
        }
        release();
      }
      consumers_sync<kConsumers>();
      if (tid < 64) {
        const AT v0 = (part[tid] + part[128 + tid]) + (part[256 + tid] + part[384 + tid]);
        const AT v1 = (part[64 + tid] + part[192 + tid]) + (part[320 + tid] + part[448 + tid]);
        y[I * 64 + tid] = acc[tid] + (v0 + v1);
      }
      consumers_sync<kConsumers>();
    }
    // backward sweep: the column tiles of row I, then its diagonal tile (no
    // tile is held while another streams in, so two ring slots suffice)
    for (int I = NT - 1; I >= 0; --I) {
      // off-diagonal tiles (transposed): warp (rb, h) takes rows 8 rb .. 8 rb + 7
      // of L_JI and its columns; 8 partials per column
      AT s[NB][2];
#pragma unroll
      for (int q = 0; q < NB; ++q) s[q][0] = s[q][1] = 0;
      for (int J = I + 1; J <= cm.last[I]; ++J) {
        const T* tl = acquire();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int r = rb * 8 + k;
          const AT xr = y[J * 64 + r];
          if constexpr (sizeof(T) < sizeof(double) && CH == 1) {  // columns 2 lane, 2 lane + 1
            const float2 x = load2(tl + r * 64 + 2 * lane);
            s[0][k & 1] = fma(x.x, xr, s[0][k & 1]);
            s[1][k & 1] = fma(x.y, xr, s[1][k & 1]);
          } else {
#pragma unroll
            for (int q = 0; q < NB; ++q)
              s[q][k & 1] = fma((AT)tl[r * 64 + (CH == 2 ? 32 * hh : 32 * q) + lane], xr, s[q][k & 1]);
          }
        }
        release();
      }
      if constexpr (sizeof(T) < sizeof(double) && CH == 1) {
        *reinterpret_cast<float2*>(part + rb * 64 + 2 * lane) = make_float2(s[0][0] + s[0][1], s[1][0] + s[1][1]);
      } else {
#pragma unroll
        for (int q = 0; q < NB; ++q) part[rb * 64 + (CH == 2 ? 32 * hh : 32 * q) + lane] = s[q][0] + s[q][1];
      }
      consumers_sync<kConsumers>();
      const T* dt = acquire();  // the diagonal tile, released after its product
      if (tid < 64) {
        const AT v0 = (part[tid] + part[128 + tid]) + (part[256 + tid] + part[384 + tid]);
        const AT v1 = (part[64 + tid] + part[192 + tid]) + (part[320 + tid] + part[448 + tid]);
        acc[tid] = y[I * 64 + tid] / (AT)dt[tid * 65] - (v0 + v1);
      }
      consumers_sync<kConsumers>();
      // x_I[a] = acc[a] + sum_{b>a} tile[a][b] acc[b]: lane (rl, g) takes row
      // a = warp*RW + 4*ps + rl and the columns 8c + g; chunks c with no b > a
      // for the pass's four rows are skipped by the whole warp
#pragma unroll
      for (int ps = 0; ps < NPASS; ++ps) {
        const int amin = warp * RW + 4 * ps, a = amin + rl;
        AT e0 = 0, e1 = 0;
        if constexpr (sizeof(T) < sizeof(double)) {  // columns 8g .. 8g + 7
          if (8 * g + 7 > a) {
            AT e[8], av[8];
            load8(dt + a * 64 + 8 * g, e);
            load8(acc + 8 * g, av);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (8 * g + u > a) {
                if (u & 1)
                  e1 = fma(e[u], av[u], e1);
                else
                  e0 = fma(e[u], av[u], e0);
              }
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (8 * c + 7 > amin) {
              const int b = 8 * c + g;
              if (b > a) {
                if (c & 1)
                  e1 = fma((AT)dt[a * 64 + b], acc[b], e1);
                else
                  e0 = fma((AT)dt[a * 64 + b], acc[b], e0);
              }
            }
          }
        }
        red[a * 9 + g] = e0 + e1;
      }
      release();
      consumers_sync<kConsumers>();
      if (tid < 64) {
        const AT* rr = red + tid * 9;
        const AT v0 = (rr[0] + rr[2]) + (rr[4] + rr[6]), v1 = (rr[1] + rr[3]) + (rr[5] + rr[7]);
        y[I * 64 + tid] = acc[tid] + (v0 + v1);
      }
      consumers_sync<kConsumers>();
    }
    for (int li = tid; li < np_; li += NC) {
      if (own[off + li]) {
        const int g = dofs[off + li];
        z[g] = add ? z[g] + (double)y[li] : (double)y[li];
      }
    }
    consumers_sync<kConsumers>();
  }
}

// ------------------------------------------- single-block solve on a cluster
// The coarsest level is one block (one CTA would use one SM's FP64 pipe), so
// its sweeps run on a cluster of CL CTAs of NW = 64 / CL warps.  Every CTA
// keeps the whole right-hand side / solution vector in its shared memory;
// CTA c owns the rows r0 .. r0 + NW - 1 (r0 = NW c) of every tile row, one
// per warp, and sends what it computes for them to every CTA (distributed
// shared memory) before a cluster barrier.
//
// Forward sweep of L y = t by tile rows, acc_I = t_I - sum_{J<I} L_IJ y_J and
// y_I = X_I acc_I (X_I = L_II^{-1}, kept in the diagonal tile).  With the
// coupling tile M_I = L_{I,I-1} X_{I-1}, the term of the newest row is
// L_{I,I-1} y_{I-1} = M_I acc_{I-1}, so step I forms acc_I from acc_{I-1}
// and y_J, J <= I - 2, and in the same pass y_{I-1} = X_{I-1} acc_{I-1}: one
// exchange per tile row.  Backward (L^T x = D^{-1} y), with N_I = X_{I+1}
// L_{I+1,I}: acc_I = y_I / d - sum_{J>I} L_JI^T x_J, the newest term
// L_{I+1,I}^T x_{I+1} = N_I^T acc_{I+1}, and x_{I+1} = X_{I+1}^T acc_{I+1}.
// Every step keeps on its critical path only the two newest tiles' products
// (in registers, loaded the step before) and one reduction of two sums over
// the warp: the older tiles' sums are formed between the arrive and the wait
// of the previous step's cluster barrier.  Cluster v of the grid solves view
// v (the coarsest block of one instance of a batch); a cluster whose
// vecs.z[v] is NULL leaves at once, all its CTAs together.
constexpr int kCl = 8;

// The non-aligned forms: a warp may reach the barrier still diverged from
// its sends (lanes 0..CL-1 and 16..16+CL-1 store), and every lane's stores
// must be ordered before its own arrival.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Shared memory of one CTA: the vector, acc double-buffered, the backward
// column partials double-buffered.
template <int CL>
size_t block_solve_smem_cl(int max_nt) {
  constexpr int NW = 64 / CL, NTH = 32 * NW;
  const size_t dbl = (size_t)max_nt * 64 + 128 + 2 * 32 * NW + 2 * 16 * NTH;
  return dbl * sizeof(double) + ((size_t)3 * max_nt * sizeof(int) + 15) / 16 * 16;
}

// One element copied global -> shared without passing through registers, so
// that no later release (the cluster barrier's arrive) has to wait for it;
// cp_stage_wait makes this thread's copies visible to it.
template <typename T>
__device__ __forceinline__ void cp_stage(T* dst, const T* src) {
  static_assert(sizeof(T) == 8 || sizeof(T) == 4, "4- or 8-byte elements");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_stage_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T, int CL>
__global__ void __launch_bounds__(32 * (64 / CL), 1) k_block_solve_cluster(const RasView* __restrict__ views,
                                                                        const __grid_constant__ RasVecs vecs,
                                                                        int add) {
  constexpr int NW = 64 / CL, NTH = 32 * NW;
  static_assert(CL >= 4 && CL <= 16, "lanes 0..CL-1 and 16..16+CL-1 send the two sums");
  using AT = typename Acc<T>::type;
  constexpr int kPre = 4;  // older tiles of a prep held in registers at once
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int me = (int)cl.block_rank();
  const int vw = blockIdx.x / CL;
  const double* __restrict__ t = vecs.t[vw];
  double* __restrict__ z = vecs.z[vw];
  if (z == nullptr) return;
  const T* __restrict__ fac = static_cast<const T*>(views[vw].fac);
  const EnvDev& E = views[vw].E;
  const int32_t* __restrict__ sub_ptr = views[vw].sub_ptr;
  const int32_t* __restrict__ dofs = views[vw].dofs;
  const int32_t* __restrict__ dir_list = views[vw].dir_list;
  const int ndir = views[vw].ndir;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p = 0;
  const int NT = E.nt[p], rb = E.trow[p];
  const int off = sub_ptr[p], np_ = sub_ptr[p + 1] - off;
  extern __shared__ unsigned char smraw[];
  AT* y = reinterpret_cast<AT*>(smraw);  // [NT*64] the whole vector, in every CTA
  AT* acc = y + NT * 64;                 // [2][64] acc of the newest tile row, by parity
  AT* redp = acc + 128;                  // [2][32][NW] backward partials: row pair, column
  AT* stg = redp + 2 * 32 * NW;          // [2][16][NTH] this thread's staged loads, by step parity
  int* efirst = reinterpret_cast<int*>(stg + 2 * 16 * NTH);  // [NT] F_I, R_I, tile offsets
  int* elast = efirst + NT;
  int* etoff = elast + NT;
  static_assert(sizeof(T) == sizeof(AT), "staged copies keep the factor's element type");
  const T* base = fac + E.fac_off[p];
  const T* Mt = fac + E.fac_off[p + 1];      // M_I at tile I
  const T* Nt = Mt + (int64_t)NT * TE;       // N_I^T at tile I
  const T* Dinv = Nt + (int64_t)NT * TE;     // 1/d, 64 per tile row
  for (int d = me * NTH + tid; d < ndir; d += CL * NTH) {
    const int g = dir_list[d];
    z[g] = add ? z[g] + t[g] : t[g];
  }
  for (int li = tid; li < NT * 64; li += NTH) y[li] = (li < np_) ? (AT)t[dofs[off + li]] : AT(0);
  for (int i = tid; i < NT; i += NTH) {
    efirst[i] = E.first[rb + i];
    elast[i] = E.last[rb + i];
    etoff[i] = E.toff[rb + i];
  }
  cl.sync();
  const int r = NW * me + warp;  // this warp's row (forward), column of acc and row of x (backward)
  auto tile = [&](int I, int J) { return base + (int64_t)(etoff[I] + (J - efirst[I])) * TE; };
  auto S = [&](int b, int slot) -> AT& { return stg[(b * 16 + slot) * NTH + tid]; };
  // Sum over the warp of a (lanes < 16 end with it) and of b (lanes >= 16):
  // the first level halves the lanes of each, so the two take 5 adds.
  auto reduce2 = [&](AT a, AT b) {
    const bool hi = lane & 16;
    AT v = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  // ---- forward: step I = 0 .. NT forms acc_I (I < NT) and y_{I-1} (I >= 1)
  // Prepared for step I: the lane sums over the tiles F_I <= J < I - 2, row r
  // of tile (I, I - 2) and of M_I (where they exist), this lane's entries of
  // row r of X_{I-1} (X[r][a] = dt[a][r], a < r).
  AT f0 = 0, f1 = 0, l20 = 0, l21 = 0, m0 = 0, m1 = 0, x0 = 0, x1 = 0;
  bool h2 = false, h1 = false;
  // Loads run two steps ahead of their use, as asynchronous copies into this
  // thread's staging slots (buffer = step parity): step I's gap finishes step
  // I + 1 from its slots and starts the copies of step I + 2, and no cluster
  // barrier's release waits on a copy in flight.  Slots: 2q, 2q + 1 the older
  // tiles, 8-9 tile (I, I - 2), 10-11 M_I, 12-13 X_{I-1}.
  int qF = 0, qnJ = 0;
  bool qh2 = false, qh1 = false;
  auto load_fwd = [&](int I) {  // the copies of step I (0 <= I <= NT)
    const int b = I & 1;
    qh2 = qh1 = false;
    qF = 0;
    qnJ = 0;
    if (I < NT) {
      qF = efirst[I];
      qnJ = I - 2 - qF;
#pragma unroll
      for (int q = 0; q < kPre; ++q)
        if (q < qnJ) {
          const T* tl = tile(I, qF + q);
          cp_stage(&S(b, 2 * q), tl + r * 64 + lane);
          cp_stage(&S(b, 2 * q + 1), tl + r * 64 + lane + 32);
        }
      qh2 = I - 2 >= qF;
      if (qh2) {
        const T* tl = tile(I, I - 2);
        cp_stage(&S(b, 8), tl + r * 64 + lane);
        cp_stage(&S(b, 9), tl + r * 64 + lane + 32);
      }
      qh1 = I - 1 >= qF;
      if (qh1) {
        const T* mt = Mt + (int64_t)I * TE;
        cp_stage(&S(b, 10), mt + r * 64 + lane);
        cp_stage(&S(b, 11), mt + r * 64 + lane + 32);
      }
    }
    if (I >= 1) {
      const T* dt = tile(I - 1, I - 1);
      if (lane < r) cp_stage(&S(b, 12), dt + lane * 64 + r);
      if (lane + 32 < r) cp_stage(&S(b, 13), dt + (lane + 32) * 64 + r);
    }
    cp_stage_commit();
  };
  auto finish_fwd = [&](int I) {  // step I's operands from its copies; reads y_J, J < I - 2
    const int b = I & 1;
    cp_stage_wait();
    h2 = qh2;
    h1 = qh1;
    l20 = h2 ? S(b, 8) : AT(0);
    l21 = h2 ? S(b, 9) : AT(0);
    m0 = h1 ? S(b, 10) : AT(0);
    m1 = h1 ? S(b, 11) : AT(0);
    x0 = (I >= 1 && lane < r) ? S(b, 12) : AT(0);
    x1 = (I >= 1 && lane + 32 < r) ? S(b, 13) : AT(0);
    f0 = f1 = AT(0);
    if (I < NT) {  // step NT forms y_{NT-1} only
      AT s0 = 0, s1 = 0;
#pragma unroll
      for (int q = 0; q < kPre; ++q)
        if (q < qnJ) {
          s0 = fma(S(b, 2 * q), y[(qF + q) * 64 + lane], s0);
          s1 = fma(S(b, 2 * q + 1), y[(qF + q) * 64 + lane + 32], s1);
        }
      for (int J = qF + kPre; J < I - 2; ++J) {  // bands wider than kPre + 2 tiles
        const T* tl = tile(I, J);
        s0 = fma((AT)tl[r * 64 + lane], y[J * 64 + lane], s0);
        s1 = fma((AT)tl[r * 64 + lane + 32], y[J * 64 + lane + 32], s1);
      }
      f0 = s0;
      f1 = s1;
    }
  };
  load_fwd(0);
  finish_fwd(0);
  if (NT >= 1) load_fwd(1);
  for (int I = 0; I <= NT; ++I) {
    const AT* ap = acc + ((I + 1) & 1) * 64;  // acc_{I-1}
    AT* an = acc + (I & 1) * 64;              // acc_I
    AT a0 = f0, a1 = f1;
    if (h2) {
      a0 = fma(l20, y[(I - 2) * 64 + lane], a0);
      a1 = fma(l21, y[(I - 2) * 64 + lane + 32], a1);
    }
    if (h1) {
      a0 = fma(m0, ap[lane], a0);
      a1 = fma(m1, ap[lane + 32], a1);
    }
    const AT yv = I >= 1 ? fma(x1, ap[lane + 32], x0 * ap[lane]) : AT(0);
    const AT v = reduce2(a0 + a1, yv);
    if (I < NT && lane < CL) cl.map_shared_rank(an, lane)[r] = y[I * 64 + r] - v;
    if (I >= 1 && lane >= 16 && lane < 16 + CL) cl.map_shared_rank(y, lane - 16)[(I - 1) * 64 + r] = ap[r] + v;
    // the next step's sums while the sends travel (the arrive's release
    // waits for them); then the copies two steps ahead, after the arrive
    if (I < NT) finish_fwd(I + 1);  // reads y_J, J < I - 1: final; the exchange writes y_{I-1} and acc_I
    cluster_arrive();
    if (I + 2 <= NT) load_fwd(I + 2);
    cluster_wait();
  }
  // ---- backward: step I = NT - 1 .. -1 forms acc_I (I >= 0) and x_{I+1} (I + 1 < NT)
  // Prepared for step I: this thread's partial of column r0 + (tid % NW) over
  // rows 2 (tid / NW), 2 (tid / NW) + 1 of the tiles I + 3 <= J <= R_I (into
  // redp), this lane's entries of column r of tile (I + 2, I) and of N_I^T's
  // row r, of row r of X_{I+1}^T (dt[r][b], b > r), and y_I[r] / d_r.
  const int pc = tid % NW, prg = tid / NW, pcol = NW * me + pc;
  AT bl0 = 0, bl1 = 0, bn0 = 0, bn1 = 0, bx0 = 0, bx1 = 0, bq = 0;
  bool bh2 = false, bh1 = false;
  // as forward: copies two steps ahead.  Slots: 2q, 2q + 1 the older tiles'
  // column entries, 8-9 tile (I + 2, I), 10-11 N_I^T, 12-13 X_{I+1}^T, 14 1/d.
  int qR = -1, qbnJ = 0;
  bool qbh2 = false, qbh1 = false;
  auto load_bwd = [&](int I) {  // the copies of step I (-1 <= I <= NT - 1)
    const int b = I & 1;
    qbh2 = qbh1 = false;
    qR = -1;
    qbnJ = 0;
    if (I >= 0) {
      qR = elast[I];
      qbnJ = qR - (I + 2);
#pragma unroll
      for (int q = 0; q < kPre; ++q)
        if (q < qbnJ) {
          const T* tl = tile(I + 3 + q, I);
          cp_stage(&S(b, 2 * q), tl + (2 * prg) * 64 + pcol);
          cp_stage(&S(b, 2 * q + 1), tl + (2 * prg + 1) * 64 + pcol);
        }
      qbh2 = I + 2 <= qR;
      if (qbh2) {
        const T* tl = tile(I + 2, I);
        cp_stage(&S(b, 8), tl + lane * 64 + r);
        cp_stage(&S(b, 9), tl + (lane + 32) * 64 + r);
      }
      qbh1 = I + 1 <= qR;
      if (qbh1) {
        const T* nt = Nt + (int64_t)I * TE;
        cp_stage(&S(b, 10), nt + r * 64 + lane);
        cp_stage(&S(b, 11), nt + r * 64 + lane + 32);
      }
      cp_stage(&S(b, 14), Dinv + I * 64 + r);
    }
    if (I + 1 < NT) {
      const T* dt = tile(I + 1, I + 1);
      if (lane > r) cp_stage(&S(b, 12), dt + r * 64 + lane);
      if (lane + 32 > r) cp_stage(&S(b, 13), dt + r * 64 + lane + 32);
    }
    cp_stage_commit();
  };
  auto finish_bwd = [&](int I) {  // step I's operands; reads x_J, J >= I + 3, and the forward y_I
    const int b = I & 1;
    cp_stage_wait();
    bh2 = qbh2;
    bh1 = qbh1;
    bl0 = bh2 ? S(b, 8) : AT(0);
    bl1 = bh2 ? S(b, 9) : AT(0);
    bn0 = bh1 ? S(b, 10) : AT(0);
    bn1 = bh1 ? S(b, 11) : AT(0);
    bx0 = (I + 1 < NT && lane > r) ? S(b, 12) : AT(0);
    bx1 = (I + 1 < NT && lane + 32 > r) ? S(b, 13) : AT(0);
    if (I >= 0) {
      AT v = 0;
#pragma unroll
      for (int q = 0; q < kPre; ++q)
        if (q < qbnJ) {
          const int J = I + 3 + q;
          v = fma(S(b, 2 * q), y[J * 64 + 2 * prg], v);
          v = fma(S(b, 2 * q + 1), y[J * 64 + 2 * prg + 1], v);
        }
      for (int J = I + 3 + kPre; J <= qR; ++J) {  // bands wider than kPre + 2 tiles
        const T* tl = tile(J, I);
        v = fma((AT)tl[(2 * prg) * 64 + pcol], y[J * 64 + 2 * prg], v);
        v = fma((AT)tl[(2 * prg + 1) * 64 + pcol], y[J * 64 + 2 * prg + 1], v);
      }
      redp[(I & 1) * 32 * NW + prg * NW + pc] = v;
      bq = S(b, 14) * y[I * 64 + r];
    }
  };
  load_bwd(NT - 1);
  finish_bwd(NT - 1);
  if (NT - 2 >= -1) load_bwd(NT - 2);
  __syncthreads();  // its partials in redp
  for (int I = NT - 1; I >= -1; --I) {
    const AT* ap = acc + ((I + 1) & 1) * 64;  // acc_{I+1}
    AT* an = acc + (I & 1) * 64;              // acc_I
    AT a = 0;
    if (I >= 0) {
      a = redp[(I & 1) * 32 * NW + lane * NW + warp];  // rows 2 lane, 2 lane + 1 of the older tiles
      if (bh2) {
        a = fma(bl0, y[(I + 2) * 64 + lane], a);
        a = fma(bl1, y[(I + 2) * 64 + lane + 32], a);
      }
      if (bh1) {
        a = fma(bn0, ap[lane], a);
        a = fma(bn1, ap[lane + 32], a);
      }
    }
    const AT xv = I + 1 < NT ? fma(bx1, ap[lane + 32], bx0 * ap[lane]) : AT(0);
    const AT v = reduce2(a, xv);
    if (I >= 0 && lane < CL) cl.map_shared_rank(an, lane)[r] = bq - v;
    if (I + 1 < NT && lane >= 16 && lane < 16 + CL) cl.map_shared_rank(y, lane - 16)[(I + 1) * 64 + r] = ap[r] + v;
    if (I >= 0) finish_bwd(I - 1);  // reads x_J, J >= I + 2, and y_{I-1}: final; the exchange writes x_{I+1}, acc_I
    cluster_arrive();
    if (I - 2 >= -1) load_bwd(I - 2);
    cluster_wait();
    __syncthreads();  // redp is written after the arrive, which orders only what came before it
  }
  for (int li = me * NTH + tid; li < np_; li += CL * NTH) {
    const int g = dofs[off + li];
    z[g] = add ? z[g] + (double)y[li] : (double)y[li];
  }
}

}  // namespace

// Ring depth of the staged solve: as many tile slots as shared memory holds,
// up to 16 (BF16 and FP32 tiles are small; more bytes in flight per SM hide
// more of the HBM latency).
constexpr size_t kMaxSlots = 16;

// Dynamic shared memory one CTA of a k_ras_solve configuration may use.
template <typename T, bool W>
size_t ras_smem_budget() {
  constexpr int C = RasCfg<T, W>::CTAS;
  if (C == 1) return (size_t)limits().smem;
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  return std::min((size_t)limits().smem, (size_t)per_sm / C - 2048);  // per-CTA reservation and static smem
}

template <typename T, bool W>
size_t ras_fixed_bytes(int max_nt) {
  using AT = typename Acc<T>::type;
  return ((size_t)max_nt * 64 + 64 + RasCfg<T, W>::NCW * 64 + 64 * 9) * sizeof(AT) + 6 * (size_t)max_nt * 4;
}

template <typename T, bool W>
int ras_slots_cfg(int max_nt) {
  const size_t fixed = ras_fixed_bytes<T, W>(max_nt);
  const size_t per_slot = (size_t)TE * sizeof(T) + 2 * sizeof(uint64_t);
  const size_t smem = ras_smem_budget<T, W>();
  if (smem <= fixed) return 0;
  return (int)std::min<size_t>(kMaxSlots, (smem - fixed) / per_slot);
}

template <typename T>
int ras_ctas_per_sm(bool wide) {
  return wide ? RasCfg<T, true>::CTAS : RasCfg<T, false>::CTAS;
}

template <typename T>
int ras_slots(int max_nt, bool wide) {
  return wide ? ras_slots_cfg<T, true>(max_nt) : ras_slots_cfg<T, false>(max_nt);
}

template <typename T, bool W>
void launch_ras_cfg(const RasView* views, int nviews, const RasVecs& vecs, const int32_t* cta_ptr,
                    const int32_t* cta_list, int grid, int max_nt, int add, int inject, cudaStream_t s,
                    int* claim, int nbins) {
  constexpr int NCW = RasCfg<T, W>::NCW, CTAS = RasCfg<T, W>::CTAS;
  auto kern = k_ras_solve<T, NCW, CTAS>;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ras_smem_budget<T, W>());
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  });
  const int nslot = ras_slots_cfg<T, W>(max_nt);  // the host checked at set-up that this is enough
  const size_t smem = (size_t)nslot * ((size_t)TE * sizeof(T) + 2 * sizeof(uint64_t)) + ras_fixed_bytes<T, W>(max_nt);
  if (grid < 1 || nviews < 1) return;
  kern<<<grid, 32 * (NCW + 1), smem, s>>>(views, nviews, vecs, cta_ptr, cta_list, add, max_nt, nslot, inject, claim,
                                          nbins);
}

template <typename T>
void launch_ras_solve(const RasView* views, int nviews, const RasVecs& vecs, const int32_t* cta_ptr,
                      const int32_t* cta_list, int grid, int max_nt, int add, bool wide, cudaStream_t s,
                      int inject, int* claim, int nbins) {
  if (wide)
    launch_ras_cfg<T, true>(views, nviews, vecs, cta_ptr, cta_list, grid, max_nt, add, inject, s, claim, nbins);
  else
    launch_ras_cfg<T, false>(views, nviews, vecs, cta_ptr, cta_list, grid, max_nt, add, inject, s, claim, nbins);
}

size_t block_solve_cluster_smem(int max_nt) { return block_solve_smem_cl<kCl>(max_nt); }

// One launch of the cluster solve with CL CTAs a cluster.
template <typename T, int CL>
cudaError_t launch_block_solve_cl(const RasView* views, int nviews, const RasVecs& vecs, int max_nt, int add,
                                  cudaStream_t s, bool query_only = false) {
  auto kern = k_block_solve_cluster<T, CL>;
  const size_t smem = block_solve_smem_cl<CL>(max_nt);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limits().smem);
    if (CL > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL * std::max(nviews, 1), 1, 1);
  cfg.blockDim = dim3(32 * (64 / CL), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr1[1];
  attr1[0].id = cudaLaunchAttributeClusterDimension;
  attr1[0].val.clusterDim.x = CL;
  attr1[0].val.clusterDim.y = 1;
  attr1[0].val.clusterDim.z = 1;
  cfg.attrs = attr1;
  cfg.numAttrs = 1;
  if (query_only) {  // can one cluster of CL CTAs be resident at all?
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    return (e == cudaSuccess && n >= 1) ? cudaSuccess : cudaErrorNotSupported;
  }
  return cudaLaunchKernelEx(&cfg, kern, views, vecs, add);
}

// Clusters of 16 CTAs (a non-portable size) where the GPU can place one:
// four warps a CTA, so each SM sub-partition's FP64 unit serves one warp of
// the critical path; else 8 CTAs of eight warps.
template <typename T>
void launch_block_solve_cluster(const RasView* views, int nviews, const RasVecs& vecs, int max_nt, int add,
                                cudaStream_t s, bool narrow) {
  if (nviews < 1) return;
  static std::once_flag pick;
  static bool wide = false;
  std::call_once(pick, [&] {
    wide = launch_block_solve_cl<T, 16>(views, nviews, vecs, max_nt, add, s, true) == cudaSuccess;
    cudaGetLastError();
  });
  if (wide && !narrow)
    launch_block_solve_cl<T, 16>(views, nviews, vecs, max_nt, add, s);
  else
    launch_block_solve_cl<T, kCl>(views, nviews, vecs, max_nt, add, s);
}

#define MSP_RAS_INST(T)                                                                          \
  template void launch_ras_solve<T>(const RasView*, int, const RasVecs&, const int32_t*, const int32_t*, \
                                    int, int, int, bool, cudaStream_t, int, int*, int);          \
  template int ras_slots<T>(int, bool);                                                          \
  template int ras_ctas_per_sm<T>(bool);
MSP_RAS_INST(double)
MSP_RAS_INST(float)
// BF16 factors: only the solve reads them (they are factored in FP32)
MSP_RAS_INST(__nv_bfloat16)
template void launch_block_solve_cluster<double>(const RasView*, int, const RasVecs&, int, int, cudaStream_t, bool);
template void launch_block_solve_cluster<float>(const RasView*, int, const RasVecs&, int, int, cudaStream_t, bool);

}  // namespace msp
