// C ABI of the msp library: device state, per-parameter assembly and
// factorisation, the V-cycle of Algorithm 2 and right-preconditioned FGMRES
// (Eq. 5).  Every arithmetic step runs in the kernels of k_sparse.cu and
// k_dense.cu; this file only allocates, uploads, orders launches on the
// instance stream and runs the small Hessenberg least-squares update of
// FGMRES on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "msp.h"
#include "msp_internal.h"
#include "msp_kernels.h"
#include "msp_profile.h"

namespace msp {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define MSP_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(MSP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

// ------------------------------------------------------- device memory
struct Allocator {
  msp_alloc_fn a = nullptr;
  msp_free_fn f = nullptr;
  void* ctx = nullptr;
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (a) return a(ctx, bytes, nullptr);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p) {
    if (!p) return;
    if (f) f(ctx, p, nullptr);
    else cudaFree(p);
  }
};

// Owns a list of device allocations made through one Allocator.
struct DevArena {
  Allocator al;
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool ok = true;
  template <typename T>
  T* alloc(size_t n) {
    size_t b = n * sizeof(T);
    void* p = al.get(b);
    if (!p) {
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (p && !v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      ok = false;
    return p;
  }
  void release() {
    for (void* p : ptrs) al.put(p);
    ptrs.clear();
    bytes = 0;
  }
};

struct DevLevel {
  int n = 0, m = 0;
  int64_t nnz = 0;
  int lpr_A = 8, lpr_P = 4, lpr_PT = 16;  // SpMV schedules (autotuned at load; 1 = row blocks)
  int32_t *rb_A = nullptr, *rb_P = nullptr, *rb_PT = nullptr;  // row blocks of the one-lane schedule
  int nrb_A = 0, nrb_P = 0, nrb_PT = 0;
  // ILU(p) subdomain factors (see HostLevel)
  bool ilu = false;
  int64_t ilu_nnz = 0, ilu_rows = 0, ilu_next = 0;
  int ilu_max_n = 0, ilu_max_row = 0;
  double ilu_flops = 0;  // algorithmic flops of one ILU factorisation of the level
  int64_t *ilu_lptr = nullptr, *ilu_ext_pos = nullptr;
  int32_t *ilu_lcol = nullptr, *ilu_ext_nz = nullptr;
  int32_t *ilu_fwd_rows = nullptr, *ilu_fwd_lvl = nullptr, *ilu_fwd_loff = nullptr;
  int32_t *ilu_bwd_rows = nullptr, *ilu_bwd_lvl = nullptr, *ilu_bwd_loff = nullptr;
  int64_t *ilu_fe_ptr = nullptr, *ilu_fe_slot = nullptr, *ilu_be_ptr = nullptr, *ilu_be_slot = nullptr;
  int32_t *ilu_fe_src = nullptr, *ilu_be_src = nullptr;
  int32_t *rowptr = nullptr, *col = nullptr, *diag = nullptr, *cptr = nullptr, *contrib = nullptr;
  uint8_t *nzflag = nullptr, *dir = nullptr;
  int32_t* dir_list = nullptr;
  int ndir = 0;
  double *xyz = nullptr, *S = nullptr, *vol = nullptr, *cen = nullptr;
  double* cwave = nullptr;  // [m][8] cos(pi a_j . c_e) of the cosine coefficient (set-up)
  int32_t* tets = nullptr;
  double* b = nullptr;  // load vector
  // subdomains
  int nsub = 0, max_nt = 0;
  int32_t *sub_ptr = nullptr, *sub_dofs = nullptr, *sub_nt = nullptr, *sub_order = nullptr;
  uint8_t* sub_own = nullptr;
  int64_t* fac_off = nullptr;
  int64_t fac_elems = 0;
  EnvDev env{};
  int64_t* ext_pos = nullptr;
  int32_t* ext_nz = nullptr;
  int64_t next = 0;
  std::vector<int> active;        // active[k] = #subdomains with NT > k
  std::vector<int> max_rows;      // max_p (R_k - k) at step k
  std::vector<double> trail_flops;  // flops of trailing step k (tile envelope)
  std::vector<double> panel_flops;  // flops of panel step k
  int64_t sum_np = 0, env_elems = 0, sum_owned = 0;
  int max_band = 0;               // max over tile rows of 1 + (R_I - I)
  bool ras_wide = false;          // the staged solve in its one-CTA-per-SM form
  int ras_grid = 0;               // CTAs of the RAS solve and their subdomain lists
  int ras_bins = 0;               // > 0: the lists come ras_grid / ras_bins to an SM (taken by SM on the device)
  int32_t *ras_cta_ptr = nullptr, *ras_cta_list = nullptr;
  bool fac_blocks = false;        // whole-block persistent factorisation on this level
  int fac_grid = 0;               // its CTAs and their block lists
  int32_t *fac_cta_ptr = nullptr, *fac_cta_list = nullptr;
  double fac_flops = 0;           // all tile steps of the level
  // prolongation from level+1 (P_*) and restriction to it (PT_*)
  int64_t P_nnz = 0, PT_nnz = 0;
  int32_t *P_rowptr = nullptr, *P_col = nullptr, *PT_rowptr = nullptr, *PT_col = nullptr;
  double *P_val = nullptr, *PT_val = nullptr;
  const int4* P_ell_col = nullptr;  // P in the four-entry form (barycentric P: at most four entries per row)
  const double2* P_ell_val = nullptr;
};

}  // namespace msp

using namespace msp;

struct msp_hierarchy {
  msp_options opt{};
  std::vector<HostLevel> host;
  std::vector<DevLevel> dev;
  DevArena arena;
  int32_t* wave = nullptr;
  int device = 0;
  bool host_only = false;
  std::mutex mu;
  size_t instance_bytes = 0;  // bytes held by live instances (budget)
};

struct msp_instance {
  msp_hierarchy* h = nullptr;
  cudaStream_t stream = nullptr;
  DevArena arena;
  size_t charged = 0;
  double* mu = nullptr;
  std::vector<double*> k, val, r, z, t;
  std::vector<void*> fac;   // per level: double, float or BF16 (level_store)
  std::vector<float*> work;  // per BF16 level: the FP32 factorisation, rounded into fac
  int* info = nullptr;
  int* ras_err = nullptr;  // bit 4: a bounded wait of the staged RAS solve expired
  RasView* rview = nullptr;  // device: this instance's view of every level for the triangular solves
  int* ras_claim = nullptr;  // device: the RAS launch's per-SM arrivals and taken lists (zeroed per launch)
  int expire_ras = 0;      // msp_debug_expire_waits: staged RAS launches left to starve of copies
  int m = 30;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *res = nullptr, *part = nullptr, *hdev = nullptr;
  double* xb = nullptr;  // device buffers used by msp_solve_host
  double* hpin = nullptr;  // pinned host staging
  cudaStream_t aux[2] = {nullptr, nullptr};  // coarser levels factor concurrently
  cudaStream_t cap = nullptr;  // private origin stream of the factorisation's graph capture
  // FP64 factors: the blocks of every persistent level as one longest-first
  // work list, one launch factors them all
  BlockItem* fz_items = nullptr;
  int32_t *fz_ptr = nullptr, *fz_list = nullptr;
  int fz_grid = 0;
  int* fz_ctr = nullptr;  // [4 fz_bins] items taken from, and CTAs on, each list (zeroed before every launch)
  int fz_bins = 0;
  int32_t *fz_ptr2 = nullptr, *fz_list2 = nullptr;  // the same items over 2 fz_bins lists (msp_debug_spread_work)
  bool spread_work = false;  // msp_debug_spread_work: twice as many work lists as SMs
  bool narrow_cluster = false;  // msp_debug_spread_work(2): the coarsest solve's 8-CTA form
  bool fz_f32 = false;
  double fz_flops = 0;
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  // per level, for the tile-step factorisation: the stream of the work off
  // the critical chain, and its events (diag done, critical panel done, bulk done)
  std::vector<cudaStream_t> bulk;
  std::vector<std::array<cudaEvent_t, 3>> bev;
  // the factorisation as a CUDA graph (see factor_all)
  int fac_calls = 0;
  cudaGraphExec_t fac_graph = nullptr;
  msp_kernel_profile fac_graph_counts[PK_COUNT] = {};
  bool assembled = false, factored = false;
  Profile prof;
};

namespace msp {
namespace {

// The level solved as one interior block (the coarsest, with MSP_COARSE_DIRECT);
// it always stays FP64.
bool direct_level(const msp_hierarchy* h, int l) { return h->host[l].direct; }

// Storage of a level's factors (the directly solved level is always FP64).
enum class Store { F64, F32, BF16 };
Store level_store(const msp_hierarchy* h, int l) {
  if (direct_level(h, l)) return Store::F64;
  if (h->host[l].ilu_fill >= 0)  // ILU levels: FP32 for either reduced precision (sparse sweeps, no tensor cores)
    return (h->opt.factor_precision == MSP_F64 || h->opt.factor_precision == MSP_F64_TC) ? Store::F64 : Store::F32;
  if (h->opt.factor_precision == MSP_F32) return Store::F32;
  if (h->opt.factor_precision == MSP_BF16) return Store::BF16;
  return Store::F64;
}
size_t store_bytes(Store t) { return t == Store::F64 ? 8 : (t == Store::F32 ? 4 : 2); }

void finish_level_stats(const HostLevel& H, DevLevel& D) {
  D.max_nt = 0;
  for (int p = 0; p < H.nsub; ++p) D.max_nt = std::max(D.max_nt, H.sub_nt[p]);
  D.active.assign(D.max_nt + 1, 0);
  D.max_rows.assign(D.max_nt + 1, 0);
  D.trail_flops.assign(D.max_nt + 1, 0.0);
  D.panel_flops.assign(D.max_nt + 1, 0.0);
  D.sum_np = D.sum_owned = 0;
  D.fac_flops = 0;
  D.env_elems = H.sub_fac_off.empty() ? 0 : H.sub_fac_off.back();
  const double tile_gemm = 2.0 * 64 * 64 * 64, tile_syrk = 2.0 * 64 * (64 * 65 / 2);
  for (int p = 0; p < H.nsub; ++p) {
    int nt = H.sub_nt[p];
    D.sum_np += H.sub_ptr[p + 1] - H.sub_ptr[p];
    const int32_t* R = &H.tile_last[H.sub_trow[p]];
    for (int k = 0; k < nt; ++k) D.max_band = std::max(D.max_band, 1 + R[k] - k);
    for (int k = 0; k < nt; ++k) {
      D.active[k]++;
      int rem = R[k] - k;
      D.max_rows[k] = std::max(D.max_rows[k], rem);
      D.trail_flops[k] += (double)rem * (rem - 1) / 2 * tile_gemm + rem * tile_syrk;
      D.panel_flops[k] += rem * (64.0 * 64 * 65);  // triangular X^T product + scaling
      D.fac_flops += (double)rem * (rem - 1) / 2 * tile_gemm + rem * tile_syrk +
                     rem * (64.0 * 64 * 65) + 2.0 * 64 * 64 * 64 / 3;
    }
  }
  for (uint8_t o : H.sub_own) D.sum_owned += o;
}

// Longest-processing-time-first assignment of items (cost) to G bins: items
// in descending cost, each to the least loaded bin; ptr/list in CSR form,
// each bin's items in descending cost.
void lpt_lists(const std::vector<int64_t>& cost, int G, std::vector<int32_t>& ptr,
               std::vector<int32_t>& list) {
  const int n = (int)cost.size();
  std::vector<int32_t> ids(n);
  for (int p = 0; p < n; ++p) ids[p] = p;
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int64_t> load(G, 0);
  std::vector<std::vector<int32_t>> bins(G);
  for (int p : ids) {
    int best = 0;
    for (int g = 1; g < G; ++g)
      if (load[g] < load[best]) best = g;
    load[best] += cost[p];
    bins[best].push_back(p);
  }
  ptr.assign(G + 1, 0);
  list.clear();
  for (int g = 0; g < G; ++g) {
    list.insert(list.end(), bins[g].begin(), bins[g].end());
    ptr[g + 1] = (int32_t)list.size();
  }
}

// Ring slots of the staged solve of level l in its form (wide or not).
int ras_slots_of(const msp_hierarchy* h, int l, bool wide) {
  const int nt = h->dev[l].max_nt;
  switch (level_store(h, l)) {
    case Store::F64: return ras_slots<double>(nt, wide);
    case Store::F32: return ras_slots<float>(nt, wide);
    default: return ras_slots<__nv_bfloat16>(nt, wide);
  }
}

int upload_level(msp_hierarchy* h, int l, cudaStream_t s) {
  HostLevel& H = h->host[l];
  DevLevel& D = h->dev[l];
  DevArena& A = h->arena;
  D.n = H.n;
  D.m = H.m;
  D.nnz = (int64_t)H.col.size();

  D.xyz = A.upload(H.xyz);
  D.tets = A.upload(H.tets);
  D.dir = A.upload(H.dir);
  D.dir_list = A.upload(H.dir_list);
  D.ndir = (int)H.dir_list.size();
  D.rowptr = A.upload(H.rowptr);
  D.col = A.upload(H.col);
  {
    const std::vector<int32_t> rb = spmv_row_blocks(H.rowptr);
    D.rb_A = A.upload(rb);
    D.nrb_A = (int)rb.size() / 2 - 1;
  }
  if (A.ok) D.lpr_A = tune_spmv(D.rowptr, D.col, H.n, H.n, H.rowptr, H.col, D.rb_A, D.nrb_A, s);
  D.diag = A.upload(H.diag);
  D.cptr = A.upload(H.cptr);
  D.contrib = A.upload(H.contrib);
  D.nzflag = A.upload(H.nzflag);
  D.S = A.alloc<double>((size_t)H.m * H.nslot);
  D.vol = A.alloc<double>(H.m);
  D.cen = A.alloc<double>((size_t)H.m * 3);
  if (h->opt.coef_kind == MSP_K_COSEXP) D.cwave = A.alloc<double>((size_t)H.m * 8);
  D.b = A.alloc<double>(H.n);
  D.nsub = H.nsub;
  D.sub_ptr = A.upload(H.sub_ptr);
  D.sub_dofs = A.upload(H.sub_dofs);
  D.sub_own = A.upload(H.sub_own);
  D.sub_nt = A.upload(H.sub_nt);
  D.sub_order = A.upload(H.sub_order);
  D.fac_off = A.upload(H.sub_fac_off);
  D.fac_elems = H.sub_fac_off.empty() ? 0 : H.sub_fac_off.back();
  D.env.fac_off = D.fac_off;
  D.env.trow = A.upload(H.sub_trow);
  D.env.first = A.upload(H.tile_first);
  D.env.last = A.upload(H.tile_last);
  D.env.toff = A.upload(H.tile_off);
  D.env.nt = D.sub_nt;
  D.ext_pos = A.upload(H.ext_pos);
  D.ext_nz = A.upload(H.ext_nz);
  D.next = (int64_t)H.ext_pos.size();
  finish_level_stats(H, D);
  if (H.ilu_fill >= 0) {  // ILU(p) subdomain factors: sparse storage, level-scheduled kernels
    D.ilu = true;
    D.ilu_nnz = H.ilu_nnz;
    D.ilu_rows = H.sub_ptr.empty() ? 0 : H.sub_ptr.back();
    D.ilu_max_n = H.ilu_max_n;
    D.ilu_max_row = H.ilu_max_row;
    D.fac_elems = 3 * D.ilu_nnz + 2 * D.ilu_rows;  // [L | D | 1/D | Lf | Lb]
    D.ilu_fe_ptr = A.upload(H.ilu_fe_ptr);
    D.ilu_fe_src = A.upload(H.ilu_fe_src);
    D.ilu_fe_slot = A.upload(H.ilu_fe_slot);
    D.ilu_be_ptr = A.upload(H.ilu_be_ptr);
    D.ilu_be_src = A.upload(H.ilu_be_src);
    D.ilu_be_slot = A.upload(H.ilu_be_slot);
    D.ilu_lptr = A.upload(H.ilu_lptr);
    D.ilu_lcol = A.upload(H.ilu_lcol);
    D.ilu_fwd_rows = A.upload(H.ilu_fwd_rows);
    D.ilu_fwd_lvl = A.upload(H.ilu_fwd_lvl);
    D.ilu_fwd_loff = A.upload(H.ilu_fwd_loff);
    D.ilu_bwd_rows = A.upload(H.ilu_bwd_rows);
    D.ilu_bwd_lvl = A.upload(H.ilu_bwd_lvl);
    D.ilu_bwd_loff = A.upload(H.ilu_bwd_loff);
    D.ilu_ext_pos = A.upload(H.ilu_ext_pos);
    D.ilu_ext_nz = A.upload(H.ilu_ext_nz);
    D.ilu_next = (int64_t)H.ilu_ext_pos.size();
    D.ilu_flops = 0;
    for (int p = 0; p < H.nsub; ++p)
      for (int64_t R = H.sub_ptr[p]; R < H.sub_ptr[p + 1]; ++R) {
        for (int64_t t = H.ilu_lptr[R]; t < H.ilu_lptr[R + 1]; ++t) {
          const int64_t K = H.sub_ptr[p] + H.ilu_lcol[t];
          D.ilu_flops += 2.0 * (double)(H.ilu_lptr[K + 1] - H.ilu_lptr[K]) + 1;
        }
        D.ilu_flops += 3.0 * (double)(H.ilu_lptr[R + 1] - H.ilu_lptr[R]) + 1;
      }
    if (!A.ok) return fail(MSP_ERR_OOM, "device allocation failed while loading level " + std::to_string(l));
    if (ilu_factor_smem(D.ilu_max_n, D.ilu_max_row, 8) > 200u * 1024u || ilu_solve_smem(D.ilu_max_n, 8) > 200u * 1024u)
      return fail(MSP_ERR_INVALID, "level " + std::to_string(l) + ": subdomain blocks too large for the ILU "
                                   "kernels (" + std::to_string(D.ilu_max_n) + " DoFs)");
  } else {
    int nsm = 0;
    MSP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    // RAS solve: persistent CTAs (1-3 per SM by precision, or the wide form
    // when the level's tile band needs more ring slots), cost = stored
    // envelope tiles (both sweeps read each once)
    std::vector<int64_t> cost(H.nsub);
    for (int p = 0; p < H.nsub; ++p) cost[p] = (H.sub_fac_off[p + 1] - H.sub_fac_off[p]) / kTileElems;
    std::vector<int32_t> cptr, clist;
    {
      const Store st = level_store(h, l);
      // FP64 and FP32: the smaller form (two / four CTAs per SM) whenever two
      // ring slots fit; BF16 (four CTAs per SM): when its slots cover the tile band
      const int need = st == Store::BF16 ? std::max(2, D.max_band) : 2;
      D.ras_wide = !direct_level(h, l) && ras_slots_of(h, l, false) < need;
      const int per_sm = st == Store::F64   ? ras_ctas_per_sm<double>(D.ras_wide)
                         : st == Store::F32 ? ras_ctas_per_sm<float>(D.ras_wide)
                                            : ras_ctas_per_sm<__nv_bfloat16>(D.ras_wide);
      const int G = nsm * per_sm;
      if (H.nsub >= G && per_sm > 1) {
        // the CTAs an SM holds share its FP64 / FP32 issue, so the SMs' sums
        // are balanced first, then each SM's share over its CTAs
        std::vector<int32_t> bptr, blist;
        lpt_lists(cost, nsm, bptr, blist);
        cptr.assign(1, 0);
        clist.clear();
        for (int b = 0; b < nsm; ++b) {
          std::vector<int64_t> sub;
          for (int k = bptr[b]; k < bptr[b + 1]; ++k) sub.push_back(cost[blist[k]]);
          std::vector<int32_t> sptr, slist;
          lpt_lists(sub, per_sm, sptr, slist);
          for (int r = 0; r < per_sm; ++r) {
            for (int k = sptr[r]; k < sptr[r + 1]; ++k) clist.push_back(blist[bptr[b] + slist[k]]);
            cptr.push_back((int32_t)clist.size());
          }
        }
        D.ras_bins = nsm;
      } else {
        lpt_lists(cost, std::max(1, std::min(H.nsub, G)), cptr, clist);
        D.ras_bins = 0;
      }
    }
    D.ras_grid = (int)cptr.size() - 1;
    D.ras_cta_ptr = A.upload(cptr);
    D.ras_cta_list = A.upload(clist);
    // factorisation: on levels with many blocks one persistent launch, as many
    // CTAs as fit on the GPU at once, cost = tile operations of all steps
    // (diagonal 1, panel 1, trailing pair 2, diagonal pair 1)
    D.fac_blocks = H.nsub >= std::max(2, nsm / 2);
    if (D.fac_blocks) {
      const Store fst = level_store(h, l);
      const int per_sm = fst == Store::BF16                    ? ldlt_blocks_tc_per_sm()
                         : fst == Store::F32                   ? ldlt_blocks_per_sm<float>()
                         : h->opt.factor_precision == MSP_F64_TC ? ldlt_blocks_oz_per_sm()
                                                               : ldlt_blocks_per_sm<double>();
      for (int p = 0; p < H.nsub; ++p) {
        const int32_t* R = &H.tile_last[H.sub_trow[p]];
        int64_t c = 0;
        for (int k = 0; k < H.sub_nt[p]; ++k) {
          const int64_t rem = R[k] - k;
          c += 1 + rem + rem * (rem - 1) + rem;
        }
        cost[p] = c;
      }
      // the tensor-core kernel fills every SM's shared memory: leave four SMs
      // to the coarsest block's tile steps, which then run beside it instead of
      // after it (4 was faster than 8 or 16 at 64^3)
      const int sms = h->opt.factor_precision == MSP_F64_TC ? std::max(1, nsm - 4) : nsm;
      lpt_lists(cost, std::max(1, std::min(H.nsub, sms * per_sm)), cptr, clist);
      D.fac_grid = (int)cptr.size() - 1;
      D.fac_cta_ptr = A.upload(cptr);
      D.fac_cta_list = A.upload(clist);
    }
    if (!A.ok) return fail(MSP_ERR_OOM, "device allocation failed while loading level " + std::to_string(l));
  }
  if (!D.ilu) {
    const int slots = ras_slots_of(h, l, D.ras_wide);
    // the sweeps hold one tile at a time, so two ring slots keep the producer
    // ahead; deeper rings (up to the tile band) prefetch more
    const bool direct = direct_level(h, l);
    if (direct && block_solve_cluster_smem(D.max_nt) > 220u * 1024u)
      return fail(MSP_ERR_INVALID, "coarsest level too large for the cluster block solve (" +
                                       std::to_string(D.max_nt) + " tiles)");
    if (!direct && slots < 2)
      return fail(MSP_ERR_INVALID, "level " + std::to_string(l) + ": subdomain blocks too large " +
                                       "for the staged triangular solve (" + std::to_string(D.max_nt) +
                                       " tiles)");
  }
  if (l + 1 < (int)h->host.size()) {
    D.P_nnz = (int64_t)H.P_col.size();
    D.PT_nnz = (int64_t)H.PT_col.size();
    D.P_rowptr = A.upload(H.P_rowptr);
    D.P_col = A.upload(H.P_col);
    D.P_val = A.upload(H.P_val);
    D.PT_rowptr = A.upload(H.PT_rowptr);
    D.PT_col = A.upload(H.PT_col);
    D.PT_val = A.upload(H.PT_val);
    {
      std::vector<int32_t> ec;
      std::vector<double> ev;
      if (spmv_ell4(H.P_rowptr, H.P_col, H.P_val, ec, ev)) {
        D.P_ell_col = reinterpret_cast<const int4*>(A.upload(ec));
        D.P_ell_val = reinterpret_cast<const double2*>(A.upload(ev));
      }
    }
    {
      const std::vector<int32_t> rbp = spmv_row_blocks(H.P_rowptr), rbt = spmv_row_blocks(H.PT_rowptr);
      D.rb_P = A.upload(rbp);
      D.nrb_P = (int)rbp.size() / 2 - 1;
      D.rb_PT = A.upload(rbt);
      D.nrb_PT = (int)rbt.size() / 2 - 1;
    }
    if (A.ok) {
      const int nc = h->host[l + 1].n;
      D.lpr_P = tune_spmv(D.P_rowptr, D.P_col, H.n, nc, H.P_rowptr, H.P_col, D.rb_P, D.nrb_P, s, D.P_ell_col,
                          D.P_ell_val);
      D.lpr_PT = tune_spmv(D.PT_rowptr, D.PT_col, nc, H.n, H.PT_rowptr, H.PT_col, D.rb_PT, D.nrb_PT, s);
    }
  }
  if (!A.ok) return fail(MSP_ERR_OOM, "device allocation failed while loading level " + std::to_string(l));
  int* bad = A.alloc<int>(1);
  if (!bad) return fail(MSP_ERR_OOM, "device allocation failed");
  MSP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  // Lame parameters of a unit Young's modulus (linear elasticity only)
  const double nu = h->opt.poisson_ratio;
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
  // element: P1, elasticity, P2, or the P2-P1 pair (whose coupling rides in `lam`)
  const int kind = H.fields == 3 ? 1 : (H.p2 ? (H.nloc == 14 ? 3 : 2) : 0);
  launch_tet_geometry(D.xyz, D.tets, D.m, kind, kind == 3 ? h->opt.coupling : lam, mu, D.S, D.vol, D.cen, bad, s);
  if (D.cwave) launch_coefficient_basis(D.cen, D.m, h->wave, D.cwave, s);
  launch_load_vector(D.xyz, D.dir, D.diag, D.cptr, D.contrib, D.vol, D.n, h->opt.load_kind, H.fields,
                     H.nslot, lam, mu, D.b, s);
  int hbad = 0;
  MSP_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA(cudaStreamSynchronize(s));
  MSP_CUDA(cudaGetLastError());
  if (hbad) return fail(MSP_ERR_INVALID, "degenerate tet on level " + std::to_string(l));
  return MSP_OK;
}

// The tcgen05 self-check (msp_tensor_selftest), once per device.
int tensor_check(int device) {
  static std::mutex mu;
  static int state[64] = {0};  // 0 unknown, 1 passed, -1 failed
  if (device < 0 || device >= 64) return fail(MSP_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (state[device] == 0) state[device] = msp_tensor_selftest(nullptr) == MSP_OK ? 1 : -1;
  if (state[device] < 0)
    return fail(MSP_ERR_INTERNAL, "the tensor-core self-check failed on this device; BF16 factors need it");
  return MSP_OK;
}

int check_options(const msp_options& o) {
  if (o.delta < 0 || o.delta > 64) return fail(MSP_ERR_INVALID, "delta out of range");
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre > 64 || o.nu_post > 64)
    return fail(MSP_ERR_INVALID, "nu out of range");
  if (o.restart < 1 || o.restart > 256) return fail(MSP_ERR_INVALID, "restart out of range");
  if (o.max_it < 1) return fail(MSP_ERR_INVALID, "max_it must be >= 1");
  if (o.factor_precision != MSP_F64 && o.factor_precision != MSP_F32 && o.factor_precision != MSP_BF16 &&
      o.factor_precision != MSP_F64_TC)
    return fail(MSP_ERR_INVALID, "unknown factor precision");
  if (o.transfer != MSP_TRANSFER_BARY && o.transfer != MSP_TRANSFER_MLS)
    return fail(MSP_ERR_INVALID, "unknown transfer");
  if (o.coarse_solver != MSP_COARSE_DIRECT && o.coarse_solver != MSP_COARSE_RAS)
    return fail(MSP_ERR_INVALID, "unknown coarse solver");
  if (o.ilu_fill_fine < -1 || o.ilu_fill_fine > 16 || o.ilu_fill_coarse < -1 || o.ilu_fill_coarse > 16)
    return fail(MSP_ERR_INVALID, "ILU fill level out of range (-1 .. 16)");
  if (o.coarse_solver == MSP_COARSE_RAS && o.nu_pre < 1)
    return fail(MSP_ERR_INVALID, "a smoothed coarsest level needs nu_pre >= 1");
  if (o.coef_kind != MSP_K_CONST && o.coef_kind != MSP_K_COSEXP)
    return fail(MSP_ERR_INVALID, "unknown coefficient family");
  if (o.load_kind != MSP_F_ONE && o.load_kind != MSP_F_SINES)
    return fail(MSP_ERR_INVALID, "unknown load");
  if (!std::isfinite(o.coef_scale)) return fail(MSP_ERR_INVALID, "non-finite coef_scale");
  if (o.pde != MSP_PDE_POISSON && o.pde != MSP_PDE_ELASTICITY && o.pde != MSP_PDE_POISSON_P2 &&
      o.pde != MSP_PDE_P2P1)
    return fail(MSP_ERR_INVALID, "unknown pde");
  const bool p2 = o.pde == MSP_PDE_POISSON_P2 || o.pde == MSP_PDE_P2P1;
  if (p2 && o.transfer != MSP_TRANSFER_BARY)
    return fail(MSP_ERR_INVALID, "P2 elements take the P2 interpolation between levels, not MLS");
  if (p2 && o.load_kind != MSP_F_ONE) return fail(MSP_ERR_INVALID, "P2 elements support the load f = 1 only");
  if (o.pde == MSP_PDE_P2P1 && !(o.coupling > 0.0 && std::isfinite(o.coupling)))
    return fail(MSP_ERR_INVALID, "the P2-P1 system needs a coupling coefficient > 0");
  if (o.pde == MSP_PDE_ELASTICITY && !(o.poisson_ratio > 0.0 && o.poisson_ratio < 0.5))
    return fail(MSP_ERR_INVALID, "linear elasticity needs a Poisson ratio in (0, 0.5)");
  if (o.pde == MSP_PDE_ELASTICITY && o.transfer != MSP_TRANSFER_BARY)
    return fail(MSP_ERR_INVALID, "linear elasticity takes the barycentric transfers (field-split P)");
  if ((o.alloc == nullptr) != (o.free == nullptr))
    return fail(MSP_ERR_INVALID, "alloc and free must be given together");
  return MSP_OK;
}

// ------------------------------------------------------------ launches
int assemble_all(msp_instance* I) {
  msp_hierarchy* h = I->h;
  cudaStream_t s = I->stream;
  for (size_t l = 0; l < h->dev.size(); ++l) {
    DevLevel& D = h->dev[l];
    ProfScope ps(I->prof, PK_ASSEMBLE, s, 2);
    launch_coefficient(D.cwave, D.m, h->opt.coef_kind, I->mu, h->opt.coef_scale, I->k[l], s);
    launch_assemble(D.cptr, D.contrib, D.nzflag, I->k[l], D.S, D.nnz,
                    h->host[l].nslot, I->val[l], s);
    ps.account((double)D.nnz * 8 + (double)D.nnz * 5 + (double)h->host[l].contrib.size() * 12 +
                   (double)D.m * (D.cwave ? 72 : 8),
               (double)h->host[l].contrib.size() * 2);
  }
  MSP_CUDA(cudaGetLastError());
  return MSP_OK;
}

template <typename T>
void factor_level(msp_instance* I, int l, T* fac, cudaStream_t s, bool tensor = false, bool defer = false) {
  msp_hierarchy* h = I->h;
  DevLevel& D = h->dev[l];
  {
    ProfScope ps(I->prof, PK_EXTRACT, s, 2);
    launch_extract<T>(D.ext_pos, D.ext_nz, D.next, I->val[l], D.fac_elems, fac, s);
    ps.account((double)D.fac_elems * sizeof(T) + (double)D.next * (12 + sizeof(T) + 8), 0);
  }
  if (D.fac_blocks && defer) {  // the blocks go into a batched launch (msp_factor_batch)
    cudaEventRecord(I->bev[l][0], s);
    return;
  }
  if (D.fac_blocks) {
    ProfScope ps(I->prof, PK_LDLT_BLOCKS, s);
    if constexpr (std::is_same<T, float>::value) {
      if (tensor) launch_ldlt_blocks_tc(fac, D.env, D.fac_cta_ptr, D.fac_cta_list, D.fac_grid, I->info, s);
      else launch_ldlt_blocks<T>(fac, D.env, D.fac_cta_ptr, D.fac_cta_list, D.fac_grid, I->info, s);
    } else if (h->opt.factor_precision == MSP_F64_TC) {
      launch_ldlt_blocks_oz(fac, D.env, D.fac_cta_ptr, D.fac_cta_list, D.fac_grid, I->info, s);
    } else {
      launch_ldlt_blocks<T>(fac, D.env, D.fac_cta_ptr, D.fac_cta_list, D.fac_grid, I->info, s);
    }
    ps.account(0, D.fac_flops);
    return;
  }
  // Tile steps with one step of lookahead.  On `s`, the chain the next
  // diagonal tile depends on: diagonal tile k, panel tile (k+1, k), trailing
  // pair (k+1, k+1).  On the level's bulk stream, the other panel tiles and
  // pairs of step k, which overlap with diagonal tile k+1.  Panel tile
  // (k+1, k) and the bulk panels of step k need the bulk pairs of step k-1.
  cudaStream_t sb = I->bulk[l];
  cudaEvent_t ev_diag = I->bev[l][0], ev_cp = I->bev[l][1], ev_bulk = I->bev[l][2];
  cudaEventRecord(ev_bulk, s);  // the extraction
  cudaStreamWaitEvent(sb, ev_bulk, 0);
  bool bulk_pending = false;
  for (int k = 0; k < D.max_nt; ++k) {
    int na = D.active[k];
    {
      ProfScope ps(I->prof, PK_LDLT_DIAG, s);
      launch_ldlt_diag<T>(fac, D.env, D.sub_order, na, k, I->info, s);
      ps.account((double)na * 2 * 4096 * sizeof(T), (double)na * (2.0 * 64 * 64 * 64 / 3));
    }
    const int rows = D.max_rows[k];
    if (rows <= 0) continue;
    const int pairs = rows * (rows + 1) / 2;
    cudaEventRecord(ev_diag, s);
    if (rows > 1) {
      cudaStreamWaitEvent(sb, ev_diag, 0);
      ProfScope ps(I->prof, PK_LDLT_PANEL, sb);
      launch_ldlt_panel<T>(fac, D.env, D.sub_order, na, k, 1, rows - 1, sb);
      ps.account(0, D.panel_flops[k] * (rows - 1) / rows);
    }
    if (bulk_pending) {
      cudaStreamWaitEvent(s, ev_bulk, 0);
      bulk_pending = false;
    }
    {
      ProfScope ps(I->prof, PK_LDLT_PANEL, s);
      launch_ldlt_panel<T>(fac, D.env, D.sub_order, na, k, 0, 1, s);
      ps.account(0, D.panel_flops[k] / rows);
    }
    cudaEventRecord(ev_cp, s);
    {
      ProfScope ps(I->prof, PK_LDLT_TRAIL, s);
      launch_ldlt_trail<T>(fac, D.env, D.sub_order, na, k, 0, 1, s);
      ps.account(0, D.trail_flops[k] / pairs);
    }
    if (pairs > 1) {
      cudaStreamWaitEvent(sb, ev_cp, 0);
      {
        ProfScope ps(I->prof, PK_LDLT_TRAIL, sb);
        launch_ldlt_trail<T>(fac, D.env, D.sub_order, na, k, 1, pairs - 1, sb);
        ps.account(0, D.trail_flops[k] * (pairs - 1) / pairs);
      }
      cudaEventRecord(ev_bulk, sb);
      bulk_pending = true;
    }
  }
  cudaEventRecord(ev_bulk, sb);  // join the bulk stream back (always: graph capture needs it)
  cudaStreamWaitEvent(s, ev_bulk, 0);
  {
    ProfScope ps(I->prof, PK_LDLT_DIAG, s);
    launch_ldlt_xfill<T>(fac, D.env, D.sub_order, D.active[0], D.max_nt, s);
    if (direct_level(h, l)) launch_ldlt_mnfill<T>(fac, D.env, D.max_nt, s);  // for the cluster solve
    ps.account(0, 0);
  }
}

// ILU(p) factors of level l in T: A's lower triangle into [L | D], the
// incomplete factorisation by dependency levels, the level-major copies.
template <typename T>
void factor_ilu(msp_instance* I, int l, T* fac, cudaStream_t s) {
  const DevLevel& D = I->h->dev[l];
  {
    ProfScope ps(I->prof, PK_EXTRACT, s, 2);
    launch_ilu_extract<T>(D.ilu_ext_pos, D.ilu_ext_nz, D.ilu_next, I->val[l], D.fac_elems, fac, s);
    ps.account((double)D.fac_elems * sizeof(T) + (double)D.ilu_next * 20, 0);
  }
  ProfScope ps(I->prof, PK_LDLT_BLOCKS, s, 2);
  launch_ilu_factor<T>(fac, D.ilu_nnz, D.ilu_rows, D.nsub, D.sub_ptr, D.ilu_lptr, D.ilu_lcol, D.ilu_fwd_rows,
                       D.ilu_fwd_lvl, D.ilu_fwd_loff, D.ilu_max_n, D.ilu_max_row, I->info, s);
  launch_ilu_gather<T>(fac, D.ilu_nnz, D.ilu_rows, D.ilu_fe_slot, D.ilu_be_slot, s);
  ps.account((double)D.ilu_nnz * sizeof(T) * 5, D.ilu_flops);
}

// Enqueues the whole factorisation on `s0` (the instance stream, or the
// private stream a graph capture starts from), with forks onto the auxiliary
// and bulk streams, all joined back.
int enqueue_factor(msp_instance* I, cudaStream_t s0, bool defer = false) {
  msp_hierarchy* h = I->h;
  MSP_CUDA(cudaMemsetAsync(I->info, 0, sizeof(int), s0));
  // The levels are independent: level 0 on the instance stream, the coarser
  // ones on two auxiliary streams forked from it and joined back.  The
  // coarsest block (a long chain of small dependent launches) goes first, on
  // the high-priority stream.
  const int L = (int)h->dev.size();
  MSP_CUDA(cudaEventRecord(I->fork, s0));
  for (int a = 0; a < 2; ++a) MSP_CUDA(cudaStreamWaitEvent(I->aux[a], I->fork, 0));
  for (int l = L - 1; l >= 0; --l) {
    const Store st = level_store(h, l);
    const DevLevel& D = h->dev[l];
    // FP32 / BF16 persistent levels one after another on the instance stream:
    // their one-CTA-per-block grids then never hold every slot of the GPU,
    // and the coarsest block's tile steps always find room beside them
    const bool serial = l > 0 && l < L - 1 && st != Store::F64 && D.fac_blocks && !D.ilu;
    cudaStream_t s = (l == 0 || serial) ? s0 : (l == L - 1 ? I->aux[0] : I->aux[1]);
    if (D.ilu) {
      if (st == Store::F64)
        factor_ilu<double>(I, l, static_cast<double*>(I->fac[l]), s);
      else
        factor_ilu<float>(I, l, static_cast<float*>(I->fac[l]), s);
    } else if (st == Store::F64) {
      factor_level<double>(I, l, static_cast<double*>(I->fac[l]), s, false, defer || I->fz_grid > 0);
    } else if (st == Store::F32) {
      factor_level<float>(I, l, static_cast<float*>(I->fac[l]), s, false, defer || I->fz_grid > 0);
    } else {
      factor_level<float>(I, l, I->work[l], s, /*tensor=*/true);
      ProfScope ps(I->prof, PK_EXTRACT, s);
      launch_round_bf16(I->work[l], static_cast<__nv_bfloat16*>(I->fac[l]), h->dev[l].fac_elems, s);
      ps.account((double)h->dev[l].fac_elems * 6, 0);
    }
  }
  // the persistent levels' blocks in one launch, once every level is extracted
  if (I->fz_grid > 0 && !defer) {
    for (int l = 1; l < L; ++l)
      if (h->dev[l].fac_blocks && !h->dev[l].ilu) MSP_CUDA(cudaStreamWaitEvent(s0, I->bev[l][0], 0));
    ProfScope ps(I->prof, PK_LDLT_BLOCKS, s0);
    const int nb = I->spread_work ? 2 * I->fz_bins : I->fz_bins;
    const int32_t* ptr = I->spread_work ? I->fz_ptr2 : I->fz_ptr;
    const int32_t* list = I->spread_work ? I->fz_list2 : I->fz_list;
    MSP_CUDA(cudaMemsetAsync(I->fz_ctr, 0, sizeof(int) * 2 * nb, s0));
    if (I->fz_f32)
      launch_ldlt_blocks_batch<float>(I->fz_items, ptr, list, I->fz_grid, s0, I->fz_ctr, nb);
    else
      launch_ldlt_blocks_batch<double>(I->fz_items, ptr, list, I->fz_grid, s0, I->fz_ctr, nb);
    ps.account(0, I->fz_flops);
  }
  for (int a = 0; a < 2; ++a) {
    MSP_CUDA(cudaEventRecord(I->join[a], I->aux[a]));
    MSP_CUDA(cudaStreamWaitEvent(s0, I->join[a], 0));
  }
  MSP_CUDA(cudaGetLastError());
  return MSP_OK;
}

// The factorisation runs the same launches for every mu, so from its second
// call on it is replayed from a CUDA graph captured once (one launch for
// hundreds of kernels, and no host gaps in the coarsest block's chain).  The
// graph is used only while no kernel class is being timed; the per-class
// launch, byte and flop counts of one factorisation are added per replay.
// The capture starts from the instance's private stream `cap`, which no other
// instance or host thread can enqueue on, so launches of other threads on the
// instance stream (a stream several instances share) are never captured and
// never invalidate the capture; the graph then runs on the instance stream.
int factor_all(msp_instance* I) {
  const bool graph_ok = I->prof.mask == 0;
  if (graph_ok && !I->fac_graph && I->fac_calls >= 1) {
    msp_kernel_profile before[PK_COUNT];
    std::memcpy(before, I->prof.c, sizeof(before));
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(I->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rc = enqueue_factor(I, I->cap);
      const cudaError_t ec = cudaStreamEndCapture(I->cap, &g);
      if (rc == MSP_OK && ec == cudaSuccess && g &&
          cudaGraphInstantiate(&I->fac_graph, g, 0) == cudaSuccess) {
        for (int k = 0; k < PK_COUNT; ++k) {
          I->fac_graph_counts[k].launches = I->prof.c[k].launches - before[k].launches;
          I->fac_graph_counts[k].bytes = I->prof.c[k].bytes - before[k].bytes;
          I->fac_graph_counts[k].flops = I->prof.c[k].flops - before[k].flops;
        }
      } else {
        I->fac_graph = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    std::memcpy(I->prof.c, before, sizeof(before));  // counted again per replay below
    cudaGetLastError();
    msp::g_last_error.clear();
  }
  if (graph_ok && I->fac_graph) {
    MSP_CUDA(cudaGraphLaunch(I->fac_graph, I->stream));
    for (int k = 0; k < PK_COUNT; ++k) {
      I->prof.c[k].launches += I->fac_graph_counts[k].launches;
      I->prof.c[k].bytes += I->fac_graph_counts[k].bytes;
      I->prof.c[k].flops += I->fac_graph_counts[k].flops;
    }
  } else {
    const int rc = enqueue_factor(I, I->stream);
    if (rc) return rc;
  }
  I->fac_calls++;
  int hinfo = 0;
  MSP_CUDA(cudaMemcpyAsync(&hinfo, I->info, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  I->prof.harvest();
  if (hinfo & 2) return fail(MSP_ERR_TIMEOUT, "a bounded tensor-core wait in the factorisation expired");
  if (hinfo) return fail(MSP_ERR_INTERNAL, "non-positive or non-finite pivot in a subdomain factor");
  I->factored = true;
  return MSP_OK;
}

void ras(msp_instance* I, int l, const double* t, double* z, int add, cudaStream_t s) {
  msp_hierarchy* h = I->h;
  DevLevel& D = h->dev[l];
  const bool coarse = direct_level(h, l);
  int kind = coarse ? PK_COARSE : (l == 0 ? PK_RAS : PK_RAS_COARSER);
  ProfScope ps(I->prof, kind, s);
  const Store st = level_store(h, l);
  size_t es = store_bytes(st);
  if (D.ilu) {
    if (st == Store::F64)
      launch_ilu_solve<double>(static_cast<const double*>(I->fac[l]), D.ilu_nnz, D.ilu_rows, D.nsub, D.sub_ptr,
                               D.sub_dofs, D.sub_own, D.ilu_fe_ptr, D.ilu_fe_src, D.ilu_be_ptr, D.ilu_be_src,
                               D.ilu_fwd_rows, D.ilu_fwd_lvl, D.ilu_fwd_loff, D.ilu_bwd_rows, D.ilu_bwd_lvl,
                               D.ilu_bwd_loff, D.ilu_max_n, D.dir_list, D.ndir, t, z, add, s);
    else
      launch_ilu_solve<float>(static_cast<const float*>(I->fac[l]), D.ilu_nnz, D.ilu_rows, D.nsub, D.sub_ptr,
                              D.sub_dofs, D.sub_own, D.ilu_fe_ptr, D.ilu_fe_src, D.ilu_be_ptr, D.ilu_be_src,
                              D.ilu_fwd_rows, D.ilu_fwd_lvl, D.ilu_fwd_loff, D.ilu_bwd_rows, D.ilu_bwd_lvl,
                              D.ilu_bwd_loff, D.ilu_max_n, D.dir_list, D.ndir, t, z, add, s);
    ps.account(2.0 * (double)D.ilu_nnz * (es + 4) + (double)D.sum_np * (13 + es) +
                   (double)D.sum_owned * (add ? 16 : 8),
               4.0 * (double)D.ilu_nnz + (double)D.sum_np);
    return;
  }
  RasVecs vv{};
  vv.t[0] = t;
  vv.z[0] = z;
  if (coarse) {  // one block: both sweeps split over a cluster of CTAs
    launch_block_solve_cluster<double>(I->rview + l, 1, vv, D.max_nt, add, s, I->narrow_cluster);
  } else {
    const int inj = I->expire_ras > 0 ? 1 : 0;
    if (inj) --I->expire_ras;
    int* claim = D.ras_bins > 0 ? I->ras_claim : nullptr;
    // msp_debug_spread_work: twice as many bins as SMs, so half of each SM's
    // CTAs find their rank beyond its share and claim a list no SM owns
    const int nb = (I->spread_work && D.ras_grid % (2 * std::max(1, D.ras_bins)) == 0) ? 2 * D.ras_bins : D.ras_bins;
    if (claim) cudaMemsetAsync(claim, 0, sizeof(int) * ((size_t)nb + D.ras_grid), s);
    if (st == Store::BF16)
      launch_ras_solve<__nv_bfloat16>(I->rview + l, 1, vv, D.ras_cta_ptr, D.ras_cta_list, D.ras_grid, D.max_nt,
                                      add, D.ras_wide, s, inj, claim, nb);
    else if (st == Store::F32)
      launch_ras_solve<float>(I->rview + l, 1, vv, D.ras_cta_ptr, D.ras_cta_list, D.ras_grid, D.max_nt, add,
                              D.ras_wide, s, inj, claim, nb);
    else
      launch_ras_solve<double>(I->rview + l, 1, vv, D.ras_cta_ptr, D.ras_cta_list, D.ras_grid, D.max_nt, add,
                               D.ras_wide, s, inj, claim, nb);
  }
  // algorithmic: the stored envelope of L read by each of the two sweeps
  // (the element count of an L and U pair), gather + scatter of the vectors
  ps.account(2.0 * (double)D.env_elems * es + (double)D.sum_np * 13 +
                 (double)D.sum_owned * (add ? 16 : 8),
             4.0 * (double)D.env_elems);
}

void spmv(msp_instance* I, int l, const double* x, double* y, const double* r, int mode,
          cudaStream_t s) {
  DevLevel& D = I->h->dev[l];
  ProfScope ps(I->prof, PK_SPMV, s);
  launch_spmv(D.rowptr, D.col, I->val[l], D.n, x, y, r, mode, SpmvPlan{D.lpr_A, D.rb_A, D.nrb_A}, s);
  ps.account((double)D.nnz * 12 + (double)(D.n + 1) * 4 + (double)D.n * (mode == SPMV_SET ? 16 : 24),
             2.0 * (double)D.nnz);
}

void transfer(msp_instance* I, int l, bool restrict_, const double* x, double* y, int mode,
              cudaStream_t s) {
  DevLevel& D = I->h->dev[l];
  int nc = I->h->dev[l + 1].n;
  ProfScope ps(I->prof, PK_TRANSFER, s);
  if (restrict_)
    launch_spmv(D.PT_rowptr, D.PT_col, D.PT_val, nc, x, y, nullptr, mode, SpmvPlan{D.lpr_PT, D.rb_PT, D.nrb_PT},
                s);
  else
    launch_spmv(D.P_rowptr, D.P_col, D.P_val, D.n, x, y, nullptr, mode,
                SpmvPlan{D.lpr_P, D.rb_P, D.nrb_P, D.P_ell_col, D.P_ell_val}, s);
  double rows = restrict_ ? nc : D.n, cols = restrict_ ? D.n : nc;
  double nnz = (double)(restrict_ ? D.PT_nnz : D.P_nnz);
  ps.account(nnz * 12 + (rows + 1) * 4 + cols * 8 + rows * (mode == SPMV_SET ? 8 : 16), 2.0 * nnz);
}

// z += B^{-1}(r - A z), `its` times; when `from_zero`, z is not read first
// (the first step is z = B^{-1} r).
void smooth(msp_instance* I, int l, const double* r, double* z, int its, bool from_zero,
            cudaStream_t s) {
  int n = I->h->dev[l].n;
  for (int it = 0; it < its; ++it) {
    if (from_zero && it == 0) {
      ras(I, l, r, z, 0, s);
    } else {
      spmv(I, l, z, I->t[l], r, SPMV_RESIDUAL, s);
      ras(I, l, I->t[l], z, 1, s);
    }
  }
  if (from_zero && its == 0) {
    ProfScope ps(I->prof, PK_VEC, s);
    launch_fill(z, 0.0, n, s);
    ps.account((double)n * 8, 0);
  }
}

// Algorithm 2 with the level transfers (P^T / P, or MLS both ways); the
// coarsest level is solved directly or, with MSP_COARSE_RAS, smoothed nu_pre
// times from z = 0 like the others.
void vcycle(msp_instance* I, const double* r0, double* z0, cudaStream_t s) {
  msp_hierarchy* h = I->h;
  const int L = (int)h->dev.size();
  std::vector<const double*> r(L);
  std::vector<double*> z(L);
  r[0] = r0;
  z[0] = z0;
  for (int l = 1; l < L; ++l) {
    r[l] = I->r[l];
    z[l] = I->z[l];
  }
  for (int l = 0; l + 1 < L; ++l) {
    smooth(I, l, r[l], z[l], h->opt.nu_pre, true, s);
    spmv(I, l, z[l], I->t[l], r[l], SPMV_RESIDUAL, s);
    transfer(I, l, true, I->t[l], I->r[l + 1], SPMV_SET, s);
  }
  if (direct_level(h, L - 1)) ras(I, L - 1, r[L - 1], z[L - 1], 0, s);
  else smooth(I, L - 1, r[L - 1], z[L - 1], h->opt.nu_pre, true, s);
  for (int l = L - 2; l >= 0; --l) {
    transfer(I, l, false, z[l + 1], z[l], SPMV_ADD, s);
    smooth(I, l, r[l], z[l], h->opt.nu_post, false, s);
  }
}

// ---------------------------------------------------------------- FGMRES
struct Dot {
  msp_instance* I;
  // out[0..nv) = V_i . w on the device, then copied to the pinned staging
  void run(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* out_dev) {
    ProfScope ps(I->prof, PK_VEC, I->stream, 2);
    launch_multidot(V, ld, nv, w, n, I->part, out_dev, I->stream);
    ps.account((double)(nv + 1) * n * 8, 2.0 * nv * n);
  }
};

int fgmres_run(msp_instance* I, const double* b, double* x, double rtol, msp_stats* st) {
  msp_hierarchy* h = I->h;
  cudaStream_t s = I->stream;
  const int64_t n = h->dev[0].n;
  const int m = I->m;
  const int maxit = h->opt.max_it;
  double* V = I->V;
  double* Z = I->Z;
  double* w = I->w;
  double* rr = I->res;
  double* hd = I->hdev;   // device: [0..m] h1, [m+1..2m+1] h2, [2m+2] norm^2
  double* hp = I->hpin;   // pinned host copy
  Dot dot{I};
  auto vec = [&](int i) { return V + (int64_t)i * n; };
  auto zvec = [&](int i) { return Z + (int64_t)i * n; };
  // ||b||
  dot.run(b, 0, 1, b, n, hd);
  MSP_CUDA(cudaMemcpyAsync(hp, hd, sizeof(double), cudaMemcpyDeviceToHost, s));
  MSP_CUDA(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(hp[0]);
  {
    ProfScope ps(I->prof, PK_VEC, s);
    launch_fill(x, 0.0, n, s);
    ps.account((double)n * 8, 0);
  }
  st->iterations = 0;
  st->rel_residual = 0.0;
  if (!(bnorm > 0.0)) {
    MSP_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(bnorm)) return fail(MSP_ERR_INVALID, "non-finite right-hand side");
    return MSP_OK;
  }
  {
    ProfScope ps(I->prof, PK_VEC, s);
    launch_copy(b, rr, n, s);
    ps.account((double)n * 16, 0);
  }
  double rnorm = bnorm;
  int it = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  int status = MSP_ERR_NOT_CONVERGED;
  while (true) {
    if (rnorm <= rtol * bnorm) {
      status = MSP_OK;
      break;
    }
    if (it >= maxit) break;
    {
      ProfScope ps(I->prof, PK_VEC, s);
      launch_scale(rr, 1.0 / rnorm, vec(0), n, s);
      ps.account((double)n * 16, (double)n);
    }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = rnorm;
    int j = 0;
    bool breakdown = false;
    for (; j < m && it < maxit; ++j) {
      vcycle(I, vec(j), zvec(j), s);
      spmv(I, 0, zvec(j), w, nullptr, SPMV_SET, s);
      // classical Gram-Schmidt, twice (CGS2)
      dot.run(V, n, j + 1, w, n, hd);
      {
        ProfScope ps(I->prof, PK_VEC, s);
        launch_multi_axpy(V, n, j + 1, hd, w, n, -1.0, s);
        ps.account((double)(j + 3) * n * 8, 2.0 * (j + 1) * n);
      }
      dot.run(V, n, j + 1, w, n, hd + (m + 1));
      {
        ProfScope ps(I->prof, PK_VEC, s);
        launch_multi_axpy(V, n, j + 1, hd + (m + 1), w, n, -1.0, s);
        ps.account((double)(j + 3) * n * 8, 2.0 * (j + 1) * n);
      }
      dot.run(w, 0, 1, w, n, hd + 2 * (m + 1));
      MSP_CUDA(cudaMemcpyAsync(hp, hd, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
      MSP_CUDA(cudaStreamSynchronize(s));
      I->prof.harvest();
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hp[i] + hp[m + 1 + i];
      double hn = std::sqrt(std::max(hp[2 * (m + 1)], 0.0));
      if (!std::isfinite(hn)) {
        st->iterations = it;
        return fail(MSP_ERR_NOT_CONVERGED, "non-finite Arnoldi vector");
      }
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      double den = std::hypot(a, c);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : c / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      if (hn <= 1e-300) {
        breakdown = true;
        ++j;
        break;
      }
      {
        ProfScope ps(I->prof, PK_VEC, s);
        launch_scale(w, 1.0 / hn, vec(j + 1), n, s);
        ps.account((double)n * 16, (double)n);
      }
      if (std::fabs(g[j + 1]) <= rtol * bnorm) {
        ++j;
        break;
      }
    }
    for (int i = j - 1; i >= 0; --i) {
      double sum = g[i];
      for (int k = i + 1; k < j; ++k) sum -= H[(size_t)i * m + k] * y[k];
      y[i] = sum / H[(size_t)i * m + i];
    }
    // x += Z y (y staged through pinned memory, then used on the device)
    for (int i = 0; i < j; ++i) hp[2 * (m + 1) + 1 + i] = y[i];
    MSP_CUDA(cudaMemcpyAsync(hd + 2 * (m + 1) + 1, hp + 2 * (m + 1) + 1, sizeof(double) * j,
                             cudaMemcpyHostToDevice, s));
    {
      ProfScope ps(I->prof, PK_VEC, s);
      launch_multi_axpy(Z, n, j, hd + 2 * (m + 1) + 1, x, n, 1.0, s);
      ps.account((double)(j + 2) * n * 8, 2.0 * j * n);
    }
    spmv(I, 0, x, rr, b, SPMV_RESIDUAL, s);
    dot.run(rr, 0, 1, rr, n, hd);
    MSP_CUDA(cudaMemcpyAsync(hp, hd, sizeof(double), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    rnorm = std::sqrt(std::max(hp[0], 0.0));
    if (!std::isfinite(rnorm)) break;
    if (breakdown && rnorm > rtol * bnorm) break;
  }
  MSP_CUDA(cudaGetLastError());
  st->iterations = it;
  st->rel_residual = rnorm / bnorm;
  if (status != MSP_OK)
    return fail(MSP_ERR_NOT_CONVERGED, "FGMRES did not reach rtol within max_it (or broke down)");
  return MSP_OK;
}

// FGMRES, then the error word of the staged RAS solves: an expired bounded
// wait makes every result of the solve meaningless, so it is reported
// (MSP_ERR_TIMEOUT) whatever the iteration itself returned, and cleared.
int fgmres(msp_instance* I, const double* b, double* x, double rtol, msp_stats* st) {
  const int rc = fgmres_run(I, b, x, rtol, st);
  const std::string msg = msp::g_last_error;
  int e = 0;
  MSP_CUDA(cudaMemcpyAsync(&e, I->ras_err, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  if (e) {
    MSP_CUDA(cudaMemsetAsync(I->ras_err, 0, sizeof(int), I->stream));
    MSP_CUDA(cudaStreamSynchronize(I->stream));
    return fail(MSP_ERR_TIMEOUT, "a bounded wait in the staged RAS solve expired");
  }
  msp::g_last_error = msg;
  return rc;
}

int alloc_instance(msp_hierarchy* h, msp_instance* I) {
  DevArena& A = I->arena;
  A.al = h->arena.al;
  const int L = (int)h->dev.size();
  I->mu = A.alloc<double>(8);
  I->info = A.alloc<int>(1);
  I->ras_err = A.alloc<int>(1);
  I->k.resize(L);
  I->val.resize(L);
  I->r.resize(L);
  I->z.resize(L);
  I->t.resize(L);
  I->fac.resize(L);
  I->work.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    DevLevel& D = h->dev[l];
    I->k[l] = A.alloc<double>(D.m);
    I->val[l] = A.alloc<double>(D.nnz);
    I->r[l] = A.alloc<double>(D.n);
    I->z[l] = A.alloc<double>(D.n);
    I->t[l] = A.alloc<double>(D.n);
    const Store st = level_store(h, l);
    if (st == Store::F64) {
      // the level solved as one block keeps its cluster solve's coupling tiles after the envelope
      I->fac[l] = A.alloc<double>(D.fac_elems + (direct_level(h, l) ? kBlockSolveExtra(D.max_nt) : 0));
    } else if (st == Store::F32) {
      I->fac[l] = A.alloc<float>(D.fac_elems);
    } else {
      I->fac[l] = A.alloc<__nv_bfloat16>(D.fac_elems);
      I->work[l] = A.alloc<float>(D.fac_elems);
    }
  }
  I->m = h->opt.restart;
  const int64_t n = h->dev[0].n;
  I->V = A.alloc<double>((size_t)(I->m + 1) * n);
  I->Z = A.alloc<double>((size_t)I->m * n);
  I->w = A.alloc<double>(n);
  I->res = A.alloc<double>(n);
  I->xb = A.alloc<double>(2 * n);
  I->part = A.alloc<double>((size_t)(I->m + 1) * kDotBlocks);
  I->hdev = A.alloc<double>(4 * (size_t)(I->m + 1) + 8);
  {
    std::vector<RasView> rv(L);
    for (int l = 0; l < L; ++l) {
      const DevLevel& D = h->dev[l];
      rv[l] = RasView{I->fac[l], D.env, D.sub_ptr, D.sub_dofs, D.sub_own, D.dir_list, D.ndir, I->ras_err};
    }
    I->rview = A.upload(rv);
    size_t claim = 0;
    for (int l = 0; l < L; ++l)
      if (h->dev[l].ras_bins > 0) claim = std::max(claim, (size_t)2 * h->dev[l].ras_bins + h->dev[l].ras_grid);
    if (claim) I->ras_claim = A.alloc<int>(claim);
  }
  if (!A.ok) return fail(MSP_ERR_OOM, "device allocation failed for an instance");
  // FP64 factors: one work list over the blocks of every persistent level
  // (cost = tile operations, as for one level), balanced longest-first over
  // the GPU, so that the small blocks of the coarser levels fill the SMs that
  // finish the fine level early.  (FP32 factors keep one launch per level: a
  // grid over every SM there slows the FP64 coarsest chain, which bounds that
  // factorisation.)
  if (h->opt.factor_precision == MSP_F64) {
    std::vector<BlockItem> items;
    std::vector<int64_t> cost;
    for (int l = 0; l < L; ++l) {
      const DevLevel& D = h->dev[l];
      const HostLevel& H = h->host[l];
      if (!D.fac_blocks || D.ilu) continue;
      I->fz_flops += D.fac_flops;
      for (int p = 0; p < H.nsub; ++p) {
        const int32_t* R = &H.tile_last[H.sub_trow[p]];
        int64_t c = 0;  // the block's FP64 flops over 64 (the FP64 pipe is the bound)
        for (int k = 0; k < H.sub_nt[p]; ++k) {
          const int64_t rem = R[k] - k;
          c += rem * (rem - 1) / 2 * 2 * 64 * 64 + rem * 64 * 65 + rem * 64 * 65 + 2 * 64 * 64 / 3;
        }
        items.push_back(BlockItem{I->fac[l], D.env, p, I->info});
        cost.push_back(c);
      }
    }
    if (!items.empty()) {
      int nsm = 0;
      MSP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
      I->fz_f32 = h->opt.factor_precision == MSP_F32;
      const int per_sm = I->fz_f32 ? ldlt_blocks_batch_per_sm<float>() : ldlt_blocks_batch_per_sm<double>();
      // One longest-first list per SM: the CTAs an SM holds share its FP64
      // pipe, so it is the SMs' sums that must come out even (balancing the
      // CTAs' lists left the busiest SM 11 % above the median, as the CTAs
      // land on SMs in an order of the hardware's).  The per_sm CTAs of an SM
      // take its items in turn; a list whose SM the launch did not reach is
      // taken by the CTAs that have finished their own.
      std::vector<int32_t> cptr, clist, sptr, slist;
      const int bins = std::max(1, std::min((int)items.size(), nsm));
      lpt_lists(cost, bins, cptr, clist);
      lpt_lists(cost, 2 * bins, sptr, slist);  // half of them no SM's own (msp_debug_spread_work)
      I->fz_items = A.upload(items);
      I->fz_ptr = A.upload(cptr);
      I->fz_list = A.upload(clist);
      I->fz_ptr2 = A.upload(sptr);
      I->fz_list2 = A.upload(slist);
      I->fz_bins = bins;
      I->fz_ctr = A.alloc<int>(4 * (size_t)bins);
      I->fz_grid = bins * per_sm;
      if (!A.ok) return fail(MSP_ERR_OOM, "device allocation failed for an instance");
    }
  }
  if (cudaMallocHost(&I->hpin, sizeof(double) * (4 * (size_t)(I->m + 1) + 8)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MSP_ERR_OOM, "pinned host allocation failed");
  }
  int prio_lo = 0, prio_hi = 0;
  MSP_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  for (int a = 0; a < 2; ++a) {
    MSP_CUDA(cudaStreamCreateWithPriority(&I->aux[a], cudaStreamNonBlocking, a == 0 ? prio_hi : prio_lo));
    MSP_CUDA(cudaEventCreateWithFlags(&I->join[a], cudaEventDisableTiming));
  }
  MSP_CUDA(cudaEventCreateWithFlags(&I->fork, cudaEventDisableTiming));
  MSP_CUDA(cudaStreamCreateWithFlags(&I->cap, cudaStreamNonBlocking));
  I->bulk.assign(L, nullptr);
  I->bev.assign(L, {nullptr, nullptr, nullptr});
  for (int l = 0; l < L; ++l) {
    if (h->dev[l].fac_blocks) {  // persistent levels: one event, "extracted", for msp_factor_batch
      MSP_CUDA(cudaEventCreateWithFlags(&I->bev[l][0], cudaEventDisableTiming));
      continue;
    }
    MSP_CUDA(cudaStreamCreateWithFlags(&I->bulk[l], cudaStreamNonBlocking));
    for (auto& e : I->bev[l]) MSP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  MSP_CUDA(cudaMemset(I->ras_err, 0, sizeof(int)));
  return MSP_OK;
}

int set_mu(msp_instance* I, const double* mu, int n_mu) {
  msp_hierarchy* h = I->h;
  double m8[8] = {0};
  if (h->opt.coef_kind == MSP_K_COSEXP) {
    if (n_mu != 8 || !mu) return fail(MSP_ERR_INVALID, "MSP_K_COSEXP needs n_mu == 8");
    for (int j = 0; j < 8; ++j) {
      if (!std::isfinite(mu[j])) return fail(MSP_ERR_INVALID, "non-finite mu");
      m8[j] = mu[j];
    }
  }
  std::copy(m8, m8 + 8, I->hpin);
  MSP_CUDA(cudaMemcpyAsync(I->mu, I->hpin, sizeof(m8), cudaMemcpyHostToDevice, I->stream));
  int rc = assemble_all(I);
  if (rc) return rc;
  MSP_CUDA(cudaStreamSynchronize(I->stream));  // the staging buffer is reused next
  I->assembled = true;
  I->factored = false;
  return MSP_OK;
}

size_t instance_need(const msp_hierarchy* h) {
  size_t need = 0;
  for (size_t l = 0; l < h->dev.size(); ++l) {
    const DevLevel& D = h->dev[l];
    need += (size_t)D.m * 8 + (size_t)D.nnz * 8 + (size_t)D.n * 24 +
            (size_t)D.fac_elems * (level_store(h, (int)l) == Store::BF16 ? 6 : store_bytes(level_store(h, (int)l)));
    if (direct_level(h, (int)l)) need += (size_t)kBlockSolveExtra(D.max_nt) * 8;
  }
  need += (size_t)(2 * h->opt.restart + 5) * h->dev[0].n * 8;
  return need;
}

// ============================================================ batched solves
// A batch fuses the V-cycles and Krylov steps of several instances (of one
// hierarchy or of several) into shared launches: at every level depth one
// staged RAS launch per (factor type, solve form) over the blocks of all
// members, one SpMV launch per (operator, schedule) over the members' stacked
// rows, one coarsest-solve launch with one cluster per member, and one launch
// per Krylov kernel.  Every member's arithmetic is that of its own msp_solve
// (the same kernels' per-row, per-block and per-slice code, the same order),
// so the results are bitwise the same; only the launches are shared.
struct BatchRas {
  Store st = Store::F64;
  bool wide = false;
  std::vector<int> members;  // view v of the launch = member members[v]
  RasView* views = nullptr;
  int32_t *cta_ptr = nullptr, *cta_list = nullptr;
  int grid = 0, max_nt = 0;
};
struct BatchCoarse {
  std::vector<int> members;
  RasView* views = nullptr;
  int max_nt = 0;
};

// The persistent-level blocks of the members whose factors the batched
// launch can take (FP64 or FP32 dense LU), per factor type.
struct BatchFac {
  bool f32 = false;
  BlockItem* items = nullptr;
  int32_t *cta_ptr = nullptr, *cta_list = nullptr;
  int grid = 0;
};

struct BatchState {
  std::vector<msp_instance*> m;
  cudaStream_t stream = nullptr;
  DevArena arena;
  int maxL = 0;
  std::vector<std::vector<BatchRas>> ras;  // [depth]: the smoothed levels at that depth
  std::vector<BatchCoarse> coarse;        // [depth]: the members whose coarsest level is at that depth
  cudaEvent_t ev = nullptr;
  // batched factorisation
  std::vector<char> deferred;             // member's persistent levels go to the batched launch
  std::vector<BatchFac> fac;
  std::vector<cudaEvent_t> join;           // per member: its own factorisation work done
  int* hinfo = nullptr;                    // pinned: every member's pivot word
  int fac_calls = 0;
  cudaGraphExec_t fac_graph = nullptr;
};

int batch_build(BatchState& B, msp_instance* const* insts, int n, cudaStream_t s) {
  if (n < 1 || n > kMaxMembers) return fail(MSP_ERR_INVALID, "a batch holds 1.." + std::to_string(kMaxMembers) +
                                                                  " instances");
  const msp_options& o0 = insts[0]->h->opt;
  for (int i = 0; i < n; ++i) {
    msp_instance* I = insts[i];
    if (!I) return fail(MSP_ERR_INVALID, "NULL instance in the batch");
    for (int k = 0; k < i; ++k)
      if (insts[k] == I) return fail(MSP_ERR_INVALID, "an instance is listed twice");
    const msp_options& o = I->h->opt;
    if (I->h->device != insts[0]->h->device) return fail(MSP_ERR_INVALID, "batch members on different devices");
    if (o.nu_pre != o0.nu_pre || o.nu_post != o0.nu_post)
      return fail(MSP_ERR_INVALID, "batch members need the same smoothing steps");
    if (o.coarse_solver != MSP_COARSE_DIRECT)
      return fail(MSP_ERR_INVALID, "batched solves need the directly solved coarsest level");
    for (const DevLevel& D : I->h->dev)
      if (D.ilu) return fail(MSP_ERR_INVALID, "batched solves take the exact subdomain LU, not ILU(p)");
  }
  B.m.assign(insts, insts + n);
  B.stream = s;
  B.arena.al = insts[0]->h->arena.al;
  B.maxL = 0;
  for (msp_instance* I : B.m) B.maxL = std::max(B.maxL, (int)I->h->dev.size());
  B.ras.assign(B.maxL, {});
  B.coarse.assign(B.maxL, {});
  int nsm = 0;
  MSP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, insts[0]->h->device));
  for (int d = 0; d < B.maxL; ++d) {
    std::vector<RasView> cv;
    for (int i = 0; i < n; ++i) {
      msp_instance* I = B.m[i];
      msp_hierarchy* h = I->h;
      const int L = (int)h->dev.size();
      if (d >= L) continue;
      const DevLevel& D = h->dev[d];
      const RasView v{I->fac[d], D.env, D.sub_ptr, D.sub_dofs, D.sub_own, D.dir_list, D.ndir, I->ras_err};
      if (d == L - 1) {  // the directly solved coarsest level
        B.coarse[d].members.push_back(i);
        B.coarse[d].max_nt = std::max(B.coarse[d].max_nt, D.max_nt);
        cv.push_back(v);
        continue;
      }
      const Store st = level_store(h, d);
      BatchRas* g = nullptr;
      for (BatchRas& x : B.ras[d])
        if (x.st == st && x.wide == D.ras_wide) g = &x;
      if (!g) {
        B.ras[d].push_back(BatchRas{});
        g = &B.ras[d].back();
        g->st = st;
        g->wide = D.ras_wide;
      }
      g->members.push_back(i);
      g->max_nt = std::max(g->max_nt, D.max_nt);
    }
    if (!cv.empty()) B.coarse[d].views = B.arena.upload(cv);
    for (BatchRas& g : B.ras[d]) {
      std::vector<RasView> views;
      std::vector<int64_t> cost;
      std::vector<int32_t> code;
      for (int v = 0; v < (int)g.members.size(); ++v) {
        msp_instance* I = B.m[g.members[v]];
        const DevLevel& D = I->h->dev[d];
        const HostLevel& H = I->h->host[d];
        views.push_back(RasView{I->fac[d], D.env, D.sub_ptr, D.sub_dofs, D.sub_own, D.dir_list, D.ndir,
                                I->ras_err});
        for (int p = 0; p < H.nsub; ++p) {
          cost.push_back((H.sub_fac_off[p + 1] - H.sub_fac_off[p]) / kTileElems);
          code.push_back((int32_t)(((uint32_t)v << kViewShift) | (uint32_t)p));
        }
      }
      // the ring depth of the shared launch is set by its largest block: every
      // member's level was checked at set-up to fit its own form, and a form
      // with fewer slots than two is refused here
      const int slots = g.st == Store::F64   ? ras_slots<double>(g.max_nt, g.wide)
                        : g.st == Store::F32 ? ras_slots<float>(g.max_nt, g.wide)
                                             : ras_slots<__nv_bfloat16>(g.max_nt, g.wide);
      if (slots < 2) return fail(MSP_ERR_INVALID, "batch: subdomain blocks too large for a shared solve");
      const int per_sm = g.st == Store::F64   ? ras_ctas_per_sm<double>(g.wide)
                         : g.st == Store::F32 ? ras_ctas_per_sm<float>(g.wide)
                                              : ras_ctas_per_sm<__nv_bfloat16>(g.wide);
      std::vector<int32_t> ptr, list;
      lpt_lists(cost, std::max(1, std::min((int)cost.size(), nsm * per_sm)), ptr, list);
      for (int32_t& q : list) q = code[q];
      g.grid = (int)ptr.size() - 1;
      g.views = B.arena.upload(views);
      g.cta_ptr = B.arena.upload(ptr);
      g.cta_list = B.arena.upload(list);
    }
  }
  // the batched factorisation: the persistent levels of FP64 / FP32 members
  // in one launch per factor type, longest blocks first, on all SMs but four,
  // which the members' coarsest-block tile steps (long chains of small
  // launches on their own streams) keep for themselves
  B.deferred.assign(n, 0);
  {
    std::vector<BlockItem> items[2];
    std::vector<int64_t> cost[2];
    for (int i = 0; i < n; ++i) {
      msp_instance* I = B.m[i];
      const msp_hierarchy* h = I->h;
      if (h->opt.factor_precision != MSP_F64 && h->opt.factor_precision != MSP_F32) continue;
      B.deferred[i] = 1;
      for (int l = 0; l < (int)h->dev.size(); ++l) {
        const DevLevel& D = h->dev[l];
        if (!D.fac_blocks) continue;
        const HostLevel& H = h->host[l];
        const int g = level_store(h, l) == Store::F64 ? 0 : 1;
        for (int p = 0; p < H.nsub; ++p) {
          const int32_t* R = &H.tile_last[H.sub_trow[p]];
          int64_t c = 0;
          for (int k = 0; k < H.sub_nt[p]; ++k) {
            const int64_t rem = R[k] - k;
            c += 1 + rem + rem * (rem - 1) + rem;
          }
          items[g].push_back(BlockItem{I->fac[l], D.env, p, I->info});
          cost[g].push_back(c);
        }
      }
    }
    const int reserve = std::min(4, nsm / 8);
    for (int g = 0; g < 2; ++g) {
      if (items[g].empty()) continue;
      const int per_sm = g == 0 ? ldlt_blocks_batch_per_sm<double>() : ldlt_blocks_batch_per_sm<float>();
      std::vector<int32_t> ptr, list;
      lpt_lists(cost[g], std::max(1, std::min((int)items[g].size(), (nsm - reserve) * per_sm)), ptr, list);
      BatchFac f;
      f.f32 = g == 1;
      f.items = B.arena.upload(items[g]);
      f.cta_ptr = B.arena.upload(ptr);
      f.cta_list = B.arena.upload(list);
      f.grid = (int)ptr.size() - 1;
      B.fac.push_back(f);
    }
  }
  if (!B.arena.ok) return fail(MSP_ERR_OOM, "device allocation failed for a batch");
  MSP_CUDA(cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming));
  B.join.assign(n, nullptr);
  for (int i = 0; i < n; ++i) MSP_CUDA(cudaEventCreateWithFlags(&B.join[i], cudaEventDisableTiming));
  if (cudaMallocHost(&B.hinfo, sizeof(int) * n) != cudaSuccess) {
    cudaGetLastError();
    B.hinfo = nullptr;
    return fail(MSP_ERR_OOM, "pinned host allocation failed");
  }
  return MSP_OK;
}

void batch_release(BatchState& B) {
  if (B.fac_graph) cudaGraphExecDestroy(B.fac_graph);
  B.fac_graph = nullptr;
  if (B.ev) cudaEventDestroy(B.ev);
  B.ev = nullptr;
  for (cudaEvent_t e : B.join)
    if (e) cudaEventDestroy(e);
  B.join.clear();
  if (B.hinfo) cudaFreeHost(B.hinfo);
  B.hinfo = nullptr;
  B.arena.release();
}

// Enqueues the factorisation of every member from B.stream: each member's
// own levels on its private streams (forked from B.stream), the persistent
// levels of the deferred members in the batched launches, all joined back.
int batch_enqueue_factor(BatchState& B) {
  const int n = (int)B.m.size();
  MSP_CUDA(cudaEventRecord(B.ev, B.stream));
  for (int i = 0; i < n; ++i) {
    msp_instance* I = B.m[i];
    MSP_CUDA(cudaStreamWaitEvent(I->cap, B.ev, 0));
    if (int rc = enqueue_factor(I, I->cap, B.deferred[i] != 0)) return rc;
  }
  for (int i = 0; i < n; ++i) {
    if (!B.deferred[i]) continue;
    const msp_hierarchy* h = B.m[i]->h;
    for (int l = 0; l < (int)h->dev.size(); ++l)
      if (h->dev[l].fac_blocks) MSP_CUDA(cudaStreamWaitEvent(B.stream, B.m[i]->bev[l][0], 0));
  }
  for (const BatchFac& f : B.fac) {
    if (f.f32) launch_ldlt_blocks_batch<float>(f.items, f.cta_ptr, f.cta_list, f.grid, B.stream);
    else launch_ldlt_blocks_batch<double>(f.items, f.cta_ptr, f.cta_list, f.grid, B.stream);
  }
  for (int i = 0; i < n; ++i) {
    MSP_CUDA(cudaEventRecord(B.join[i], B.m[i]->cap));
    MSP_CUDA(cudaStreamWaitEvent(B.stream, B.join[i], 0));
  }
  MSP_CUDA(cudaGetLastError());
  return MSP_OK;
}

// The batched factorisation; from its second call on it is replayed from a
// CUDA graph captured once (the launches are the same for every parameter).
int batch_factor(BatchState& B) {
  const int n = (int)B.m.size();
  for (msp_instance* I : B.m)
    if (!I->assembled) return fail(MSP_ERR_INVALID, "a batch member is not assembled");
  // B.stream after every member's own stream (its assembly)
  for (msp_instance* I : B.m) {
    if (I->stream == B.stream) continue;
    MSP_CUDA(cudaEventRecord(B.ev, I->stream));
    MSP_CUDA(cudaStreamWaitEvent(B.stream, B.ev, 0));
  }
  if (!B.fac_graph && B.fac_calls >= 1) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rc = batch_enqueue_factor(B);
      const cudaError_t ec = cudaStreamEndCapture(B.stream, &g);
      if (rc != MSP_OK || ec != cudaSuccess || !g || cudaGraphInstantiate(&B.fac_graph, g, 0) != cudaSuccess)
        B.fac_graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    msp::g_last_error.clear();
  }
  if (B.fac_graph) {
    MSP_CUDA(cudaGraphLaunch(B.fac_graph, B.stream));
  } else {
    if (int rc = batch_enqueue_factor(B)) return rc;
  }
  B.fac_calls++;
  for (int i = 0; i < n; ++i)
    MSP_CUDA(cudaMemcpyAsync(B.hinfo + i, B.m[i]->info, sizeof(int), cudaMemcpyDeviceToHost, B.stream));
  MSP_CUDA(cudaStreamSynchronize(B.stream));
  int rc = MSP_OK;
  for (int i = 0; i < n; ++i) {
    msp_instance* I = B.m[i];
    I->prof.harvest();
    if (B.hinfo[i] & 2) {
      I->factored = false;
      if (rc == MSP_OK) rc = fail(MSP_ERR_TIMEOUT, "a bounded tensor-core wait in the factorisation of member " +
                                                       std::to_string(i) + " expired");
    } else if (B.hinfo[i]) {
      I->factored = false;
      if (rc == MSP_OK) rc = fail(MSP_ERR_INTERNAL, "non-positive or non-finite pivot in a subdomain factor of "
                                                        "member " + std::to_string(i));
    } else {
      I->factored = true;
    }
  }
  return rc;
}

// Re-assembly of every member for its parameter (mu: n_mu per member), each on
// its own stream, one synchronisation for all.
int batch_assemble(BatchState& B, const double* mu, int n_mu) {
  const int n = (int)B.m.size();
  for (int i = 0; i < n; ++i) {
    msp_instance* I = B.m[i];
    msp_hierarchy* h = I->h;
    const double* mi = mu ? mu + (size_t)i * n_mu : nullptr;
    double m8[8] = {0};
    if (h->opt.coef_kind == MSP_K_COSEXP) {
      if (n_mu != 8 || !mi) return fail(MSP_ERR_INVALID, "MSP_K_COSEXP needs n_mu == 8");
      for (int j = 0; j < 8; ++j) {
        if (!std::isfinite(mi[j])) return fail(MSP_ERR_INVALID, "non-finite mu for member " + std::to_string(i));
        m8[j] = mi[j];
      }
    }
    std::copy(m8, m8 + 8, I->hpin);
    MSP_CUDA(cudaMemcpyAsync(I->mu, I->hpin, sizeof(m8), cudaMemcpyHostToDevice, I->stream));
    if (int rc = assemble_all(I)) return rc;
    I->assembled = true;
    I->factored = false;
    if (I->stream != B.stream) {
      MSP_CUDA(cudaEventRecord(B.ev, I->stream));
      MSP_CUDA(cudaStreamWaitEvent(B.stream, B.ev, 0));
    }
  }
  MSP_CUDA(cudaStreamSynchronize(B.stream));  // the staging buffers are reused next
  return MSP_OK;
}

// Per-member vectors of one V-cycle: level-d right-hand side and correction.
struct BatchLevelVecs {
  std::vector<std::vector<const double*>> r;  // [member][depth]
  std::vector<std::vector<double*>> z;
};

// One SpMV family at depth d over the members in `on` (J, P or the
// restriction), one launch per schedule among them.
enum BatchOp { BOP_J = 0, BOP_P = 1, BOP_R = 2 };
void batch_spmv(BatchState& B, int d, int op, const std::vector<int>& on,
                const std::vector<const double*>& x, const std::vector<double*>& y,
                const std::vector<const double*>& r, int mode) {
  std::vector<std::pair<int, int>> todo;  // (lpr, member)
  for (int i : on) {
    const DevLevel& D = B.m[i]->h->dev[d];
    todo.push_back({op == BOP_J ? D.lpr_A : (op == BOP_P ? D.lpr_P : D.lpr_PT), i});
  }
  std::sort(todo.begin(), todo.end());
  size_t k = 0;
  while (k < todo.size()) {
    SpmvBatch S;
    S.lpr = todo[k].first;
    S.mode = mode;
    size_t e = k;
    while (e < todo.size() && todo[e].first == S.lpr) ++e;
    for (size_t q = k; q < e; ++q) {
      const int i = todo[q].second, b = S.nb++;
      msp_instance* I = B.m[i];
      const DevLevel& D = I->h->dev[d];
      int64_t rows = 0;
      if (op == BOP_J) {
        S.rowptr[b] = D.rowptr; S.col[b] = D.col; S.val[b] = I->val[d];
        S.row_blk[b] = D.rb_A; S.nblk[b] = D.nrb_A;
        rows = D.n;
      } else if (op == BOP_P) {
        S.rowptr[b] = D.P_rowptr; S.col[b] = D.P_col; S.val[b] = D.P_val;
        S.row_blk[b] = D.rb_P; S.nblk[b] = D.nrb_P;
        S.ell_col[b] = D.P_ell_col; S.ell_val[b] = D.P_ell_val;
        rows = D.n;
      } else {
        S.rowptr[b] = D.PT_rowptr; S.col[b] = D.PT_col; S.val[b] = D.PT_val;
        S.row_blk[b] = D.rb_PT; S.nblk[b] = D.nrb_PT;
        rows = I->h->dev[d + 1].n;
      }
      S.x[b] = x[i];
      S.y[b] = y[i];
      S.r[b] = r.empty() ? nullptr : r[i];
      S.start[b + 1] = S.start[b] + (S.lpr == 1 ? S.nblk[b] : rows);
    }
    launch_spmv_batch(S, B.stream);
    k = e;
  }
}

// The staged RAS solves of depth d for the members in `on`: t -> z (add).
void batch_ras(BatchState& B, int d, const std::vector<char>& on, const std::vector<const double*>& t,
               const std::vector<double*>& z, int add) {
  for (BatchRas& g : B.ras[d]) {
    RasVecs vv{};
    bool any = false;
    for (size_t v = 0; v < g.members.size(); ++v) {
      const int i = g.members[v];
      if (!on[i]) continue;
      vv.t[v] = t[i];
      vv.z[v] = z[i];
      any = true;
    }
    if (!any) continue;
    const int nv = (int)g.members.size();
    if (g.st == Store::BF16)
      launch_ras_solve<__nv_bfloat16>(g.views, nv, vv, g.cta_ptr, g.cta_list, g.grid, g.max_nt, add, g.wide,
                                      B.stream);
    else if (g.st == Store::F32)
      launch_ras_solve<float>(g.views, nv, vv, g.cta_ptr, g.cta_list, g.grid, g.max_nt, add, g.wide, B.stream);
    else
      launch_ras_solve<double>(g.views, nv, vv, g.cta_ptr, g.cta_list, g.grid, g.max_nt, add, g.wide, B.stream);
  }
}

// One V-cycle (Algorithm 2, as vcycle()) for every member in `act`, from
// r0[i] into z0[i], all launches shared by depth.
void batch_vcycle(BatchState& B, const std::vector<char>& act, const std::vector<const double*>& r0,
                  const std::vector<double*>& z0) {
  const int n = (int)B.m.size();
  const int nu_pre = B.m[0]->h->opt.nu_pre, nu_post = B.m[0]->h->opt.nu_post;
  auto rv = [&](int i, int d) -> const double* { return d == 0 ? r0[i] : B.m[i]->r[d]; };
  auto zv = [&](int i, int d) -> double* { return d == 0 ? z0[i] : B.m[i]->z[d]; };
  std::vector<const double*> r(n), t_in(n);
  std::vector<double*> z(n), t(n);
  for (int d = 0; d < B.maxL; ++d) {
    std::vector<char> on(n, 0);
    std::vector<int> onl, crs;
    for (int i = 0; i < n; ++i) {
      const int L = (int)B.m[i]->h->dev.size();
      if (!act[i] || d >= L) continue;
      r[i] = rv(i, d);
      z[i] = zv(i, d);
      t[i] = B.m[i]->t[d];
      t_in[i] = t[i];
      if (d < L - 1) {
        on[i] = 1;
        onl.push_back(i);
      } else {
        crs.push_back(i);
      }
    }
    if (!onl.empty()) {
      for (int it = 0; it < nu_pre; ++it) {
        if (it == 0) {
          batch_ras(B, d, on, r, z, 0);
        } else {
          batch_spmv(B, d, BOP_J, onl, std::vector<const double*>(z.begin(), z.end()), t, r, SPMV_RESIDUAL);
          batch_ras(B, d, on, t_in, z, 1);
        }
      }
      if (nu_pre == 0) {
        VecBatch V;
        int64_t nmax = 0;
        for (int i : onl) {
          V.y[V.nb] = z[i];
          V.a[V.nb] = 0.0;
          V.n[V.nb++] = B.m[i]->h->dev[d].n;
          nmax = std::max<int64_t>(nmax, B.m[i]->h->dev[d].n);
        }
        launch_vec_batch(V, VEC_FILL, nmax, B.stream);
      }
      batch_spmv(B, d, BOP_J, onl, std::vector<const double*>(z.begin(), z.end()), t, r, SPMV_RESIDUAL);
      std::vector<double*> rn(n, nullptr);
      for (int i : onl) rn[i] = B.m[i]->r[d + 1];
      batch_spmv(B, d, BOP_R, onl, t_in, rn, {}, SPMV_SET);
    }
    if (!crs.empty()) {
      RasVecs vv{};
      for (size_t v = 0; v < B.coarse[d].members.size(); ++v) {
        const int i = B.coarse[d].members[v];
        if (!act[i]) continue;
        vv.t[v] = r[i];
        vv.z[v] = z[i];
      }
      launch_block_solve_cluster<double>(B.coarse[d].views, (int)B.coarse[d].members.size(), vv,
                                         B.coarse[d].max_nt, 0, B.stream);
    }
  }
  for (int d = B.maxL - 2; d >= 0; --d) {
    std::vector<char> on(n, 0);
    std::vector<int> onl;
    for (int i = 0; i < n; ++i) {
      const int L = (int)B.m[i]->h->dev.size();
      if (!act[i] || d >= L - 1) continue;
      r[i] = rv(i, d);
      z[i] = zv(i, d);
      t[i] = B.m[i]->t[d];
      t_in[i] = t[i];
      on[i] = 1;
      onl.push_back(i);
    }
    if (onl.empty()) continue;
    std::vector<const double*> zc(n, nullptr);
    for (int i : onl) zc[i] = zv(i, d + 1);
    batch_spmv(B, d, BOP_P, onl, zc, z, {}, SPMV_ADD);
    for (int it = 0; it < nu_post; ++it) {
      batch_spmv(B, d, BOP_J, onl, std::vector<const double*>(z.begin(), z.end()), t, r, SPMV_RESIDUAL);
      batch_ras(B, d, on, t_in, z, 1);
    }
  }
}

// FGMRES of fgmres_run() for every member, in lockstep.
struct FgMember {
  msp_instance* I = nullptr;
  int64_t n = 0;
  int m = 0;
  const double* b = nullptr;
  double* x = nullptr;
  double bnorm = 0, rnorm = 0;
  int it = 0, j = 0;
  bool breakdown = false;
  enum { CHECK, START, INNER, RESTART, DONE } phase = CHECK;
  int status = MSP_ERR_NOT_CONVERGED;
  std::string msg;
  std::vector<double> H, cs, sn, g, y;
};

int fgmres_batch(BatchState& B, const double* const* b, double* const* x, double rtol, msp_stats* st) {
  const int n = (int)B.m.size();
  cudaStream_t s = B.stream;
  std::vector<FgMember> F(n);
  int64_t nmax = 0;
  for (int i = 0; i < n; ++i) {
    msp_instance* I = B.m[i];
    FgMember& f = F[i];
    f.I = I;
    f.n = I->h->dev[0].n;
    f.m = I->m;
    f.b = (b && b[i]) ? b[i] : I->h->dev[0].b;
    f.x = x[i];
    f.H.assign((size_t)(f.m + 1) * f.m, 0.0);
    f.cs.assign(f.m, 0.0);
    f.sn.assign(f.m, 0.0);
    f.g.assign(f.m + 1, 0.0);
    f.y.assign(f.m, 0.0);
    nmax = std::max(nmax, f.n);
  }
  auto vec = [&](FgMember& f, int k) { return f.I->V + (int64_t)k * f.n; };
  auto zvec = [&](FgMember& f, int k) { return f.I->Z + (int64_t)k * f.n; };
  auto sync_copy = [&](const std::vector<int>& who, int count) -> int {
    for (int i : who)
      MSP_CUDA(cudaMemcpyAsync(F[i].I->hpin, F[i].I->hdev, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    return MSP_OK;
  };
  auto dots = [&](const std::vector<int>& who, auto V_of, auto ld_of, auto nv_of, auto w_of, int off) {
    DotBatch D;
    int nvmax = 0;
    for (int i : who) {
      FgMember& f = F[i];
      const int b2 = D.nb++;
      D.V[b2] = V_of(f);
      D.ld[b2] = ld_of(f);
      D.nv[b2] = nv_of(f);
      D.w[b2] = w_of(f);
      D.n[b2] = f.n;
      D.part[b2] = f.I->part;
      D.out[b2] = f.I->hdev + off;
      nvmax = std::max(nvmax, D.nv[b2]);
    }
    launch_multidot_batch(D, nvmax, s);
  };
  std::vector<int> all(n);
  for (int i = 0; i < n; ++i) all[i] = i;
  // ||b||
  dots(all, [](FgMember& f) { return f.b; }, [](FgMember&) { return (int64_t)0; }, [](FgMember&) { return 1; },
       [](FgMember& f) { return f.b; }, 0);
  if (int rc = sync_copy(all, 1)) return rc;
  {
    VecBatch V;
    for (int i : all) {
      V.y[V.nb] = F[i].x;
      V.a[V.nb] = 0.0;
      V.n[V.nb++] = F[i].n;
    }
    launch_vec_batch(V, VEC_FILL, nmax, s);
  }
  VecBatch cp;
  for (int i : all) {
    FgMember& f = F[i];
    f.bnorm = std::sqrt(f.I->hpin[0]);
    if (!(f.bnorm > 0.0)) {
      f.phase = FgMember::DONE;
      f.status = std::isfinite(f.bnorm) ? MSP_OK : MSP_ERR_INVALID;
      f.msg = std::isfinite(f.bnorm) ? "" : "non-finite right-hand side";
      continue;
    }
    cp.x[cp.nb] = f.b;
    cp.y[cp.nb] = f.I->res;
    cp.n[cp.nb++] = f.n;
    f.rnorm = f.bnorm;
  }
  launch_vec_batch(cp, VEC_COPY, nmax, s);
  for (;;) {
    // checks, and the start of a cycle
    VecBatch sc;
    for (FgMember& f : F) {
      if (f.phase != FgMember::CHECK) continue;
      if (f.rnorm <= rtol * f.bnorm) {
        f.status = MSP_OK;
        f.phase = FgMember::DONE;
      } else if (f.it >= f.I->h->opt.max_it) {
        f.phase = FgMember::DONE;
      } else {
        sc.x[sc.nb] = f.I->res;
        sc.y[sc.nb] = vec(f, 0);
        sc.a[sc.nb] = 1.0 / f.rnorm;
        sc.n[sc.nb++] = f.n;
        std::fill(f.g.begin(), f.g.end(), 0.0);
        f.g[0] = f.rnorm;
        f.j = 0;
        f.breakdown = false;
        f.phase = FgMember::INNER;
      }
    }
    launch_vec_batch(sc, VEC_SCALE, nmax, s);
    std::vector<int> inner;
    for (int i = 0; i < n; ++i)
      if (F[i].phase == FgMember::INNER) inner.push_back(i);
    if (!inner.empty()) {
      std::vector<char> act(n, 0);
      std::vector<const double*> r0(n, nullptr);
      std::vector<double*> z0(n, nullptr);
      for (int i : inner) {
        act[i] = 1;
        r0[i] = vec(F[i], F[i].j);
        z0[i] = zvec(F[i], F[i].j);
      }
      batch_vcycle(B, act, r0, z0);
      {
        std::vector<const double*> zx(n, nullptr);
        std::vector<double*> wy(n, nullptr);
        for (int i : inner) {
          zx[i] = z0[i];
          wy[i] = F[i].I->w;
        }
        batch_spmv(B, 0, BOP_J, inner, zx, wy, {}, SPMV_SET);
      }
      auto axpy = [&](int off) {
        AxpyBatch A;
        for (int i : inner) {
          FgMember& f = F[i];
          const int b2 = A.nb++;
          A.V[b2] = f.I->V;
          A.ld[b2] = f.n;
          A.nv[b2] = f.j + 1;
          A.h[b2] = f.I->hdev + off * (f.m + 1);
          A.w[b2] = f.I->w;
          A.n[b2] = f.n;
        }
        launch_multi_axpy_batch(A, nmax, -1.0, s);
      };
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice (CGS2)
        DotBatch D;
        int nvmax = 0;
        for (int i : inner) {
          FgMember& f = F[i];
          const int b2 = D.nb++;
          D.V[b2] = f.I->V;
          D.ld[b2] = f.n;
          D.nv[b2] = f.j + 1;
          D.w[b2] = f.I->w;
          D.n[b2] = f.n;
          D.part[b2] = f.I->part;
          D.out[b2] = f.I->hdev + pass * (f.m + 1);
          nvmax = std::max(nvmax, f.j + 1);
        }
        launch_multidot_batch(D, nvmax, s);
        axpy(pass);
      }
      {
        DotBatch D;
        for (int i : inner) {
          FgMember& f = F[i];
          const int b2 = D.nb++;
          D.V[b2] = f.I->w;
          D.ld[b2] = 0;
          D.nv[b2] = 1;
          D.w[b2] = f.I->w;
          D.n[b2] = f.n;
          D.part[b2] = f.I->part;
          D.out[b2] = f.I->hdev + 2 * (f.m + 1);
        }
        launch_multidot_batch(D, 1, s);
      }
      for (int i : inner)
        MSP_CUDA(cudaMemcpyAsync(F[i].I->hpin, F[i].I->hdev, sizeof(double) * (2 * (F[i].m + 1) + 1),
                                 cudaMemcpyDeviceToHost, s));
      MSP_CUDA(cudaStreamSynchronize(s));
      VecBatch nx;
      for (int i : inner) {
        FgMember& f = F[i];
        const int m = f.m, j = f.j;
        const double* hp = f.I->hpin;
        std::vector<double>& H = f.H;
        for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = hp[k] + hp[m + 1 + k];
        const double hn = std::sqrt(std::max(hp[2 * (m + 1)], 0.0));
        if (!std::isfinite(hn)) {
          f.status = MSP_ERR_NOT_CONVERGED;
          f.msg = "non-finite Arnoldi vector";
          f.phase = FgMember::DONE;
          continue;
        }
        H[(size_t)(j + 1) * m + j] = hn;
        for (int k = 0; k < j; ++k) {
          const double a = H[(size_t)k * m + j], c = H[(size_t)(k + 1) * m + j];
          H[(size_t)k * m + j] = f.cs[k] * a + f.sn[k] * c;
          H[(size_t)(k + 1) * m + j] = -f.sn[k] * a + f.cs[k] * c;
        }
        const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        const double den = std::hypot(a, c);
        f.cs[j] = den == 0.0 ? 1.0 : a / den;
        f.sn[j] = den == 0.0 ? 0.0 : c / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        f.g[j + 1] = -f.sn[j] * f.g[j];
        f.g[j] = f.cs[j] * f.g[j];
        ++f.it;
        if (hn <= 1e-300) {
          f.breakdown = true;
          f.j = j + 1;
          f.phase = FgMember::RESTART;
          continue;
        }
        nx.x[nx.nb] = f.I->w;
        nx.y[nx.nb] = vec(f, j + 1);
        nx.a[nx.nb] = 1.0 / hn;
        nx.n[nx.nb++] = f.n;
        f.j = j + 1;
        if (std::fabs(f.g[j + 1]) <= rtol * f.bnorm || f.j >= m || f.it >= f.I->h->opt.max_it)
          f.phase = FgMember::RESTART;
      }
      launch_vec_batch(nx, VEC_SCALE, nmax, s);
    }
    std::vector<int> rs;
    for (int i = 0; i < n; ++i)
      if (F[i].phase == FgMember::RESTART) rs.push_back(i);
    if (!rs.empty()) {
      AxpyBatch A;
      for (int i : rs) {
        FgMember& f = F[i];
        const int m = f.m, j = f.j;
        for (int k = j - 1; k >= 0; --k) {
          double sum = f.g[k];
          for (int q = k + 1; q < j; ++q) sum -= f.H[(size_t)k * m + q] * f.y[q];
          f.y[k] = sum / f.H[(size_t)k * m + k];
        }
        double* hp = f.I->hpin;
        for (int k = 0; k < j; ++k) hp[2 * (m + 1) + 1 + k] = f.y[k];
        MSP_CUDA(cudaMemcpyAsync(f.I->hdev + 2 * (m + 1) + 1, hp + 2 * (m + 1) + 1, sizeof(double) * j,
                                 cudaMemcpyHostToDevice, s));
        const int b2 = A.nb++;
        A.V[b2] = f.I->Z;
        A.ld[b2] = f.n;
        A.nv[b2] = j;
        A.h[b2] = f.I->hdev + 2 * (m + 1) + 1;
        A.w[b2] = f.x;
        A.n[b2] = f.n;
      }
      launch_multi_axpy_batch(A, nmax, 1.0, s);
      {
        std::vector<const double*> xx(n, nullptr), bb(n, nullptr);
        std::vector<double*> rr(n, nullptr);
        for (int i : rs) {
          xx[i] = F[i].x;
          rr[i] = F[i].I->res;
          bb[i] = F[i].b;
        }
        batch_spmv(B, 0, BOP_J, rs, xx, rr, bb, SPMV_RESIDUAL);
      }
      dots(rs, [](FgMember& f) { return (const double*)f.I->res; }, [](FgMember&) { return (int64_t)0; },
           [](FgMember&) { return 1; }, [](FgMember& f) { return (const double*)f.I->res; }, 0);
      if (int rc = sync_copy(rs, 1)) return rc;
      for (int i : rs) {
        FgMember& f = F[i];
        f.rnorm = std::sqrt(std::max(f.I->hpin[0], 0.0));
        f.phase = FgMember::CHECK;
        if (!std::isfinite(f.rnorm) || (f.breakdown && f.rnorm > rtol * f.bnorm)) f.phase = FgMember::DONE;
      }
    }
    bool live = false;
    for (const FgMember& f : F) live = live || f.phase != FgMember::DONE;
    if (!live) break;
  }
  MSP_CUDA(cudaGetLastError());
  // statuses: an expired bounded wait in a member's staged solves first
  int worst = MSP_OK;
  std::string worst_msg;
  for (int i = 0; i < n; ++i) {
    FgMember& f = F[i];
    int e = 0;
    MSP_CUDA(cudaMemcpyAsync(&e, f.I->ras_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    int rc = f.status;
    std::string msg = f.msg;
    if (e) {
      MSP_CUDA(cudaMemsetAsync(f.I->ras_err, 0, sizeof(int), s));
      MSP_CUDA(cudaStreamSynchronize(s));
      rc = MSP_ERR_TIMEOUT;
      msg = "a bounded wait in the staged RAS solve expired";
    } else if (rc == MSP_ERR_NOT_CONVERGED && msg.empty()) {
      msg = "FGMRES did not reach rtol within max_it (or broke down)";
    }
    if (st) {
      std::memset(&st[i], 0, sizeof(msp_stats));
      st[i].status = rc;
      st[i].iterations = f.it;
      st[i].rel_residual = f.bnorm > 0 ? f.rnorm / f.bnorm : 0.0;
    }
    if (rc != MSP_OK && worst == MSP_OK) {
      worst = rc;
      worst_msg = "member " + std::to_string(i) + ": " + msg;
    }
  }
  if (worst != MSP_OK) return fail(worst, worst_msg);
  return MSP_OK;
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace
}  // namespace msp

// =============================================================== C ABI
extern "C" {

void msp_default_options(msp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->delta = 1;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->restart = 30;
  o->max_it = 1000;
  o->factor_precision = MSP_F64;
  o->coef_kind = MSP_K_CONST;
  o->coef_scale = 1.0;
  o->load_kind = MSP_F_ONE;
  o->transfer = MSP_TRANSFER_BARY;
  o->restrict_scaling = 1;
  o->coarse_solver = MSP_COARSE_DIRECT;
  o->ilu_fill_fine = -1;
  o->ilu_fill_coarse = -1;
  o->pde = MSP_PDE_POISSON;
  o->poisson_ratio = 0.3;
  o->coupling = 1.0;
}

const char* msp_last_error(void) { return msp::g_last_error.c_str(); }
const char* msp_version(void) { return "msp 0.1 (sm_103a)"; }

int msp_load_hierarchy(const msp_level_desc* lv, int nlevels, const msp_options* o,
                       msp_hierarchy** out) {
  msp::g_last_error.clear();
  if (!lv || !o || !out || nlevels < 1) return fail(MSP_ERR_INVALID, "NULL argument or nlevels < 1");
  int rc = check_options(*o);
  if (rc) return rc;
  std::unique_ptr<msp_hierarchy> h(new (std::nothrow) msp_hierarchy());
  if (!h) return fail(MSP_ERR_OOM, "host allocation failed");
  h->opt = *o;
  h->host_only = o->host_only != 0;
  try {
    std::string err = build_host_levels(lv, nlevels, *o, h->host);
    if (!err.empty()) return fail(MSP_ERR_INVALID, err);
  } catch (const std::bad_alloc&) {
    return fail(MSP_ERR_OOM, "host allocation failed during set-up");
  }
  if (!h->host_only) {
    MSP_CUDA(cudaGetDevice(&h->device));
    if (o->factor_precision == MSP_BF16 || o->factor_precision == MSP_F64_TC) {  // these use the tensor cores
      rc = tensor_check(h->device);
      if (rc) return rc;
    }
    h->arena.al.a = o->alloc;
    h->arena.al.f = o->free;
    h->arena.al.ctx = o->alloc_ctx;
    h->dev.resize(nlevels);
    std::vector<int32_t> wave(24);
    for (int j = 0; j < 8; ++j)
      for (int d = 0; d < 3; ++d) wave[3 * j + d] = o->wave[j][d];
    h->wave = h->arena.upload(wave);
    cudaStream_t s;
    MSP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (int l = 0; l < nlevels; ++l) {
      rc = upload_level(h.get(), l, s);
      if (rc) {
        cudaStreamDestroy(s);
        h->arena.release();
        return rc;
      }
    }
    cudaStreamDestroy(s);
  }
  *out = h.release();
  return MSP_OK;
}

void msp_free_hierarchy(msp_hierarchy* h) {
  if (!h) return;
  if (!h->host_only) cudaDeviceSynchronize();
  h->arena.release();
  delete h;
}

int msp_instance_bytes(const msp_hierarchy* h, size_t* bytes) {
  if (!h || !bytes) return fail(MSP_ERR_INVALID, "NULL argument");
  if (h->host_only) return fail(MSP_ERR_INVALID, "host-only hierarchy");
  *bytes = instance_need(h);
  return MSP_OK;
}

int msp_hierarchy_info(const msp_hierarchy* h, int level, msp_level_info* info) {
  if (!h || !info || level < 0 || level >= (int)h->host.size())
    return fail(MSP_ERR_INVALID, "bad hierarchy, level or info pointer");
  const HostLevel& H = h->host[level];
  info->n_nodes = H.nv;
  info->n_dofs = H.n;
  info->n_tets = H.m;
  info->nnz = (int64_t)H.col.size();
  info->n_sub = H.direct ? 0 : H.nsub;
  info->sub_dofs = H.sub_ptr.empty() ? 0 : H.sub_ptr.back();
  info->factor_elems = H.sub_fac_off.empty() ? 0 : H.sub_fac_off.back();
  info->P_nnz = (int64_t)H.P_col.size();
  info->R_nnz = (int64_t)H.PT_col.size();
  info->fac_ctas = 0;
  info->ras_ctas = 0;
  info->spmv_lanes[0] = info->spmv_lanes[1] = info->spmv_lanes[2] = 0;
  if (!h->host_only) {
    const msp::DevLevel& D = h->dev[level];
    info->fac_ctas = D.fac_blocks ? D.fac_grid : 0;
    info->ras_ctas = H.direct ? 0 : D.ras_grid;
    info->spmv_lanes[0] = D.lpr_A;
    info->spmv_lanes[1] = H.P_col.empty() ? 0 : D.lpr_P;
    info->spmv_lanes[2] = H.PT_col.empty() ? 0 : D.lpr_PT;
  }
  return MSP_OK;
}

int msp_assemble(msp_hierarchy* h, const double* mu, int n_mu, void* stream, msp_instance** out) {
  msp::g_last_error.clear();
  if (!h || !out) return fail(MSP_ERR_INVALID, "NULL argument");
  if (h->host_only) return fail(MSP_ERR_INVALID, "host-only hierarchy");
  std::unique_ptr<msp_instance> I(new (std::nothrow) msp_instance());
  if (!I) return fail(MSP_ERR_OOM, "host allocation failed");
  I->h = h;
  I->stream = static_cast<cudaStream_t>(stream);
  // budget check before allocating
  const size_t need = instance_need(h);
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->opt.mem_budget_bytes && h->arena.bytes + h->instance_bytes + need > h->opt.mem_budget_bytes)
      return fail(MSP_ERR_OOM, "memory budget exceeded: instance needs " + std::to_string(need) + " bytes");
    h->instance_bytes += need;
  }
  I->charged = need;
  auto undo = [&](int rc) {
    I->arena.release();
    if (I->hpin) cudaFreeHost(I->hpin);
    for (int a = 0; a < 2; ++a) {
      if (I->aux[a]) cudaStreamDestroy(I->aux[a]);
      if (I->join[a]) cudaEventDestroy(I->join[a]);
    }
    if (I->fork) cudaEventDestroy(I->fork);
    if (I->cap) cudaStreamDestroy(I->cap);
    for (auto b : I->bulk)
      if (b) cudaStreamDestroy(b);
    for (auto& e : I->bev)
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    std::lock_guard<std::mutex> lk(h->mu);
    h->instance_bytes -= need;
    return rc;
  };
  int rc = alloc_instance(h, I.get());
  if (rc) return undo(rc);
  I->prof.init(I->stream);
  rc = set_mu(I.get(), mu, n_mu);
  if (rc) return undo(rc);
  *out = I.release();
  return MSP_OK;
}

int msp_reassemble(msp_instance* I, const double* mu, int n_mu) {
  msp::g_last_error.clear();
  if (!I) return fail(MSP_ERR_INVALID, "NULL instance");
  return set_mu(I, mu, n_mu);
}

void msp_free_instance(msp_instance* I) {
  if (!I) return;
  cudaStreamSynchronize(I->stream);
  for (int a = 0; a < 2; ++a) {
    if (I->aux[a]) cudaStreamDestroy(I->aux[a]);
    if (I->join[a]) cudaEventDestroy(I->join[a]);
  }
  if (I->fork) cudaEventDestroy(I->fork);
  if (I->cap) cudaStreamDestroy(I->cap);
  for (auto b : I->bulk)
    if (b) cudaStreamDestroy(b);
  for (auto& e : I->bev)
    for (auto x : e)
      if (x) cudaEventDestroy(x);
  if (I->fac_graph) cudaGraphExecDestroy(I->fac_graph);
  I->prof.destroy();
  I->arena.release();
  if (I->hpin) cudaFreeHost(I->hpin);
  {
    std::lock_guard<std::mutex> lk(I->h->mu);
    I->h->instance_bytes -= I->charged;
  }
  delete I;
}

int msp_factor(msp_instance* I) {
  msp::g_last_error.clear();
  if (!I || !I->assembled) return fail(MSP_ERR_INVALID, "instance not assembled");
  return factor_all(I);
}

int msp_factor_batch(msp_instance* const* insts, int n, void* stream) {
  msp::g_last_error.clear();
  if (!insts || n < 1) return fail(MSP_ERR_INVALID, "no instances");
  for (int i = 0; i < n; ++i) {
    msp_instance* I = insts[i];
    if (!I || !I->assembled) return fail(MSP_ERR_INVALID, "instance " + std::to_string(i) + " not assembled");
    for (int j = 0; j < i; ++j)
      if (insts[j] == I) return fail(MSP_ERR_INVALID, "an instance appears twice in the batch");
    const msp_hierarchy* h = I->h;
    for (int l = 0; l < (int)h->dev.size(); ++l)
      if (h->dev[l].ilu || level_store(h, l) == Store::BF16 || h->opt.factor_precision == MSP_F64_TC)
        return fail(MSP_ERR_INVALID, "batched factorisation takes FP64 / FP32 dense LU levels only");
  }
  cudaStream_t bs = stream ? static_cast<cudaStream_t>(stream) : insts[0]->stream;
  // every level of every instance on the instance's own streams, except the
  // blocks of the persistent levels, which are only extracted
  std::vector<BlockItem> items[2];  // FP64, FP32
  std::vector<int64_t> cost[2];
  for (int i = 0; i < n; ++i) {
    msp_instance* I = insts[i];
    int rc = enqueue_factor(I, I->stream, /*defer=*/true);
    if (rc) return rc;
    const msp_hierarchy* h = I->h;
    for (int l = 0; l < (int)h->dev.size(); ++l) {
      const DevLevel& D = h->dev[l];
      if (!D.fac_blocks) continue;
      MSP_CUDA(cudaStreamWaitEvent(bs, I->bev[l][0], 0));
      const HostLevel& H = h->host[l];
      const int g = level_store(h, l) == Store::F64 ? 0 : 1;
      for (int p = 0; p < H.nsub; ++p) {
        const int32_t* R = &H.tile_last[H.sub_trow[p]];
        int64_t c = 0;
        for (int k = 0; k < H.sub_nt[p]; ++k) {
          const int64_t rem = R[k] - k;
          c += 1 + rem + rem * (rem - 1) + rem;
        }
        items[g].push_back(BlockItem{I->fac[l], D.env, p, I->info});
        cost[g].push_back(c);
      }
    }
  }
  // one persistent launch per factor type, longest blocks first over the GPU
  int nsm = 0;
  MSP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, insts[0]->h->device));
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    for (void* b : bufs) cudaFree(b);
  };
  for (int g = 0; g < 2; ++g) {
    if (items[g].empty()) continue;
    const int per_sm = g == 0 ? ldlt_blocks_batch_per_sm<double>() : ldlt_blocks_batch_per_sm<float>();
    std::vector<int32_t> cptr, clist;
    lpt_lists(cost[g], std::max(1, std::min((int)items[g].size(), nsm * per_sm)), cptr, clist);
    void *d_items = nullptr, *d_ptr = nullptr, *d_list = nullptr;
    const size_t bi = items[g].size() * sizeof(BlockItem), bp = cptr.size() * 4, bl = clist.size() * 4;
    if (cudaMalloc(&d_items, bi) != cudaSuccess || cudaMalloc(&d_ptr, bp) != cudaSuccess ||
        cudaMalloc(&d_list, bl) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_items);
      cudaFree(d_ptr);
      cleanup();
      return fail(MSP_ERR_OOM, "device allocation failed for the batch work lists");
    }
    bufs.push_back(d_items);
    bufs.push_back(d_ptr);
    bufs.push_back(d_list);
    if (cudaMemcpy(d_items, items[g].data(), bi, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_ptr, cptr.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_list, clist.data(), bl, cudaMemcpyHostToDevice) != cudaSuccess) {
      cleanup();
      return fail(MSP_ERR_CUDA, "copying the batch work lists failed");
    }
    const int grid = (int)cptr.size() - 1;
    if (g == 0)
      launch_ldlt_blocks_batch<double>(static_cast<const BlockItem*>(d_items), static_cast<const int32_t*>(d_ptr),
                                       static_cast<const int32_t*>(d_list), grid, bs);
    else
      launch_ldlt_blocks_batch<float>(static_cast<const BlockItem*>(d_items), static_cast<const int32_t*>(d_ptr),
                                      static_cast<const int32_t*>(d_list), grid, bs);
  }
  cudaEvent_t done = nullptr;
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(done, bs) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(bs);
  } else {
    for (int i = 0; i < n; ++i) cudaStreamWaitEvent(insts[i]->stream, done, 0);
  }
  int rc = MSP_OK;
  for (int i = 0; i < n; ++i) {
    msp_instance* I = insts[i];
    int hinfo = 0;
    if (cudaMemcpyAsync(&hinfo, I->info, sizeof(int), cudaMemcpyDeviceToHost, I->stream) != cudaSuccess ||
        cudaStreamSynchronize(I->stream) != cudaSuccess) {
      rc = fail(MSP_ERR_CUDA, std::string("batched factorisation: ") + cudaGetErrorString(cudaGetLastError()));
      continue;
    }
    I->prof.harvest();
    if (hinfo) {
      rc = fail(MSP_ERR_INTERNAL, "non-positive or non-finite pivot in a subdomain factor of instance " +
                                      std::to_string(i));
      I->factored = false;
    } else {
      I->factored = true;
    }
  }
  cudaStreamSynchronize(bs);
  if (done) cudaEventDestroy(done);
  cleanup();
  return rc;
}

int msp_apply(msp_instance* I, const double* r, double* z, void* stream) {
  msp::g_last_error.clear();
  if (!I || !r || !z) return fail(MSP_ERR_INVALID, "NULL argument");
  if (!I->factored) return fail(MSP_ERR_INVALID, "instance not factored");
  if (r == z) return fail(MSP_ERR_INVALID, "r and z must not alias");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : I->stream;
  vcycle(I, r, z, s);
  MSP_CUDA(cudaGetLastError());
  return MSP_OK;
}

int msp_apply_op(msp_instance* I, int op, int level, const double* x, double* y, void* stream) {
  msp::g_last_error.clear();
  if (!I || !x || !y) return fail(MSP_ERR_INVALID, "NULL argument");
  msp_hierarchy* h = I->h;
  const int L = (int)h->dev.size();
  if (level < 0 || level >= L) return fail(MSP_ERR_INVALID, "level out of range");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : I->stream;
  switch (op) {
    case MSP_OP_SPMV: spmv(I, level, x, y, nullptr, SPMV_SET, s); break;
    case MSP_OP_RESIDUAL: spmv(I, level, x, y, nullptr, SPMV_SUB_FROM, s); break;
    case MSP_OP_INTERP:
      if (level + 1 >= L) return fail(MSP_ERR_INVALID, "no coarser level");
      transfer(I, level, false, x, y, SPMV_SET, s);
      break;
    case MSP_OP_RESTRICT:
      if (level + 1 >= L) return fail(MSP_ERR_INVALID, "no coarser level");
      transfer(I, level, true, x, y, SPMV_SET, s);
      break;
    case MSP_OP_RAS:
      if (direct_level(h, level)) return fail(MSP_ERR_INVALID, "the coarsest level is solved, not smoothed");
      if (!I->factored) return fail(MSP_ERR_INVALID, "instance not factored");
      ras(I, level, x, y, 0, s);
      break;
    case MSP_OP_COARSE:
      if (level != L - 1 || !direct_level(h, level))
        return fail(MSP_ERR_INVALID, "MSP_OP_COARSE needs the directly solved coarsest level");
      if (!I->factored) return fail(MSP_ERR_INVALID, "instance not factored");
      ras(I, level, x, y, 0, s);
      break;
    default: return fail(MSP_ERR_INVALID, "unknown op");
  }
  MSP_CUDA(cudaGetLastError());
  return MSP_OK;
}

int msp_solve(msp_instance* I, const double* b, double* x, double rtol, msp_stats* st) {
  msp::g_last_error.clear();
  msp_stats dummy;
  if (!st) st = &dummy;
  std::memset(st, 0, sizeof(*st));
  int rc;
  if (!I || !x) rc = fail(MSP_ERR_INVALID, "NULL argument");
  else if (!I->factored) rc = fail(MSP_ERR_INVALID, "instance not factored");
  else if (!(rtol > 0.0) || !std::isfinite(rtol)) rc = fail(MSP_ERR_INVALID, "rtol must be > 0");
  else {
    Timer tm;
    rc = fgmres(I, b ? b : I->h->dev[0].b, x, rtol, st);
    I->prof.harvest();
    st->ms_solve = tm.ms();
  }
  st->status = rc;
  return rc;
}

int msp_solve_host(msp_instance* I, const double* mu, int n_mu, const double* b_host,
                   double* x_host, double rtol, msp_stats* st) {
  msp::g_last_error.clear();
  msp_stats dummy;
  if (!st) st = &dummy;
  std::memset(st, 0, sizeof(*st));
  if (!I || !x_host) return st->status = fail(MSP_ERR_INVALID, "NULL argument");
  const int64_t n = I->h->dev[0].n;
  Timer t0;
  int rc = set_mu(I, mu, n_mu);
  st->ms_assemble = t0.ms();
  if (rc) return st->status = rc;
  Timer t1;
  rc = factor_all(I);
  st->ms_factor = t1.ms();
  if (rc) return st->status = rc;
  const double* b = nullptr;
  if (b_host) {
    if (cudaMemcpyAsync(I->xb + n, b_host, n * sizeof(double), cudaMemcpyHostToDevice, I->stream) != cudaSuccess)
      return st->status = fail(MSP_ERR_CUDA, "copy of b failed");
    b = I->xb + n;
  }
  double a = st->ms_assemble, f = st->ms_factor;
  rc = msp_solve(I, b, I->xb, rtol, st);
  st->ms_assemble = a;
  st->ms_factor = f;
  if (rc && rc != MSP_ERR_NOT_CONVERGED) return rc;
  int rc2 = rc;
  if (cudaMemcpyAsync(x_host, I->xb, n * sizeof(double), cudaMemcpyDeviceToHost, I->stream) != cudaSuccess ||
      cudaStreamSynchronize(I->stream) != cudaSuccess)
    return st->status = fail(MSP_ERR_CUDA, "copy of x failed");
  st->status = rc2;
  return rc2;
}

int msp_hierarchy_copy(const msp_hierarchy* h, int level, int what, void* dst, size_t cap,
                       size_t* bytes_out) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(MSP_ERR_INVALID, "bad hierarchy or level");
  const HostLevel& H = h->host[level];
  const void* src = nullptr;
  size_t bytes = 0;
  bool on_device = false;
  auto pick = [&](const auto& v) {
    src = v.data();
    bytes = v.size() * sizeof(v[0]);
  };
  switch (what) {
    case MSP_ARR_ROWPTR: pick(H.rowptr); break;
    case MSP_ARR_COL: pick(H.col); break;
    case MSP_ARR_SUB_PTR: pick(H.sub_ptr); break;
    case MSP_ARR_SUB_DOFS: pick(H.sub_dofs); break;
    case MSP_ARR_SUB_OWN: pick(H.sub_own); break;
    case MSP_ARR_P_ROWPTR: pick(H.P_rowptr); break;
    case MSP_ARR_P_COL: pick(H.P_col); break;
    case MSP_ARR_P_VAL: pick(H.P_val); break;
    case MSP_ARR_PT_ROWPTR: pick(H.PT_rowptr); break;
    case MSP_ARR_PT_COL: pick(H.PT_col); break;
    case MSP_ARR_PT_VAL: pick(H.PT_val); break;
    case MSP_ARR_SUB_NT: pick(H.sub_nt); break;
    case MSP_ARR_TILE_FIRST: pick(H.tile_first); break;
    case MSP_ARR_ILU_PTR: pick(H.ilu_lptr); break;
    case MSP_ARR_ILU_COL: pick(H.ilu_lcol); break;
    case MSP_ARR_LOAD:
      if (h->host_only) return fail(MSP_ERR_INVALID, "host-only hierarchy has no load vector");
      src = h->dev[level].b;
      bytes = (size_t)H.n * sizeof(double);
      on_device = true;
      break;
    default: return fail(MSP_ERR_INVALID, "unknown hierarchy array");
  }
  if (bytes_out) *bytes_out = bytes;
  if (!dst) return MSP_OK;
  if (cap < bytes) return fail(MSP_ERR_INVALID, "destination too small");
  if (bytes == 0) return MSP_OK;
  if (on_device) MSP_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  else std::memcpy(dst, src, bytes);
  return MSP_OK;
}

int msp_instance_copy(const msp_instance* I, int level, int what, int sub, void* dst, size_t cap,
                      size_t* bytes_out) {
  if (!I || level < 0 || level >= (int)I->h->dev.size()) return fail(MSP_ERR_INVALID, "bad instance or level");
  const msp_hierarchy* h = I->h;
  const DevLevel& D = h->dev[level];
  const HostLevel& H = h->host[level];
  const void* src = nullptr;
  size_t bytes = 0;
  if (what == MSP_ARR_VAL) {
    src = I->val[level];
    bytes = (size_t)D.nnz * sizeof(double);
  } else if (what == MSP_ARR_ILU_VAL || what == MSP_ARR_ILU_D) {
    if (!D.ilu) return fail(MSP_ERR_INVALID, "level has no ILU factors");
    const size_t es = store_bytes(level_store(h, level));  // double, or float for reduced precision
    const char* f = static_cast<const char*>(I->fac[level]);
    src = what == MSP_ARR_ILU_VAL ? f : f + (size_t)D.ilu_nnz * es;
    bytes = (size_t)(what == MSP_ARR_ILU_VAL ? D.ilu_nnz : D.ilu_rows) * es;
  } else if (what == MSP_ARR_FACTOR && D.ilu) {
    return fail(MSP_ERR_INVALID, "ILU level: read MSP_ARR_ILU_VAL / MSP_ARR_ILU_D");
  } else if (what == MSP_ARR_FACTOR) {
    const bool coarse = direct_level(h, level);
    int p = coarse ? 0 : sub;
    if (p < 0 || p >= H.nsub || (coarse && sub != -1 && sub != 0))
      return fail(MSP_ERR_INVALID, "subdomain out of range");
    size_t es = store_bytes(level_store(h, level));
    src = static_cast<const char*>(I->fac[level]) + (size_t)H.sub_fac_off[p] * es;
    bytes = (size_t)(H.sub_fac_off[p + 1] - H.sub_fac_off[p]) * es;
  } else {
    return fail(MSP_ERR_INVALID, "unknown instance array");
  }
  if (bytes_out) *bytes_out = bytes;
  if (!dst) return MSP_OK;
  if (cap < bytes) return fail(MSP_ERR_INVALID, "destination too small");
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  MSP_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  return MSP_OK;
}

// ---- per-kernel accounting (launch counts, algorithmic bytes/flops, and
// CUDA-event durations while profiling is on)
}  // extern "C"

struct msp_batch {
  msp::BatchState st;
};

extern "C" {

int msp_batch_create(msp_instance* const* insts, int n, void* stream, msp_batch** out) {
  msp::g_last_error.clear();
  if (!insts || !out) return fail(MSP_ERR_INVALID, "NULL argument");
  std::unique_ptr<msp_batch> b(new (std::nothrow) msp_batch());
  if (!b) return fail(MSP_ERR_OOM, "host allocation failed");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : (n > 0 && insts[0] ? insts[0]->stream : nullptr);
  const int rc = msp::batch_build(b->st, insts, n, s);
  if (rc) {
    msp::batch_release(b->st);
    return rc;
  }
  *out = b.release();
  return MSP_OK;
}

void msp_batch_free(msp_batch* b) {
  if (!b) return;
  msp::batch_release(b->st);
  delete b;
}

int msp_batch_assemble(msp_batch* bt, const double* mu, int n_mu) {
  msp::g_last_error.clear();
  if (!bt) return fail(MSP_ERR_INVALID, "NULL batch");
  return msp::batch_assemble(bt->st, mu, n_mu);
}

int msp_batch_factor(msp_batch* bt) {
  msp::g_last_error.clear();
  if (!bt) return fail(MSP_ERR_INVALID, "NULL batch");
  return msp::batch_factor(bt->st);
}

int msp_solve_batch(msp_batch* bt, const double* const* b_dev, double* const* x_dev, double rtol, msp_stats* st) {
  msp::g_last_error.clear();
  if (!bt || !x_dev) return fail(MSP_ERR_INVALID, "NULL argument");
  msp::BatchState& B = bt->st;
  const int n = (int)B.m.size();
  if (st) std::memset(st, 0, sizeof(msp_stats) * n);
  if (!(rtol > 0.0) || !std::isfinite(rtol)) return fail(MSP_ERR_INVALID, "rtol must be > 0");
  for (int i = 0; i < n; ++i) {
    if (!x_dev[i]) return fail(MSP_ERR_INVALID, "NULL solution pointer");
    if (!B.m[i]->factored) return fail(MSP_ERR_INVALID, "batch member " + std::to_string(i) + " not factored");
  }
  // the batch stream after every member's own stream, and back
  for (msp_instance* I : B.m) {
    if (I->stream == B.stream) continue;
    MSP_CUDA(cudaEventRecord(B.ev, I->stream));
    MSP_CUDA(cudaStreamWaitEvent(B.stream, B.ev, 0));
  }
  Timer tm;
  const int rc = msp::fgmres_batch(B, b_dev, x_dev, rtol, st);
  const double ms = tm.ms();
  if (st)
    for (int i = 0; i < n; ++i) st[i].ms_solve = ms;
  for (msp_instance* I : B.m) {
    if (I->stream == B.stream) continue;
    MSP_CUDA(cudaEventRecord(B.ev, B.stream));
    MSP_CUDA(cudaStreamWaitEvent(I->stream, B.ev, 0));
  }
  return rc;
}

int msp_debug_expire_waits(msp_instance* I, int count) {
  msp::g_last_error.clear();
  if (!I || count < 0) return fail(MSP_ERR_INVALID, "NULL instance or negative count");
  I->expire_ras = count;
  return MSP_OK;
}

int msp_debug_spread_work(msp_instance* I, int on) {
  msp::g_last_error.clear();
  if (!I) return fail(MSP_ERR_INVALID, "NULL instance");
  I->narrow_cluster = (on & 2) != 0;
  if (I->spread_work != ((on & 1) != 0)) {
    I->spread_work = (on & 1) != 0;
    if (I->fac_graph) {  // the captured factorisation holds the lists it was captured with
      MSP_CUDA(cudaStreamSynchronize(I->stream));
      cudaGraphExecDestroy(I->fac_graph);
      I->fac_graph = nullptr;
    }
  }
  return MSP_OK;
}

int msp_profile_enable(msp_instance* I, uint32_t class_mask) {
  if (!I) return fail(MSP_ERR_INVALID, "NULL instance");
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  I->prof.harvest();
  I->prof.mask = class_mask;
  return MSP_OK;
}

int msp_profile_reset(msp_instance* I) {
  if (!I) return fail(MSP_ERR_INVALID, "NULL instance");
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  I->prof.harvest();
  I->prof.reset();
  return MSP_OK;
}

int msp_profile_read(msp_instance* I, int kclass, msp_kernel_profile* out) {
  if (!I || !out || kclass < 0 || kclass >= PK_COUNT) return fail(MSP_ERR_INVALID, "bad argument");
  MSP_CUDA(cudaStreamSynchronize(I->stream));
  I->prof.harvest();
  *out = I->prof.c[kclass];
  return MSP_OK;
}

}  // extern "C"
