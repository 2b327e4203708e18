// Host-callable launchers of the msp CUDA kernels (sm_103a).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace msp {

// ---- per-tet geometry (set-up) and per-parameter coefficient / assembly
// kind 0 (P1): S[e*10+slot] = |T| grad(lambda_a).grad(lambda_b); kind 1
// (elasticity): the 78 upper-triangle slots of the unit-k 12 x 12 elasticity
// matrix (Lame lam, mu); kind 2 (P2): the 55 upper-triangle slots of the
// unit-k 10 x 10 quadratic-element matrix; kind 3 (P2-P1 pair): the 105
// slots of the 14 x 14 coupled element with coupling sigma = lam; vol[e] =
// |T|; cen[e*3] centroid
void launch_tet_geometry(const double* xyz, const int32_t* tets, int m, int kind, double lam, double mu,
                         double* S, double* vol, double* cen, int* bad, cudaStream_t s);
// b_i = f_c(x_v) * sum_{e containing v} |T_e| / 4 (ascending e) for DoF i =
// fields*v + c, 0 on Dirichlet DoFs; ns slots per tet in the contributions.
// With P2 elements (ns == 55, f = 1): b_i = sum_e int_e phi_i, -|T|/20 for a
// vertex DoF and |T|/5 for an edge DoF.
void launch_load_vector(const double* xyz, const uint8_t* dir, const int32_t* diag,
                        const int32_t* cptr, const int32_t* contrib, const double* vol, int n,
                        int load_kind, int fields, int ns, double lam, double mu, double* b,
                        cudaStream_t s);
// cw[8e + j] = cos(pi a_j . c_e), once per hierarchy (cosine coefficient)
void launch_coefficient_basis(const double* cen, int m, const int32_t* wave24, double* cw, cudaStream_t s);
// k_e = exp(s * sum_j mu_j 0.5 cw[8e + j])  (or 1; cw unused)
void launch_coefficient(const double* cw, int m, int coef_kind, const double* mu8, double scale, double* k,
                        cudaStream_t s);
// val[q] = sum_{c in contrib(q)} k[c/ns] * S[c]  (ascending e), Dirichlet flags
void launch_assemble(const int32_t* cptr, const int32_t* contrib, const uint8_t* nzflag,
                     const double* k, const double* S, int64_t nnz, int ns, double* val, cudaStream_t s);

// ---- CSR SpMV family (FP64)
enum SpmvMode { SPMV_SET = 0, SPMV_SUB_FROM = 1, SPMV_ADD = 2, SPMV_RESIDUAL = 3 };
// SET: y = A x; SUB_FROM: y = y - A x; ADD: y += A x; RESIDUAL: y = r - A x.
// Schedule: lpr = lanes per row (2, 4, 8, 16 or 32), or 1: one lane per row over
// the row blocks row_blk[0..nblk] (spmv_row_blocks), staged in shared memory.
struct SpmvPlan {
  int lpr = 8;
  const int32_t* row_blk = nullptr;  // device: nblk + 1 row offsets, then their nblk + 1 first nonzeros
  int nblk = 0;
  // lpr == kSpmvEll4: one thread per row of an operator with at most four
  // entries per row, stored as four columns and four values per row (padded
  // with weight 0 at column 0)
  const int4* ell_col = nullptr;
  const double2* ell_val = nullptr;
};
constexpr int kSpmvEll4 = 64;
// The four-entry form of a CSR matrix whose rows have at most four entries
// (empty when a row has more): columns [rows][4], values [rows][4].
bool spmv_ell4(const std::vector<int32_t>& rowptr, const std::vector<int32_t>& col, const std::vector<double>& val,
               std::vector<int32_t>& ecol, std::vector<double>& eval);
std::vector<int32_t> spmv_row_blocks(const std::vector<int32_t>& rowptr);
void launch_spmv(const int32_t* rowptr, const int32_t* col, const double* val, int nrows,
                 const double* x, double* y, const double* r, int mode, const SpmvPlan& plan,
                 cudaStream_t s);
// the fastest schedule (lpr) for this matrix, measured on the device with the
// L2 evicted before each launch (cached per structure for the life of the
// process); row_blk / nblk: its row blocks on the device (NULL: not a candidate);
// ell_col / ell_val: its four-entry form (NULL: not a candidate)
int tune_spmv(const int32_t* rowptr, const int32_t* col, int nrows, int ncols,
              const std::vector<int32_t>& h_rowptr, const std::vector<int32_t>& h_col,
              const int32_t* row_blk, int nblk, cudaStream_t s, const int4* ell_col = nullptr,
              const double2* ell_val = nullptr);

// ---- dense subdomain blocks (templated on the factor type T = double | float)
// Device view of a level's tile envelopes (see msp_internal.h).
struct EnvDev {
  const int64_t* fac_off;  // [nsub+1] element offset of each subdomain's tiles
  const int32_t* trow;     // [nsub+1] offset of subdomain p's tile rows
  const int32_t* first;    // F_I per tile row
  const int32_t* last;     // R_I per tile row
  const int32_t* toff;     // tile index of (I, F_I) in the subdomain's storage
  const int32_t* nt;       // NT_p
};
// zero the level's factor storage, then scatter the CSR values (or 1 on the
// padding diagonals, nz == -1) to their absolute positions
template <typename T>
void launch_extract(const int64_t* ext_pos, const int32_t* ext_nz, int64_t nent,
                    const double* val, int64_t fac_elems, T* fac, cudaStream_t s);
// step k of the blocked L D L^T over the first `nactive` subdomains of `order`
// (sorted by descending tile count, so those are exactly the ones with NT > k)
template <typename T>
void launch_ldlt_diag(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                      int* info, cudaStream_t s);
// panel tiles i = k+1+off .. k+off+max_rows of step k
template <typename T>
void launch_ldlt_panel(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                       int off, int max_rows, cudaStream_t s);
// trailing pairs pair0 .. pair0+max_pairs-1 of step k, numbered (1,1), (2,1),
// (2,2), (3,1), ... from k+1 (pair 0 is the next diagonal tile)
template <typename T>
void launch_ldlt_trail(T* fac, const EnvDev& E, const int32_t* order, int nactive, int k,
                       int pair0, int max_pairs, cudaStream_t s);
// after the tile steps of a level: the off-diagonal blocks of X in every
// diagonal tile (the diagonal kernel of the steps forms X's diagonal blocks
// only), over the first nblocks blocks of `order`
template <typename T>
void launch_ldlt_xfill(T* fac, const EnvDev& E, const int32_t* order, int nblocks, int max_nt, cudaStream_t s);
// after the factorisation of a level solved as one block on a cluster (block
// 0, nt tile rows): the coupling tiles M_I = L_{I,I-1} X_{I-1} and
// N_I^T = (X_{I+1} L_{I+1,I})^T and the reciprocals of D, written after the
// block's envelope (kBlockSolveExtra(nt) elements of T)
template <typename T>
void launch_ldlt_mnfill(T* fac, const EnvDev& E, int nt, cudaStream_t s);
constexpr int64_t kBlockSolveExtra(int nt) { return (int64_t)nt * (2 * 4096 + 64); }
// The whole L D L^T of many blocks in one persistent launch: CTA b factors
// cta_list[cta_ptr[b] .. cta_ptr[b+1]) through every tile step.
template <typename T>
void launch_ldlt_blocks(T* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                        int grid, int* info, cudaStream_t s);
template <typename T>
int ldlt_blocks_per_sm();
// Blocks of several levels / instances in one persistent launch: item q is
// block p of the level whose envelope is E, stored at fac (T*), status word
// info; CTA b factors items cta_list[cta_ptr[b] .. cta_ptr[b+1]).
struct BlockItem {
  void* fac;
  EnvDev E;
  int32_t p;
  int* info;
};
// sm_ctr == nullptr: CTA b factors the items cta_list[cta_ptr[b] .. cta_ptr[b+1]).
// Else the lists are per SM (nbins of them): a CTA takes items from its own
// SM's list, then from lists no CTA of their SM works on; sm_ctr[2 nbins]
// must be zero at launch.
template <typename T>
void launch_ldlt_blocks_batch(const BlockItem* items, const int32_t* cta_ptr, const int32_t* cta_list, int grid,
                              cudaStream_t s, int* sm_ctr = nullptr, int nbins = 0);
template <typename T>
int ldlt_blocks_batch_per_sm();
// Persistent factorisation of the blocks of a level whose factors are stored
// in BF16: FP32 diagonal tiles and panels, trailing updates on the tensor
// cores (BF16 operands, FP32 accumulation), fac = the FP32 working envelope.
void launch_ldlt_blocks_tc(float* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                           int grid, int* info, cudaStream_t s);
int ldlt_blocks_tc_per_sm();
// FP64 factors with the panel and trailing products on the BF16 tensor cores
// by exact digit slices (one CTA per SM); status bit 2 on an expired wait
void launch_ldlt_blocks_oz(double* fac, const EnvDev& E, const int32_t* cta_ptr, const int32_t* cta_list,
                           int grid, int* info, cudaStream_t s);
int ldlt_blocks_oz_per_sm();
// ---- ILU(p) subdomain factors (k_ilu.cu); fac = [L (nnz) | D (rows) | 1/D (rows)]
// of T = double or float (factorisation and sweeps in T).  es = sizeof(T).
size_t ilu_factor_smem(int max_n, int max_row, size_t es);  // max_row: most strictly-lower entries of a row
size_t ilu_solve_smem(int max_n, size_t es);
template <typename T>
void launch_ilu_extract(const int64_t* pos, const int32_t* nz, int64_t nent, const double* val, int64_t total,
                        T* fac, cudaStream_t s);
template <typename T>
void launch_ilu_factor(T* fac, int64_t nnz, int64_t rows, int nsub, const int32_t* sub_ptr,
                       const int64_t* lptr, const int32_t* lcol, const int32_t* fwd_rows,
                       const int32_t* fwd_lvl, const int32_t* fwd_loff, int max_n, int max_row, int* info,
                       cudaStream_t s);
// fac = [L | D | 1/D | Lf | Lb]: Lf, Lb the level-major copies (launch_ilu_gather)
template <typename T>
void launch_ilu_gather(T* fac, int64_t nnz, int64_t rows, const int64_t* fe_slot, const int64_t* be_slot,
                       cudaStream_t s);
template <typename T>
void launch_ilu_solve(const T* fac, int64_t nnz, int64_t rows, int nsub, const int32_t* sub_ptr,
                      const int32_t* dofs, const uint8_t* own, const int64_t* fe_ptr, const int32_t* fe_src,
                      const int64_t* be_ptr, const int32_t* be_src, const int32_t* fwd_rows,
                      const int32_t* fwd_lvl, const int32_t* fwd_loff, const int32_t* bwd_rows,
                      const int32_t* bwd_lvl, const int32_t* bwd_loff, int max_n,
                      const int32_t* dir_list, int ndir, const double* t, double* z, int add, cudaStream_t s);
// BF16 storage of factors computed in FP32: dst = bf16(src) to nearest even,
// n a multiple of 4.
void launch_round_bf16(const float* src, __nv_bfloat16* dst, int64_t n, cudaStream_t s);
// ---- triangular solves with the tiled factors (k_ras.cu)
// One level of one instance as the solves see it: its factors (T*), their
// envelope, the subdomains (DoF lists, owned flags), the Dirichlet DoFs and
// the error word of the staged solve.  A launch takes an array of views (the
// same level of several instances of a batch, or a single one) and, per view,
// its input t and output z (z == NULL: the view sits the launch out).
constexpr int kMaxBatch = 32;
constexpr int kViewShift = 20;  // CTA-list entries (view << kViewShift) | block, block < 2^20
struct RasView {
  const void* fac;
  EnvDev E;
  const int32_t* sub_ptr;
  const int32_t* dofs;
  const uint8_t* own;
  const int32_t* dir_list;
  int ndir;
  int* err;
};
struct RasVecs {
  const double* t[kMaxBatch];
  double* z[kMaxBatch];
};
// z = B^{-1} t on one level: per subdomain y = (L D L^T)^{-1} t[dofs], owned
// entries written (add = 0) or added (add = 1) to z; Dirichlet nodes get t.
// CTA b solves the items cta_list[cta_ptr[b] .. cta_ptr[b+1]) (a
// longest-first balanced assignment built on the host); a bounded mbarrier
// wait that expires sets bit 4 of the item's view's err.  The factor tiles
// stream through ras_slots<T>(max_nt) shared-memory slots (max_nt: the most
// tiles per side of any block of any view); each sweep holds one tile at a
// time (the backward sweep takes a row's column tiles, then its diagonal
// tile), so two slots are enough to make progress (checked on the host at
// set-up); deeper rings let the producer run further ahead.
// `wide`: one CTA of 16 consumer warps per SM (always the FP64 form); else
// FP32 / BF16 run 2 / 3 smaller CTAs per SM, each with fewer ring slots.
// `inject` != 0 (failure-injection tests only): no tile copy is issued, every
// wait on a full slot runs out after a short limit and bit 4 of err is set.
template <typename T>
int ras_slots(int max_nt, bool wide);
// CTAs of k_ras_solve that share an SM (the persistent grid is this x SMs)
template <typename T>
int ras_ctas_per_sm(bool wide);
// claim != nullptr: the grid's lists come per_sm to each of nbins SMs and a
// CTA takes its SM's (claim[nbins + grid] ints, zero at launch); else CTA b
// takes list b.
template <typename T>
void launch_ras_solve(const RasView* views, int nviews, const RasVecs& vecs, const int32_t* cta_ptr,
                      const int32_t* cta_list, int grid, int max_nt, int add, bool wide, cudaStream_t s,
                      int inject = 0, int* claim = nullptr, int nbins = 0);
// y = (L D L^T)^{-1} t of a level made of ONE block (the coarsest level) for
// each of `nviews` views, each on a cluster of 16 CTAs (8 where the GPU cannot
// place 16) that split every tile row of both sweeps and exchange partial
// results through distributed shared memory, one exchange per tile row; the factor must carry the coupling
// tiles of launch_ldlt_mnfill after its envelope.  Dirichlet nodes get t.
// Written (add = 0) or added (add = 1) to z.
size_t block_solve_cluster_smem(int max_nt);  // dynamic shared memory of one CTA
template <typename T>
void launch_block_solve_cluster(const RasView* views, int nviews, const RasVecs& vecs, int max_nt, int add,
                                cudaStream_t s, bool narrow = false);  // narrow: always the 8-CTA form

// ---- batched launches: one launch for several instances of a batch, each
// member's arithmetic exactly that of its own one-member launch.  Members are
// described in parameter arrays of kMaxBatch entries; a member whose output
// pointer is NULL sits the launch out.
constexpr int kMaxMembers = 32;
// One SpMV family over the members' stacked rows (row blocks for lpr == 1):
// member b owns start[b] .. start[b+1]; every member uses the schedule lpr.
struct SpmvBatch {
  int nb = 0, lpr = 8, mode = 0;
  int64_t start[kMaxMembers + 1] = {};
  const int32_t* rowptr[kMaxMembers] = {};
  const int32_t* col[kMaxMembers] = {};
  const double* val[kMaxMembers] = {};
  const int32_t* row_blk[kMaxMembers] = {};  // lpr == 1: nblk + 1 row offsets, then their first nonzeros
  int nblk[kMaxMembers] = {};
  const int4* ell_col[kMaxMembers] = {};
  const double2* ell_val[kMaxMembers] = {};
  const double* x[kMaxMembers] = {};
  double* y[kMaxMembers] = {};
  const double* r[kMaxMembers] = {};
};
void launch_spmv_batch(const SpmvBatch& B, cudaStream_t s);
// out_b[i] = V_b[i] . w_b, i < nv[b], partials in part_b (nv[b] x kDotBlocks)
struct DotBatch {
  int nb = 0;
  const double* V[kMaxMembers] = {};
  int64_t ld[kMaxMembers] = {};
  int nv[kMaxMembers] = {};
  const double* w[kMaxMembers] = {};
  int64_t n[kMaxMembers] = {};
  double* part[kMaxMembers] = {};
  double* out[kMaxMembers] = {};
};
void launch_multidot_batch(const DotBatch& B, int nv_max, cudaStream_t s);
// w_b -= / += sum_i h_b[i] V_b[i], i < nv[b] (h on the device)
struct AxpyBatch {
  int nb = 0;
  const double* V[kMaxMembers] = {};
  int64_t ld[kMaxMembers] = {};
  int nv[kMaxMembers] = {};
  const double* h[kMaxMembers] = {};
  double* w[kMaxMembers] = {};
  int64_t n[kMaxMembers] = {};
};
void launch_multi_axpy_batch(const AxpyBatch& B, int64_t n_max, double sign, cudaStream_t s);
enum VecOp { VEC_SCALE = 0, VEC_COPY = 1, VEC_FILL = 2 };
struct VecBatch {
  int nb = 0;
  const double* x[kMaxMembers] = {};
  double* y[kMaxMembers] = {};
  double a[kMaxMembers] = {};
  int64_t n[kMaxMembers] = {};
};
void launch_vec_batch(const VecBatch& B, int op, int64_t n_max, cudaStream_t s);

// ---- Krylov helpers (deterministic two-stage reductions)
// out[i] = sum_k V[i*ld + k] * w[k], i < nv; part: scratch of nv * kDotBlocks doubles
constexpr int kDotBlocks = 296;
void launch_multidot(const double* V, int64_t ld, int nv, const double* w, int64_t n,
                     double* part, double* out, cudaStream_t s);
// w -= sum_i h[i] V_i  (h on the device)
void launch_multi_axpy(const double* V, int64_t ld, int nv, const double* h, double* w,
                       int64_t n, double sign, cudaStream_t s);
// y = alpha * x (alpha read from the host argument)
void launch_scale(const double* x, double alpha, double* y, int64_t n, cudaStream_t s);
void launch_axpy(double alpha, const double* x, double* y, int64_t n, cudaStream_t s);
void launch_add_vec(const double* a, double* b, int64_t n, cudaStream_t s);  // b += a
void launch_fill(double* y, double v, int64_t n, cudaStream_t s);
void launch_copy(const double* x, double* y, int64_t n, cudaStream_t s);

}  // namespace msp
