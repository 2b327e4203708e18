// Internal data structures of the msp library (host set-up + device state).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "msp.h"

namespace msp {

constexpr int kTile = MSP_TILE;             // factor tile edge
constexpr int kTileElems = kTile * kTile;   // elements per tile

// Pair slot of the symmetric 4x4 element matrix: (a,b), a <= b, row-major
// over the upper triangle: (0,0)=0 (0,1)=1 (0,2)=2 (0,3)=3 (1,1)=4 (1,2)=5
// (1,3)=6 (2,2)=7 (2,3)=8 (3,3)=9.
inline int pair_slot(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  static const int base[4] = {0, 4, 7, 9};
  return base[a] + (b - a);
}

inline int64_t tri_tiles(int nt) { return (int64_t)nt * (nt + 1) / 2; }

// Slot of entry (r, s) of the symmetric 12 x 12 element matrix of linear
// elasticity (row 3a+i: field i of local vertex a), row-major over the upper
// triangle: 78 slots.
inline int elastic_slot(int r, int s) {
  if (r > s) { int t = r; r = s; s = t; }
  return 12 * r - r * (r - 1) / 2 + (s - r);
}
constexpr int kElasticSlots = 78;

// Quadratic (P2) elements: local DoFs of a tet are its vertices 0..3, then
// its edges 01, 02, 03, 12, 13, 23; the symmetric 10 x 10 element matrix is
// stored by its upper triangle, row-major: 55 slots.
constexpr int kP2Slots = 55;
// The coupled two-field element (a P2 field u, local DoFs 0..9 as above, and
// a P1 field p, local DoFs 10..13 at the vertices): 14 x 14, 105 slots.
constexpr int kP2P1Slots = 105;
// slot of (r, s) in the upper triangle, row-major, of an n x n symmetric matrix
inline int sym_slot(int n, int r, int s) {
  if (r > s) { int t = r; r = s; s = t; }
  return n * r - r * (r - 1) / 2 + (s - r);
}
constexpr int kP2EdgeEnd[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Host-side structures of one level, built once per hierarchy.
struct HostLevel {
  // n: DoFs = fields x nv; xyz / tets are per vertex; dir, owner and dir_list
  // are per DoF (field c of vertex v is DoF fields*v + c)
  int n = 0, m = 0;
  int nv = 0, fields = 1;
  int nslot = 10;  // element-matrix slots per tet: 10 (P1), 78 (elasticity), 55 (P2), 105 (P2-P1)
  // P2 only: the global DoF of each of the 10 local DoFs of every tet, and
  // the point of every DoF (a vertex, or an edge's midpoint)
  bool p2 = false;
  int nloc = 10;                 // local DoFs per tet of the P2 forms: 10, or 14 with the P1 field p
  std::vector<int32_t> tdof;
  std::vector<double> dofx;
  std::vector<uint8_t> pdof;     // P2-P1: 1 for the DoFs of the P1 field
  std::vector<double> xyz;
  std::vector<int32_t> tets;
  std::vector<uint8_t> dir;
  std::vector<int32_t> owner;
  std::vector<int32_t> dir_list;       // Dirichlet DoF ids, ascending

  // CSR pattern of J (Section 2.1): vertices sharing a tet
  std::vector<int32_t> rowptr, col, diag;
  // element -> nonzero contributions: for nonzero q, contrib[cptr[q]..cptr[q+1])
  // are e*S+slot in ascending e (S = 10 element-matrix slots for one field,
  // 78 for elasticity); nzflag[q]: 0 assemble, 1 Dirichlet diagonal
  // (value 1), 2 Dirichlet-coupled (value 0)
  std::vector<int32_t> cptr, contrib;
  std::vector<uint8_t> nzflag;

  // subdomains (Section 2.2) on smoothed levels; one block of all interior
  // DoFs on the coarsest level
  bool direct = false;  // solved as one interior block (the coarsest, MSP_COARSE_DIRECT)
  int nsub = 0;
  std::vector<int32_t> sub_ptr;         // [nsub+1] offsets into sub_dofs
  std::vector<int32_t> sub_dofs;        // sorted DoFs of each subdomain
  std::vector<uint8_t> sub_own;         // owned flag (R^0) per entry of sub_dofs
  std::vector<int32_t> sub_nt;          // tiles per side NT_p
  // Tile envelope of every block (the blocks are ordered by ascending global
  // DoF id, which makes them banded): tile row I of subdomain p holds the
  // tiles (I, F_I) .. (I, I) contiguously; entries left of F_I are zero and
  // stay zero through the factorisation (fill stays inside the envelope).
  // Per-tile-row arrays are indexed by sub_trow[p] + I.
  std::vector<int32_t> sub_trow;        // [nsub+1] offsets into the per-tile-row arrays
  std::vector<int32_t> tile_first;      // F_I, nondecreasing in I
  std::vector<int32_t> tile_last;       // R_I = last tile row J with F_J <= I
  std::vector<int32_t> tile_off;        // index of tile (I, F_I) inside the subdomain storage
  std::vector<int64_t> sub_fac_off;     // [nsub+1] element offsets of each factor
  // dense extraction map: for subdomain p, entries ext_ptr[p]..ext_ptr[p+1]
  // give (absolute position in the level's factor storage, CSR nonzero index,
  // or -1 for a padding diagonal that is set to 1)
  std::vector<int64_t> ext_ptr;
  std::vector<int64_t> ext_pos;
  std::vector<int32_t> ext_nz;
  // work list of the factorisation: subdomains sorted by descending NT
  std::vector<int32_t> sub_order;

  // ILU(p) subdomain factors (Section 4.4) instead of the dense envelope when
  // ilu_fill >= 0.  Rows are numbered globally, row R = sub_ptr[p] + i for
  // local row i of subdomain p.  The factor is stored in symmetric form
  // (L unit lower, D; U = D L^T):
  //   ilu_lptr[R]..ilu_lptr[R+1]: strict lower pattern of row R, local
  //     columns ilu_lcol, values at the same positions of the L array;
  //   ilu_tptr/ilu_tcol/ilu_tslot: the transposed pattern (column R of L:
  //     rows j > i, with the L position of (j, i));
  //   ilu_fwd_rows / ilu_bwd_rows: local rows grouped by dependency level
  //     for the forward (rows need the rows of their pattern) and the
  //     backward sweep (rows need the rows whose pattern holds them); block p
  //     owns ilu_*_lvl[ilu_*_loff[p] .. ilu_*_loff[p+1]) (its level count + 1
  //     boundaries), level q spanning positions ilu_*_lvl[loff + q] ..
  //     ilu_*_lvl[loff + q + 1] of the rows arrays;
  //   ilu_ext_pos / ilu_ext_nz: extraction of the lower triangle of A_p into
  //     [L | D] (positions >= nnzL address D).
  //   ilu_fe_* / ilu_be_*: the entries each sweep reads, in the order the
  //     levels visit them (row position rr of ilu_*_rows owns entries
  //     ilu_*e_ptr[rr] .. [rr+1]: source column and L position), so that a
  //     level's entries are contiguous and can be fetched ahead;
  //   ilu_max_row: the most strictly-lower entries of one row.
  int ilu_fill = -1;
  int64_t ilu_nnz = 0;
  int ilu_max_n = 0, ilu_max_row = 0;
  std::vector<int64_t> ilu_fe_ptr, ilu_fe_slot, ilu_be_ptr, ilu_be_slot;
  std::vector<int32_t> ilu_fe_src, ilu_be_src;
  std::vector<int64_t> ilu_lptr, ilu_tptr, ilu_tslot, ilu_ext_pos;
  std::vector<int32_t> ilu_lcol, ilu_tcol, ilu_ext_nz;
  std::vector<int32_t> ilu_fwd_rows, ilu_fwd_lvl, ilu_fwd_loff;
  std::vector<int32_t> ilu_bwd_rows, ilu_bwd_lvl, ilu_bwd_loff;

  // prolongation from level+1 to this level (P or MLS) and restriction to
  // level+1 (P^T or MLS)
  std::vector<int32_t> P_rowptr, P_col, PT_rowptr, PT_col;
  std::vector<double> P_val, PT_val;
};

// Builds every host structure of a hierarchy; returns an empty string or an
// error message.
std::string build_host_levels(const msp_level_desc* lv, int nlevels, const msp_options& o,
                              std::vector<HostLevel>& out);

}  // namespace msp
