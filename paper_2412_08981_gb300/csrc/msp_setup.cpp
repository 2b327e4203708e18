// Host-side set-up of a mesh hierarchy (done once, reused for every mu).
//
// Everything here is index bookkeeping and geometry that the paper treats as
// set-up (Algorithm 2, "construct the hierarchy"; Section 2.2 partition and
// overlap; the point location behind the interpolation weights):
//   * CSR pattern of J on every level and the element->nonzero map used by
//     the device assembly kernel,
//   * delta-overlapping subdomains and their dense extraction maps,
//   * the transfers between consecutive levels: barycentric interpolation P
//     and P^T, or the overlapping MLS operators of Section 3.2 (the weights
//     are set-up; applying them is a sparse product on the device).
#include <algorithm>
#include <climits>
#include <functional>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "msp_internal.h"

namespace msp {
namespace {

// vertex -> incident tets, ascending tet id (counting sort)
void vertex_tets(const HostLevel& L, std::vector<int32_t>& ptr, std::vector<int32_t>& adj) {
  ptr.assign(L.n + 1, 0);
  for (int64_t k = 0; k < 4 * (int64_t)L.m; ++k) ptr[L.tets[k] + 1]++;
  for (int i = 0; i < L.n; ++i) ptr[i + 1] += ptr[i];
  adj.resize(ptr[L.n]);
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
  for (int e = 0; e < L.m; ++e)
    for (int a = 0; a < 4; ++a) adj[fill[L.tets[4 * e + a]]++] = e;
}

int32_t find_in_row(const HostLevel& L, int i, int j) {
  const int32_t* b = L.col.data() + L.rowptr[i];
  const int32_t* e = L.col.data() + L.rowptr[i + 1];
  const int32_t* it = std::lower_bound(b, e, j);
  return (it != e && *it == j) ? (int32_t)(it - L.col.data()) : -1;
}

void build_pattern_and_contribs(HostLevel& L) {
  std::vector<int32_t> vptr, vadj;
  vertex_tets(L, vptr, vadj);
  // pattern: per row, the sorted distinct vertices of the incident tets
  L.rowptr.assign(L.n + 1, 0);
  std::vector<int32_t> buf;
  std::vector<std::vector<int32_t>> rows(L.n);
  for (int i = 0; i < L.n; ++i) {
    buf.clear();
    for (int k = vptr[i]; k < vptr[i + 1]; ++k) {
      const int32_t* t = &L.tets[4 * (int64_t)vadj[k]];
      buf.insert(buf.end(), t, t + 4);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    rows[i] = buf;
    L.rowptr[i + 1] = L.rowptr[i] + (int32_t)buf.size();
  }
  L.col.resize(L.rowptr[L.n]);
  L.diag.resize(L.n);
  for (int i = 0; i < L.n; ++i) {
    std::copy(rows[i].begin(), rows[i].end(), L.col.begin() + L.rowptr[i]);
    L.diag[i] = find_in_row(L, i, i);
  }
  rows.clear();
  rows.shrink_to_fit();
  const int64_t nnz = L.col.size();
  // nonzero flags and contribution lists (ascending tet id per nonzero)
  L.nzflag.assign(nnz, 0);
  std::vector<int32_t> cnt(nnz, 0);
  for (int i = 0; i < L.n; ++i)
    for (int q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
      int j = L.col[q];
      if (L.dir[i]) L.nzflag[q] = (i == j) ? 1 : 2;
      else if (L.dir[j]) L.nzflag[q] = 2;
    }
  for (int i = 0; i < L.n; ++i) {
    if (L.dir[i]) continue;
    for (int k = vptr[i]; k < vptr[i + 1]; ++k) {
      const int32_t* t = &L.tets[4 * (int64_t)vadj[k]];
      for (int b = 0; b < 4; ++b) {
        int32_t q = find_in_row(L, i, t[b]);
        if (L.nzflag[q] == 0) cnt[q]++;
      }
    }
  }
  L.cptr.assign(nnz + 1, 0);
  for (int64_t q = 0; q < nnz; ++q) L.cptr[q + 1] = L.cptr[q] + cnt[q];
  L.contrib.resize(L.cptr[nnz]);
  std::vector<int32_t> fill(L.cptr.begin(), L.cptr.end() - 1);
  for (int i = 0; i < L.n; ++i) {
    if (L.dir[i]) continue;
    for (int k = vptr[i]; k < vptr[i + 1]; ++k) {  // tets in ascending id
      int e = vadj[k];
      const int32_t* t = &L.tets[4 * (int64_t)e];
      int a = 0;
      while (t[a] != i) ++a;
      for (int b = 0; b < 4; ++b) {
        int32_t q = find_in_row(L, i, t[b]);
        if (L.nzflag[q] == 0) L.contrib[fill[q]++] = e * 10 + pair_slot(a, b);
      }
    }
  }
}

// Subdomains: one per partition id owning a non-Dirichlet vertex, ascending
// id; overlap by delta breadth-first layers over the vertex graph (a layer
// adds every vertex of every tet touching the current set).
void build_subdomains(HostLevel& L, int delta) {
  std::vector<int32_t> ids;
  for (int i = 0; i < L.n; ++i)
    if (!L.dir[i]) ids.push_back(L.owner[i]);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  L.nsub = (int)ids.size();
  // vertices grouped by owner id (all vertices, Dirichlet ones included)
  std::vector<int32_t> order(L.n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return L.owner[a] < L.owner[b]; });
  std::vector<std::vector<int32_t>> dofs(L.nsub);
  std::vector<std::vector<uint8_t>> own(L.nsub);
  auto work = [&](int p0, int p1) {
    std::vector<int32_t> stamp(L.n, -1), frontier, next, members;
    for (int p = p0; p < p1; ++p) {
      int id = ids[p];
      auto lo = std::lower_bound(order.begin(), order.end(), id,
                                 [&](int v, int key) { return L.owner[v] < key; });
      members.clear();
      frontier.clear();
      for (auto it = lo; it != order.end() && L.owner[*it] == id; ++it) {
        stamp[*it] = p;
        members.push_back(*it);
        frontier.push_back(*it);
      }
      for (int layer = 0; layer < delta; ++layer) {
        next.clear();
        for (int v : frontier)
          for (int q = L.rowptr[v]; q < L.rowptr[v + 1]; ++q) {
            int w = L.col[q];
            if (stamp[w] != p) {
              stamp[w] = p;
              members.push_back(w);
              next.push_back(w);
            }
          }
        frontier.swap(next);
      }
      std::vector<int32_t> d;
      for (int v : members)
        if (!L.dir[v]) d.push_back(v);
      std::sort(d.begin(), d.end());
      std::vector<uint8_t> o(d.size());
      for (size_t k = 0; k < d.size(); ++k) o[k] = (L.owner[d[k]] == id) ? 1 : 0;
      dofs[p] = std::move(d);
      own[p] = std::move(o);
    }
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  nth = std::min(nth, std::max(1, L.nsub));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)L.nsub * t / nth), (int)((int64_t)L.nsub * (t + 1) / nth));
  for (auto& t : th) t.join();
  L.sub_ptr.assign(L.nsub + 1, 0);
  for (int p = 0; p < L.nsub; ++p) L.sub_ptr[p + 1] = L.sub_ptr[p] + (int32_t)dofs[p].size();
  L.sub_dofs.resize(L.sub_ptr[L.nsub]);
  L.sub_own.resize(L.sub_ptr[L.nsub]);
  for (int p = 0; p < L.nsub; ++p) {
    std::copy(dofs[p].begin(), dofs[p].end(), L.sub_dofs.begin() + L.sub_ptr[p]);
    std::copy(own[p].begin(), own[p].end(), L.sub_own.begin() + L.sub_ptr[p]);
  }
}

void build_coarsest_block(HostLevel& L) {
  L.nsub = 1;
  L.sub_ptr.assign(2, 0);
  L.sub_dofs.clear();
  for (int i = 0; i < L.n; ++i)
    if (!L.dir[i]) L.sub_dofs.push_back(i);
  L.sub_ptr[1] = (int32_t)L.sub_dofs.size();
  L.sub_own.assign(L.sub_dofs.size(), 1);
}

// Tiled envelope layout and the CSR -> dense-block extraction map.  Only the
// lower triangle (li >= lj) is extracted: the blocks are symmetric.
void build_factor_layout(HostLevel& L) {
  L.sub_nt.resize(L.nsub);
  L.sub_trow.assign(L.nsub + 1, 0);
  for (int p = 0; p < L.nsub; ++p) {
    int np_ = L.sub_ptr[p + 1] - L.sub_ptr[p];
    L.sub_nt[p] = (np_ + kTile - 1) / kTile;
    L.sub_trow[p + 1] = L.sub_trow[p] + L.sub_nt[p];
  }
  const int ntr = L.sub_trow[L.nsub];
  L.tile_first.assign(ntr, 0);
  L.tile_last.assign(ntr, 0);
  L.tile_off.assign(ntr, 0);
  L.sub_fac_off.assign(L.nsub + 1, 0);
  std::vector<int32_t> loc(L.n, -1);
  // pass 1: envelope of every block
  for (int p = 0; p < L.nsub; ++p) {
    const int32_t* d = &L.sub_dofs[L.sub_ptr[p]];
    const int np_ = L.sub_ptr[p + 1] - L.sub_ptr[p];
    const int nt = L.sub_nt[p];
    int32_t* F = &L.tile_first[L.sub_trow[p]];
    for (int I = 0; I < nt; ++I) F[I] = I;
    for (int li = 0; li < np_; ++li) loc[d[li]] = li;
    for (int li = 0; li < np_; ++li) {
      int i = d[li];
      for (int q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
        int lj = loc[L.col[q]];
        if (lj >= 0 && lj <= li) F[li / kTile] = std::min(F[li / kTile], lj / kTile);
      }
    }
    for (int li = 0; li < np_; ++li) loc[d[li]] = -1;
    for (int I = nt - 2; I >= 0; --I) F[I] = std::min(F[I], F[I + 1]);  // monotone
    int32_t* R = &L.tile_last[L.sub_trow[p]];
    int32_t* O = &L.tile_off[L.sub_trow[p]];
    int64_t ntiles = 0;
    for (int I = 0; I < nt; ++I) {
      O[I] = (int32_t)ntiles;
      ntiles += I - F[I] + 1;
      int J = I;
      while (J + 1 < nt && F[J + 1] <= I) ++J;
      R[I] = J;
    }
    L.sub_fac_off[p + 1] = L.sub_fac_off[p] + ntiles * kTileElems;
  }
  // pass 2: extraction positions
  L.ext_ptr.assign(L.nsub + 1, 0);
  std::vector<int64_t> pos;
  std::vector<int32_t> nz;
  for (int p = 0; p < L.nsub; ++p) {
    const int64_t base = L.sub_fac_off[p];
    const int32_t* d = &L.sub_dofs[L.sub_ptr[p]];
    const int np_ = L.sub_ptr[p + 1] - L.sub_ptr[p];
    const int32_t* F = &L.tile_first[L.sub_trow[p]];
    const int32_t* O = &L.tile_off[L.sub_trow[p]];
    auto at = [&](int li, int lj) {
      int I = li / kTile, J = lj / kTile;
      return base + (int64_t)(O[I] + (J - F[I])) * kTileElems + (li % kTile) * kTile + (lj % kTile);
    };
    for (int li = 0; li < np_; ++li) loc[d[li]] = li;
    for (int li = 0; li < np_; ++li) {
      int i = d[li];
      for (int q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
        int lj = loc[L.col[q]];
        if (lj < 0 || lj > li) continue;
        pos.push_back(at(li, lj));
        nz.push_back(q);
      }
    }
    for (int li = np_; li < L.sub_nt[p] * kTile; ++li) {  // identity padding
      pos.push_back(at(li, li));
      nz.push_back(-1);
    }
    for (int li = 0; li < np_; ++li) loc[d[li]] = -1;
    L.ext_ptr[p + 1] = (int64_t)pos.size();
  }
  L.ext_pos.swap(pos);
  L.ext_nz.swap(nz);
  L.sub_order.resize(L.nsub);
  std::iota(L.sub_order.begin(), L.sub_order.end(), 0);
  std::stable_sort(L.sub_order.begin(), L.sub_order.end(),
                   [&](int a, int b) { return L.sub_nt[a] > L.sub_nt[b]; });
}

// ------------------------------------------------------ point location
// Barycentric coordinates by Cramer's rule on the 3x3 edge system.
inline double det3(const double* a, const double* b, const double* c) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
         a[2] * (b[0] * c[1] - b[1] * c[0]);
}

void bary(const HostLevel& C, int e, const double* x, double lam[4]) {
  const int32_t* t = &C.tets[4 * (int64_t)e];
  const double* p0 = &C.xyz[3 * (int64_t)t[0]];
  double c1[3], c2[3], c3[3], d[3];
  for (int k = 0; k < 3; ++k) {
    c1[k] = C.xyz[3 * (int64_t)t[1] + k] - p0[k];
    c2[k] = C.xyz[3 * (int64_t)t[2] + k] - p0[k];
    c3[k] = C.xyz[3 * (int64_t)t[3] + k] - p0[k];
    d[k] = x[k] - p0[k];
  }
  // columns c1 c2 c3: solve [c1 c2 c3] l = d
  double D = det3(c1, c2, c3);
  lam[1] = det3(d, c2, c3) / D;
  lam[2] = det3(c1, d, c3) / D;
  lam[3] = det3(c1, c2, d) / D;
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

struct TetGrid {
  int G = 1;
  double lo[3], inv[3];
  std::vector<int32_t> ptr, ids;
  int cell(double v, int d) const {
    int c = (int)std::floor((v - lo[d]) * inv[d]);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
  }
};

void build_grid(const HostLevel& C, TetGrid& g) {
  double hi[3] = {-1e300, -1e300, -1e300};
  for (int d = 0; d < 3; ++d) g.lo[d] = 1e300;
  // the mesh's vertices (xyz holds nv points; with P2 elements n also counts
  // the edge DoFs)
  for (int i = 0; i < C.nv; ++i)
    for (int d = 0; d < 3; ++d) {
      g.lo[d] = std::min(g.lo[d], C.xyz[3 * (int64_t)i + d]);
      hi[d] = std::max(hi[d], C.xyz[3 * (int64_t)i + d]);
    }
  g.G = std::max(1, (int)std::lround(std::cbrt((double)C.m / 2.0)));
  double ext[3];
  for (int d = 0; d < 3; ++d) {
    ext[d] = std::max(hi[d] - g.lo[d], 1e-300);
    g.inv[d] = g.G / ext[d];
  }
  size_t ncell = (size_t)g.G * g.G * g.G;
  std::vector<int32_t> cnt(ncell + 1, 0);
  auto range = [&](int e, int c0[3], int c1[3]) {
    double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) {
        double v = C.xyz[3 * (int64_t)C.tets[4 * (int64_t)e + a] + d];
        blo[d] = std::min(blo[d], v);
        bhi[d] = std::max(bhi[d], v);
      }
    for (int d = 0; d < 3; ++d) {
      double pad = 1e-8 * ext[d];
      c0[d] = g.cell(blo[d] - pad, d);
      c1[d] = g.cell(bhi[d] + pad, d);
    }
  };
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int32_t> fill;
    if (pass == 1) {
      g.ptr.assign(ncell + 1, 0);
      for (size_t c = 0; c < ncell; ++c) g.ptr[c + 1] = g.ptr[c] + cnt[c];
      g.ids.resize(g.ptr[ncell]);
      fill.assign(g.ptr.begin(), g.ptr.end() - 1);
    }
    for (int e = 0; e < C.m; ++e) {  // ascending id: each cell list is sorted
      int c0[3], c1[3];
      range(e, c0, c1);
      for (int k = c0[2]; k <= c1[2]; ++k)
        for (int j = c0[1]; j <= c1[1]; ++j)
          for (int i = c0[0]; i <= c1[0]; ++i) {
            size_t c = (size_t)i + (size_t)g.G * ((size_t)j + (size_t)g.G * k);
            if (pass == 0) cnt[c]++;
            else g.ids[fill[c]++] = e;
          }
    }
  }
}

// P: rows of fine non-Dirichlet nodes hold the barycentric weights of the
// containing coarse tet (smallest id among those whose weights are all
// >= -1e-12; if none, the tet whose smallest weight is largest), on that tet's
// non-Dirichlet vertices, columns ascending.
void build_interp(const HostLevel& F, const HostLevel& C, HostLevel& out) {
  TetGrid g;
  build_grid(C, g);
  std::vector<int32_t> tet_of(F.n, -1);
  std::vector<double> lam_of(4 * (size_t)F.n, 0.0);
  auto work = [&](int f0, int f1) {
    for (int f = f0; f < f1; ++f) {
      if (F.dir[f]) continue;
      const double* x = &F.xyz[3 * (int64_t)f];
      size_t c = (size_t)g.cell(x[0], 0) +
                 (size_t)g.G * ((size_t)g.cell(x[1], 1) + (size_t)g.G * g.cell(x[2], 2));
      int best = -1;
      double lam[4];
      for (int k = g.ptr[c]; k < g.ptr[c + 1]; ++k) {
        bary(C, g.ids[k], x, lam);
        if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
          best = g.ids[k];
          break;
        }
      }
      if (best < 0) {
        double bm = -1e300;
        double l2[4];
        for (int e = 0; e < C.m; ++e) {
          bary(C, e, x, l2);
          double mn = std::min(std::min(l2[0], l2[1]), std::min(l2[2], l2[3]));
          if (mn > bm) {
            bm = mn;
            best = e;
            std::copy(l2, l2 + 4, lam);
          }
        }
      }
      tet_of[f] = best;
      std::copy(lam, lam + 4, &lam_of[4 * (size_t)f]);
    }
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)F.n * t / nth), (int)((int64_t)F.n * (t + 1) / nth));
  for (auto& t : th) t.join();
  out.P_rowptr.assign(F.n + 1, 0);
  out.P_col.clear();
  out.P_val.clear();
  for (int f = 0; f < F.n; ++f) {
    if (tet_of[f] >= 0) {
      const int32_t* t = &C.tets[4 * (int64_t)tet_of[f]];
      int idx[4] = {0, 1, 2, 3};
      std::sort(idx, idx + 4, [&](int a, int b) { return t[a] < t[b]; });
      for (int k = 0; k < 4; ++k) {
        int a = idx[k];
        if (C.dir[t[a]]) continue;
        out.P_col.push_back(t[a]);
        out.P_val.push_back(lam_of[4 * (size_t)f + a]);
      }
    }
    out.P_rowptr[f + 1] = (int32_t)out.P_col.size();
  }
  // P^T by counting sort over columns (fine rows visited in ascending order)
  out.PT_rowptr.assign(C.n + 1, 0);
  for (int32_t c : out.P_col) out.PT_rowptr[c + 1]++;
  for (int i = 0; i < C.n; ++i) out.PT_rowptr[i + 1] += out.PT_rowptr[i];
  out.PT_col.resize(out.P_col.size());
  out.PT_val.resize(out.P_col.size());
  std::vector<int32_t> fill(out.PT_rowptr.begin(), out.PT_rowptr.end() - 1);
  for (int f = 0; f < F.n; ++f)
    for (int q = out.P_rowptr[f]; q < out.P_rowptr[f + 1]; ++q) {
      int32_t d = fill[out.P_col[q]]++;
      out.PT_col[d] = f;
      out.PT_val[d] = out.P_val[q];
    }
}

// --------------------------------------------- MLS transfer (Section 3.2)
// Source nodes in uniform cubic cells over their bounding box (ids ascending
// within a cell), for radius queries.
struct NodeGrid {
  double lo[3] = {0, 0, 0}, cell = 1;
  int G[3] = {1, 1, 1};
  std::vector<int32_t> ptr, ids;
  int idx(double v, int d) const {
    double c = std::floor((v - lo[d]) / cell);
    return c < 0 ? 0 : (c >= G[d] ? G[d] - 1 : (int)c);
  }
};

void build_node_grid(const HostLevel& S, double cell, NodeGrid& g) {
  double hi[3] = {-1e300, -1e300, -1e300};
  for (int d = 0; d < 3; ++d) g.lo[d] = 1e300;
  for (int i = 0; i < S.n; ++i)
    for (int d = 0; d < 3; ++d) {
      g.lo[d] = std::min(g.lo[d], S.xyz[3 * (int64_t)i + d]);
      hi[d] = std::max(hi[d], S.xyz[3 * (int64_t)i + d]);
    }
  g.cell = cell;
  for (int d = 0; d < 3; ++d) g.G[d] = std::max(1, std::min(1024, (int)((hi[d] - g.lo[d]) / cell) + 1));
  const size_t nc = (size_t)g.G[0] * g.G[1] * g.G[2];
  std::vector<int32_t> c_of(S.n);
  g.ptr.assign(nc + 1, 0);
  for (int i = 0; i < S.n; ++i) {
    const double* x = &S.xyz[3 * (int64_t)i];
    c_of[i] = g.idx(x[0], 0) + g.G[0] * (g.idx(x[1], 1) + g.G[1] * g.idx(x[2], 2));
    g.ptr[c_of[i] + 1]++;
  }
  for (size_t c = 0; c < nc; ++c) g.ptr[c + 1] += g.ptr[c];
  g.ids.resize(S.n);
  std::vector<int32_t> fill(g.ptr.begin(), g.ptr.end() - 1);
  for (int i = 0; i < S.n; ++i) g.ids[fill[c_of[i]]++] = i;
}

// h = cbrt(6 |bounding box| / tets): the edge of the cube cells that would
// hold the mesh's tets (the Kuhn split puts 6 tets in each).
double mls_unit(const HostLevel& C) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < C.n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], C.xyz[3 * (int64_t)i + d]);
      hi[d] = std::max(hi[d], C.xyz[3 * (int64_t)i + d]);
    }
  double vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  return std::cbrt(6.0 * vol / C.m);
}

// Lumped nodal volumes |w_i| = sum over the tets at i of |T|/4 (ascending tet).
std::vector<double> nodal_volume(const HostLevel& L) {
  std::vector<double> v(L.n, 0.0);
  for (int e = 0; e < L.m; ++e) {
    const int32_t* t = &L.tets[4 * (int64_t)e];
    const double* p0 = &L.xyz[3 * (int64_t)t[0]];
    double c[3][3];
    for (int a = 1; a < 4; ++a)
      for (int k = 0; k < 3; ++k) c[a - 1][k] = L.xyz[3 * (int64_t)t[a] + k] - p0[k];
    const double q = std::fabs(det3(c[0], c[1], c[2])) / 6.0 / 4.0;
    for (int a = 0; a < 4; ++a) v[t[a]] += q;
  }
  return v;
}

// y = M^{-1} e_1 for the symmetric 4x4 moment matrix M = L D L^T; false when a
// pivot D_k is not above tol (rank < 4).
bool moment_solve(const double* M, double tol, double y[4]) {
  double Lm[4][4] = {{0}}, D[4];
  for (int k = 0; k < 4; ++k) {
    double d = M[5 * k];
    for (int j = 0; j < k; ++j) d -= Lm[k][j] * Lm[k][j] * D[j];
    if (!(d > tol)) return false;
    D[k] = d;
    for (int i = k + 1; i < 4; ++i) {
      double v = M[4 * i + k];
      for (int j = 0; j < k; ++j) v -= Lm[i][j] * Lm[k][j] * D[j];
      Lm[i][k] = v / d;
    }
  }
  double z[4] = {1.0, 0.0, 0.0, 0.0};
  for (int i = 1; i < 4; ++i)
    for (int j = 0; j < i; ++j) z[i] -= Lm[i][j] * z[j];
  for (int i = 0; i < 4; ++i) z[i] /= D[i];
  for (int i = 2; i >= 0; --i)
    for (int j = i + 1; j < 4; ++j) z[i] -= Lm[j][i] * z[j];
  std::copy(z, z + 4, y);
  return true;
}

struct MlsRow {
  std::vector<int32_t> col;
  std::vector<double> val;
};

// One MLS row at x: the admitted source nodes (stamp[n] == key, or all when
// stamp is null) within rho = c h, c = 1.5, 1.5^2, ..., until the moment matrix
// of the linear basis [1, (x_n - x)/rho] has rank 4; row_n = w_n [1, (x_n - x)/rho] . y
// with y = M^{-1} p(x), p(x) = e_1 in this basis.
bool mls_row(const HostLevel& S, const NodeGrid& g, const double* x, double h,
             const int32_t* stamp, int32_t key, std::vector<int32_t>& cand, MlsRow& out) {
  double c = 1.5;
  for (int it = 0; it < 16; ++it, c *= 1.5) {
    const double rho = c * h;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = g.idx(x[d] - rho, d);
      hi[d] = g.idx(x[d] + rho, d);
    }
    cand.clear();
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int cc = i + g.G[0] * (j + g.G[1] * k);
          for (int q = g.ptr[cc]; q < g.ptr[cc + 1]; ++q) {
            const int32_t n = g.ids[q];
            if (stamp && stamp[n] != key) continue;
            const double* y = &S.xyz[3 * (int64_t)n];
            const double d0 = y[0] - x[0], d1 = y[1] - x[1], d2 = y[2] - x[2];
            if (d0 * d0 + d1 * d1 + d2 * d2 < rho * rho) cand.push_back(n);
          }
        }
    if (cand.size() < 4) continue;
    std::sort(cand.begin(), cand.end());
    const size_t N = cand.size();
    std::vector<double> wq(5 * N);  // per neighbour: w, then the basis values
    double M[16] = {0};
    for (size_t a = 0; a < N; ++a) {
      const double* y = &S.xyz[3 * (int64_t)cand[a]];
      const double d0 = y[0] - x[0], d1 = y[1] - x[1], d2 = y[2] - x[2];
      const double s = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) / rho;
      const double w = 1.0 - 6.0 * s * s + 8.0 * s * s * s - 3.0 * s * s * s * s;  // Eq. 15
      const double q[4] = {1.0, d0 / rho, d1 / rho, d2 / rho};
      wq[5 * a] = w;
      for (int i = 0; i < 4; ++i) {
        wq[5 * a + 1 + i] = q[i];
        for (int j = 0; j < 4; ++j) M[4 * i + j] += w * q[i] * q[j];
      }
    }
    double yv[4];
    if (!moment_solve(M, 1e-9 * M[0], yv)) continue;
    out.col.assign(cand.begin(), cand.end());
    out.val.resize(N);
    for (size_t a = 0; a < N; ++a) {
      double t = 0.0;
      for (int i = 0; i < 4; ++i) t += yv[i] * (wq[5 * a] * wq[5 * a + 1 + i]);
      out.val[a] = t;
    }
    return true;
  }
  return false;
}

// The MLS operator from S to the nodes of T: rows of T's non-Dirichlet nodes,
// columns of S's non-Dirichlet nodes (ascending).  With `scale` every entry is
// multiplied by |w_t| / |w_n|.  Returns "" or an error message.
std::string build_mls(const HostLevel& S, const HostLevel& T, double h, int delta, bool scale,
                      std::vector<int32_t>& rowptr, std::vector<int32_t>& col,
                      std::vector<double>& val) {
  NodeGrid g;
  build_node_grid(S, 1.5 * h, g);
  // subdomain q of S pairs with subdomain q of T when both partitions use the
  // same id set
  std::vector<int32_t> ids_s, ids_t;
  bool part = !S.owner.empty() && !T.owner.empty();
  if (part) {
    ids_s = S.owner;
    ids_t = T.owner;
    for (auto* v : {&ids_s, &ids_t}) {
      std::sort(v->begin(), v->end());
      v->erase(std::unique(v->begin(), v->end()), v->end());
    }
    part = (ids_s == ids_t);
  }
  // work groups: target nodes by owner id (one group when unpaired)
  std::vector<int32_t> gptr, gnodes;
  std::vector<int32_t> gid;  // owner id of each group
  if (part) {
    gid = ids_t;
    gptr.assign(gid.size() + 1, 0);
    std::vector<int32_t> gi(T.n);
    for (int t = 0; t < T.n; ++t) {
      gi[t] = (int32_t)(std::lower_bound(gid.begin(), gid.end(), T.owner[t]) - gid.begin());
      gptr[gi[t] + 1]++;
    }
    for (size_t k = 0; k < gid.size(); ++k) gptr[k + 1] += gptr[k];
    gnodes.resize(T.n);
    std::vector<int32_t> fill(gptr.begin(), gptr.end() - 1);
    for (int t = 0; t < T.n; ++t) gnodes[fill[gi[t]]++] = t;
  } else {
    const int nchunk = 64;
    gptr.resize(nchunk + 1);
    for (int k = 0; k <= nchunk; ++k) gptr[k] = (int32_t)((int64_t)T.n * k / nchunk);
    gnodes.resize(T.n);
    std::iota(gnodes.begin(), gnodes.end(), 0);
  }
  // source vertices by owner id, for the overlap growth
  std::vector<int32_t> sptr, snodes;
  if (part) {
    sptr.assign(ids_s.size() + 1, 0);
    std::vector<int32_t> si(S.n);
    for (int n = 0; n < S.n; ++n) {
      si[n] = (int32_t)(std::lower_bound(ids_s.begin(), ids_s.end(), S.owner[n]) - ids_s.begin());
      sptr[si[n] + 1]++;
    }
    for (size_t k = 0; k < ids_s.size(); ++k) sptr[k + 1] += sptr[k];
    snodes.resize(S.n);
    std::vector<int32_t> fill(sptr.begin(), sptr.end() - 1);
    for (int n = 0; n < S.n; ++n) snodes[fill[si[n]]++] = n;
  }
  std::vector<MlsRow> rows(T.n);
  const int ngroups = (int)gptr.size() - 1;
  std::vector<int> failed(ngroups, -1);
  auto work = [&](int g0, int g1) {
    std::vector<int32_t> stamp(part ? S.n : 0, -1), frontier, next, cand;
    for (int k = g0; k < g1; ++k) {
      if (part) {  // Omega^delta_q: owned vertices, then delta layers over the mesh graph
        frontier.assign(snodes.begin() + sptr[k], snodes.begin() + sptr[k + 1]);
        for (int32_t v : frontier) stamp[v] = k;
        for (int layer = 0; layer < delta; ++layer) {
          next.clear();
          for (int32_t v : frontier)
            for (int q = S.rowptr[v]; q < S.rowptr[v + 1]; ++q)
              if (stamp[S.col[q]] != k) {
                stamp[S.col[q]] = k;
                next.push_back(S.col[q]);
              }
          frontier.swap(next);
        }
      }
      for (int q = gptr[k]; q < gptr[k + 1]; ++q) {
        const int t = gnodes[q];
        if (T.dir[t]) continue;
        if (!mls_row(S, g, &T.xyz[3 * (int64_t)t], h, part ? stamp.data() : nullptr, k, cand, rows[t])) {
          failed[k] = t;
          break;
        }
      }
    }
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  nth = std::min(nth, ngroups);
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)ngroups * t / nth), (int)((int64_t)ngroups * (t + 1) / nth));
  for (auto& t : th) t.join();
  for (int k = 0; k < ngroups; ++k)
    if (failed[k] >= 0)
      return "MLS neighbourhood of node " + std::to_string(failed[k]) + " never reached rank 4";
  std::vector<double> vs, vt;
  if (scale) {
    vs = nodal_volume(S);
    vt = nodal_volume(T);
  }
  rowptr.assign(T.n + 1, 0);
  col.clear();
  val.clear();
  for (int t = 0; t < T.n; ++t) {
    const MlsRow& r = rows[t];
    for (size_t a = 0; a < r.col.size(); ++a) {
      const int32_t n = r.col[a];
      if (S.dir[n]) continue;  // the transferred vectors vanish there
      col.push_back(n);
      val.push_back(scale ? vt[t] * r.val[a] / vs[n] : r.val[a]);
    }
    rowptr[t + 1] = (int32_t)col.size();
  }
  return "";
}

// ------------------------------------------------- ILU(p) symbolic (set-up)
// For each subdomain block A_p (local numbering = position in the sorted DoF
// list): the strict lower part of the level-of-fill pattern of ILU(p) (A_p and
// its pattern are symmetric, so the upper part is the transpose), computed row
// by row: the candidate columns of row i come out of a min-heap in ascending
// order; eliminating with an earlier row k (level lev_ik <= p) proposes every
// column j of row k's upper part (the transposed lower lists of the finished
// rows j < i) at level lev_ik + lev_kj + 1, kept if <= p.  Then the
// dependency levels of both triangular sweeps and the extraction map.
struct IluSub {
  std::vector<int32_t> lptr, lcol;             // local strict lower pattern
  std::vector<int32_t> fwd_rows, fwd_lvl, bwd_rows, bwd_lvl;
};

void ilu_block(const HostLevel& L, int p, int fill, IluSub& out) {
  const int32_t* dofs = &L.sub_dofs[L.sub_ptr[p]];
  const int n = L.sub_ptr[p + 1] - L.sub_ptr[p];
  auto local = [&](int g) {
    const int32_t* it = std::lower_bound(dofs, dofs + n, g);
    return (it != dofs + n && *it == g) ? (int)(it - dofs) : -1;
  };
  std::vector<std::vector<std::pair<int32_t, int32_t>>> up(n);  // (j, level) of row k's upper part
  std::vector<int32_t> lev(n, INT32_MAX);
  std::vector<int32_t> heap;
  out.lptr.assign(n + 1, 0);
  out.lcol.clear();
  std::vector<int32_t> row, rowlev;
  for (int i = 0; i < n; ++i) {
    heap.clear();
    const int g = dofs[i];
    for (int q = L.rowptr[g]; q < L.rowptr[g + 1]; ++q) {
      const int k = local(L.col[q]);
      if (k >= 0 && k < i && lev[k] == INT32_MAX) {
        lev[k] = 0;
        heap.push_back(k);
      }
    }
    std::make_heap(heap.begin(), heap.end(), std::greater<int32_t>());
    row.clear();
    rowlev.clear();
    while (!heap.empty()) {
      std::pop_heap(heap.begin(), heap.end(), std::greater<int32_t>());
      const int k = heap.back();
      heap.pop_back();
      row.push_back(k);
      rowlev.push_back(lev[k]);
      for (const auto& e : up[k]) {
        const int j = e.first;
        if (j >= i) break;  // lists are sorted by j
        const int nl = lev[k] + e.second + 1;
        if (nl > fill || nl >= lev[j]) continue;
        if (lev[j] == INT32_MAX) {
          heap.push_back(j);
          std::push_heap(heap.begin(), heap.end(), std::greater<int32_t>());
        }
        lev[j] = nl;
      }
    }
    for (size_t t = 0; t < row.size(); ++t) {
      out.lcol.push_back(row[t]);
      up[row[t]].push_back({i, rowlev[t]});
      lev[row[t]] = INT32_MAX;
    }
    out.lptr[i + 1] = (int32_t)out.lcol.size();
  }
  // dependency levels: forward (row i after the rows of its pattern),
  // backward (row i after every row j > i whose pattern holds i)
  std::vector<int32_t> lf(n, 0), lb(n, 0);
  int nf = 0, nb = 0;
  for (int i = 0; i < n; ++i) {
    for (int t = out.lptr[i]; t < out.lptr[i + 1]; ++t) lf[i] = std::max(lf[i], lf[out.lcol[t]] + 1);
    nf = std::max(nf, lf[i] + 1);
  }
  for (int i = n - 1; i >= 0; --i) {
    for (const auto& e : up[i]) lb[i] = std::max(lb[i], lb[e.first] + 1);
    nb = std::max(nb, lb[i] + 1);
  }
  auto group = [&](const std::vector<int32_t>& lv, int nl, std::vector<int32_t>& rows,
                   std::vector<int32_t>& ptr) {
    ptr.assign(nl + 1, 0);
    for (int i = 0; i < n; ++i) ptr[lv[i] + 1]++;
    for (int q = 0; q < nl; ++q) ptr[q + 1] += ptr[q];
    rows.resize(n);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n; ++i) rows[fill[lv[i]]++] = i;
  };
  group(lf, nf, out.fwd_rows, out.fwd_lvl);
  group(lb, nb, out.bwd_rows, out.bwd_lvl);
}

void build_ilu(HostLevel& L, int fill) {
  L.ilu_fill = fill;
  std::vector<IluSub> subs(L.nsub);
  auto work = [&](int p0, int p1) {
    for (int p = p0; p < p1; ++p) ilu_block(L, p, fill, subs[p]);
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  nth = std::min(nth, std::max(1, L.nsub));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)L.nsub * t / nth), (int)((int64_t)L.nsub * (t + 1) / nth));
  for (auto& t : th) t.join();
  const int64_t rows = L.sub_ptr[L.nsub];
  L.ilu_lptr.assign(rows + 1, 0);
  L.ilu_lcol.clear();
  L.ilu_max_n = 0;
  for (int p = 0; p < L.nsub; ++p) {
    const int n = L.sub_ptr[p + 1] - L.sub_ptr[p];
    L.ilu_max_n = std::max(L.ilu_max_n, n);
    const int64_t base = L.ilu_lptr[L.sub_ptr[p]];
    for (int i = 0; i < n; ++i) L.ilu_lptr[L.sub_ptr[p] + i + 1] = base + subs[p].lptr[i + 1];
    L.ilu_lcol.insert(L.ilu_lcol.end(), subs[p].lcol.begin(), subs[p].lcol.end());
  }
  L.ilu_nnz = L.ilu_lptr[rows];
  L.ilu_max_row = 0;
  for (int64_t R = 0; R < rows; ++R)
    L.ilu_max_row = std::max(L.ilu_max_row, (int)(L.ilu_lptr[R + 1] - L.ilu_lptr[R]));
  // transposed pattern
  L.ilu_tptr.assign(rows + 1, 0);
  for (int p = 0; p < L.nsub; ++p)
    for (int64_t R = L.sub_ptr[p]; R < L.sub_ptr[p + 1]; ++R)
      for (int64_t t = L.ilu_lptr[R]; t < L.ilu_lptr[R + 1]; ++t) L.ilu_tptr[L.sub_ptr[p] + L.ilu_lcol[t] + 1]++;
  for (int64_t R = 0; R < rows; ++R) L.ilu_tptr[R + 1] += L.ilu_tptr[R];
  L.ilu_tcol.assign(L.ilu_nnz, 0);
  L.ilu_tslot.assign(L.ilu_nnz, 0);
  {
    std::vector<int64_t> fill_at(L.ilu_tptr.begin(), L.ilu_tptr.end() - 1);
    for (int p = 0; p < L.nsub; ++p)
      for (int64_t R = L.sub_ptr[p]; R < L.sub_ptr[p + 1]; ++R)  // rows ascending: columns of T sorted
        for (int64_t t = L.ilu_lptr[R]; t < L.ilu_lptr[R + 1]; ++t) {
          const int64_t d = fill_at[L.sub_ptr[p] + L.ilu_lcol[t]]++;
          L.ilu_tcol[d] = (int32_t)(R - L.sub_ptr[p]);
          L.ilu_tslot[d] = t;
        }
  }
  // level schedules
  L.ilu_fwd_rows.clear();
  L.ilu_bwd_rows.clear();
  L.ilu_fwd_lvl.clear();
  L.ilu_bwd_lvl.clear();
  L.ilu_fwd_loff.assign(L.nsub + 1, 0);
  L.ilu_bwd_loff.assign(L.nsub + 1, 0);
  for (int p = 0; p < L.nsub; ++p) {
    const int32_t base = L.sub_ptr[p];
    for (int32_t r : subs[p].fwd_rows) L.ilu_fwd_rows.push_back(r);
    for (int32_t r : subs[p].bwd_rows) L.ilu_bwd_rows.push_back(r);
    for (int32_t v : subs[p].fwd_lvl) L.ilu_fwd_lvl.push_back(base + v);
    for (int32_t v : subs[p].bwd_lvl) L.ilu_bwd_lvl.push_back(base + v);
    L.ilu_fwd_loff[p + 1] = (int32_t)L.ilu_fwd_lvl.size();
    L.ilu_bwd_loff[p + 1] = (int32_t)L.ilu_bwd_lvl.size();
  }
  // level-major entry lists of both sweeps
  {
    const int64_t nrows = rows;
    L.ilu_fe_ptr.assign(nrows + 1, 0);
    L.ilu_be_ptr.assign(nrows + 1, 0);
    L.ilu_fe_src.clear();
    L.ilu_fe_slot.clear();
    L.ilu_be_src.clear();
    L.ilu_be_slot.clear();
    for (int p = 0; p < L.nsub; ++p) {
      const int64_t R0 = L.sub_ptr[p];
      for (int64_t rr = R0; rr < L.sub_ptr[p + 1]; ++rr) {
        const int64_t Rf = R0 + L.ilu_fwd_rows[rr];
        for (int64_t t = L.ilu_lptr[Rf]; t < L.ilu_lptr[Rf + 1]; ++t) {
          L.ilu_fe_src.push_back(L.ilu_lcol[t]);
          L.ilu_fe_slot.push_back(t);
        }
        L.ilu_fe_ptr[rr + 1] = (int64_t)L.ilu_fe_src.size();
        const int64_t Rb = R0 + L.ilu_bwd_rows[rr];
        for (int64_t u = L.ilu_tptr[Rb]; u < L.ilu_tptr[Rb + 1]; ++u) {
          L.ilu_be_src.push_back(L.ilu_tcol[u]);
          L.ilu_be_slot.push_back(L.ilu_tslot[u]);
        }
        L.ilu_be_ptr[rr + 1] = (int64_t)L.ilu_be_src.size();
      }
    }
  }
  // extraction of the lower triangle of every block (diagonal into D)
  L.ilu_ext_pos.clear();
  L.ilu_ext_nz.clear();
  for (int p = 0; p < L.nsub; ++p) {
    const int32_t* dofs = &L.sub_dofs[L.sub_ptr[p]];
    const int n = L.sub_ptr[p + 1] - L.sub_ptr[p];
    for (int i = 0; i < n; ++i) {
      const int64_t R = L.sub_ptr[p] + i;
      const int g = dofs[i];
      for (int q = L.rowptr[g]; q < L.rowptr[g + 1]; ++q) {
        const int32_t* it = std::lower_bound(dofs, dofs + n, L.col[q]);
        if (it == dofs + n || *it != L.col[q]) continue;
        const int k = (int)(it - dofs);
        if (k > i) continue;
        int64_t pos;
        if (k == i) {
          pos = L.ilu_nnz + R;
        } else {
          const int32_t* b = &L.ilu_lcol[L.ilu_lptr[R]];
          const int32_t* e = &L.ilu_lcol[L.ilu_lptr[R + 1]];
          pos = L.ilu_lptr[R] + (std::lower_bound(b, e, k) - b);  // A_p entries are in the pattern
        }
        L.ilu_ext_pos.push_back(pos);
        L.ilu_ext_nz.push_back(q);
      }
    }
  }
}

// Three fields per vertex (linear elasticity): the vertex-level pattern,
// contributions, subdomains and transfers become DoF-level ones, DoF 3v + c
// for field c of vertex v.  A vertex nonzero (v, w) becomes a 3 x 3 block;
// its contribution e*10 + pair(a, b) becomes e*78 + slot(3a'+i, 3b'+j) with
// a', b' the local indices of v and w in tet e.  Subdomains take all fields
// of their vertices; the transfers become P (x) I_3 (the field-splitting
// interpolation with the scalar P for every field).
void expand_csr(int nrows, const std::vector<int32_t>& rp, const std::vector<int32_t>& cl,
                const std::vector<double>& vl, std::vector<int32_t>& orp, std::vector<int32_t>& ocl,
                std::vector<double>& ovl) {
  orp.assign(3 * (size_t)nrows + 1, 0);
  ocl.clear();
  ovl.clear();
  for (int i = 0; i < nrows; ++i)
    for (int c = 0; c < 3; ++c) {
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        ocl.push_back(3 * cl[q] + c);
        ovl.push_back(vl[q]);
      }
      orp[3 * i + c + 1] = (int32_t)ocl.size();
    }
}

void expand_fields(HostLevel& L) {
  const int nv = L.nv, n = 3 * nv;
  const std::vector<int32_t> vrp = L.rowptr, vcol = L.col, vcptr = L.cptr, vcon = L.contrib;
  const std::vector<uint8_t> vdir = L.dir;
  std::vector<int32_t> rp(n + 1, 0), col;
  col.reserve(9 * vcol.size());
  for (int v = 0; v < nv; ++v)
    for (int c = 0; c < 3; ++c) {
      for (int q = vrp[v]; q < vrp[v + 1]; ++q)
        for (int c2 = 0; c2 < 3; ++c2) col.push_back(3 * vcol[q] + c2);
      rp[3 * v + c + 1] = (int32_t)col.size();
    }
  L.rowptr.swap(rp);
  L.col.swap(col);
  L.n = n;
  L.fields = 3;
  L.dir.assign(n, 0);
  for (int i = 0; i < n; ++i) L.dir[i] = vdir[i / 3];
  L.dir_list.clear();
  for (int i = 0; i < n; ++i)
    if (L.dir[i]) L.dir_list.push_back(i);
  if (!L.owner.empty()) {
    std::vector<int32_t> ow(n);
    for (int i = 0; i < n; ++i) ow[i] = L.owner[i / 3];
    L.owner.swap(ow);
  }
  L.diag.assign(n, -1);
  for (int i = 0; i < n; ++i) L.diag[i] = find_in_row(L, i, i);
  const int64_t nnz = L.col.size();
  L.nzflag.assign(nnz, 0);
  for (int i = 0; i < n; ++i)
    for (int q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
      const int j = L.col[q];
      if (L.dir[i]) L.nzflag[q] = (i == j) ? 1 : 2;
      else if (L.dir[j]) L.nzflag[q] = 2;
    }
  // DoF nonzero (3v+i, 3w+j) sits at position 3*(vertex pos of (v,w)) + j of
  // row 3v+i: the contributions of the vertex nonzero, re-slotted
  L.cptr.assign(nnz + 1, 0);
  for (int v = 0; v < nv; ++v)
    for (int i = 0; i < 3; ++i)
      for (int qv = vrp[v]; qv < vrp[v + 1]; ++qv)
        for (int j = 0; j < 3; ++j) {
          const int64_t q = L.rowptr[3 * v + i] + 3 * (int64_t)(qv - vrp[v]) + j;
          L.cptr[q + 1] = L.nzflag[q] == 0 ? vcptr[qv + 1] - vcptr[qv] : 0;
        }
  for (int64_t q = 0; q < nnz; ++q) L.cptr[q + 1] += L.cptr[q];
  L.contrib.assign(L.cptr[nnz], 0);
  for (int v = 0; v < nv; ++v)
    for (int i = 0; i < 3; ++i)
      for (int qv = vrp[v]; qv < vrp[v + 1]; ++qv) {
        const int w = vcol[qv];
        for (int j = 0; j < 3; ++j) {
          const int64_t q = L.rowptr[3 * v + i] + 3 * (int64_t)(qv - vrp[v]) + j;
          if (L.nzflag[q] != 0) continue;
          int32_t k = L.cptr[q];
          for (int c = vcptr[qv]; c < vcptr[qv + 1]; ++c) {
            const int e = vcon[c] / 10;
            const int32_t* t = &L.tets[4 * (int64_t)e];
            int a = 0, b = 0;
            while (t[a] != v) ++a;
            while (t[b] != w) ++b;
            L.contrib[k++] = e * kElasticSlots + elastic_slot(3 * a + i, 3 * b + j);
          }
        }
      }
  // subdomains: all fields of each vertex
  std::vector<int32_t> sp(L.nsub + 1, 0), sd;
  std::vector<uint8_t> so;
  for (int p = 0; p < L.nsub; ++p) {
    for (int k = L.sub_ptr[p]; k < L.sub_ptr[p + 1]; ++k)
      for (int c = 0; c < 3; ++c) {
        sd.push_back(3 * L.sub_dofs[k] + c);
        so.push_back(L.sub_own[k]);
      }
    sp[p + 1] = (int32_t)sd.size();
  }
  L.sub_ptr.swap(sp);
  L.sub_dofs.swap(sd);
  L.sub_own.swap(so);
}

// ------------------------------------------------ quadratic (P2) elements
// One DoF per vertex and one per edge (the DoF distribution N = (1,1,0,0) of
// the mesh perspective, Section 2.1).  The edges are the distinct vertex
// pairs of the tets.  Numbering: each vertex is followed by its edges to
// higher-numbered vertices, ascending, so that the DoF of vertex v is
// v + (edges of the vertices before v) and a block's DoFs stay banded.  A
// vertex DoF is Dirichlet as its vertex; an edge DoF when the edge lies on a
// boundary face (a face of exactly one tet) with three Dirichlet vertices.
// The pattern couples the DoFs of each tet; contribution e*55 + slot(li, lj)
// of tet e (ascending e) feeds the nonzero of its local DoFs li, lj.
// With `twofield` (the coupled P2-P1 system) every vertex also carries the
// DoF of the P1 field p, right after its u DoF (vertex 0's u, its p, its
// edges, vertex 1's u, ...); local DoFs 10..13 of a tet are its vertices' p
// DoFs, Dirichlet and owned as their vertex; contributions address the
// 105-slot element matrix.
std::string build_p2_level(HostLevel& L, const int32_t* vowner, int delta, bool smoothed, bool twofield) {
  const int nv = L.nv;
  const int nb = twofield ? 2 : 1;        // vertex DoFs per vertex
  const int NL = twofield ? 14 : 10;      // local DoFs per tet
  const int NS = twofield ? kP2P1Slots : kP2Slots;
  std::vector<int32_t> vptr, vadj;
  vertex_tets(L, vptr, vadj);
  // upper neighbours of every vertex through the edges of its tets
  std::vector<int32_t> uptr(nv + 1, 0), ucol;
  {
    std::vector<std::vector<int32_t>> up(nv);
    for (int e = 0; e < L.m; ++e)
      for (int k = 0; k < 6; ++k) {
        int a = L.tets[4 * (int64_t)e + kP2EdgeEnd[k][0]], b = L.tets[4 * (int64_t)e + kP2EdgeEnd[k][1]];
        if (a > b) std::swap(a, b);
        up[a].push_back(b);
      }
    for (int v = 0; v < nv; ++v) {
      std::sort(up[v].begin(), up[v].end());
      up[v].erase(std::unique(up[v].begin(), up[v].end()), up[v].end());
      uptr[v + 1] = uptr[v] + (int32_t)up[v].size();
    }
    ucol.reserve(uptr[nv]);
    for (int v = 0; v < nv; ++v) ucol.insert(ucol.end(), up[v].begin(), up[v].end());
  }
  const int64_t ne = uptr[nv];
  if (nv + ne > INT32_MAX / 2) return "too many P2 DoFs";
  auto vdof = [&](int v) { return nb * v + uptr[v]; };
  auto edof_at = [&](int v, int32_t k) { return (int32_t)(nb * v + nb + k); };  // CSR position k of v's edges
  auto edof = [&](int a, int b) {  // a != b
    if (a > b) std::swap(a, b);
    const int32_t* lo = ucol.data() + uptr[a];
    const int32_t* hi = ucol.data() + uptr[a + 1];
    const int32_t* it = std::lower_bound(lo, hi, b);
    return edof_at(a, (int32_t)(it - ucol.data()));
  };
  const int n = (int)(nb * (int64_t)nv + ne);
  std::vector<uint8_t> vdir = L.dir;
  L.p2 = true;
  L.nloc = NL;
  L.nslot = NS;
  L.n = n;
  L.tdof.assign(NL * (size_t)L.m, 0);
  for (int e = 0; e < L.m; ++e) {
    const int32_t* t = &L.tets[4 * (int64_t)e];
    for (int a = 0; a < 4; ++a) L.tdof[NL * (size_t)e + a] = vdof(t[a]);
    for (int k = 0; k < 6; ++k) L.tdof[NL * (size_t)e + 4 + k] = edof(t[kP2EdgeEnd[k][0]], t[kP2EdgeEnd[k][1]]);
    if (twofield)
      for (int a = 0; a < 4; ++a) L.tdof[NL * (size_t)e + 10 + a] = vdof(t[a]) + 1;
  }
  L.dofx.assign(3 * (size_t)n, 0.0);
  L.dir.assign(n, 0);
  L.pdof.assign(twofield ? n : 0, 0);
  for (int v = 0; v < nv; ++v) {
    for (int f = 0; f < nb; ++f) {
      for (int d = 0; d < 3; ++d) L.dofx[3 * (size_t)(vdof(v) + f) + d] = L.xyz[3 * (size_t)v + d];
      L.dir[vdof(v) + f] = vdir[v];
    }
    if (twofield) L.pdof[vdof(v) + 1] = 1;
    for (int32_t k = uptr[v]; k < uptr[v + 1]; ++k)
      for (int d = 0; d < 3; ++d)
        L.dofx[3 * (size_t)edof_at(v, k) + d] = 0.5 * (L.xyz[3 * (size_t)v + d] + L.xyz[3 * (size_t)ucol[k] + d]);
  }
  // boundary faces: faces that no other tet shares
  for (int e = 0; e < L.m; ++e) {
    const int32_t* t = &L.tets[4 * (int64_t)e];
    for (int skip = 0; skip < 4; ++skip) {
      int f[3], c = 0;
      for (int a = 0; a < 4; ++a)
        if (a != skip) f[c++] = t[a];
      if (!(vdir[f[0]] && vdir[f[1]] && vdir[f[2]])) continue;
      int shared = 0;
      for (int k = vptr[f[0]]; k < vptr[f[0] + 1] && !shared; ++k) {
        const int e2 = vadj[k];
        if (e2 == e) continue;
        const int32_t* t2 = &L.tets[4 * (int64_t)e2];
        int hit = 0;
        for (int a = 0; a < 4; ++a) hit += (t2[a] == f[1]) + (t2[a] == f[2]);
        shared = hit == 2;
      }
      if (shared) continue;
      L.dir[edof(f[0], f[1])] = 1;
      L.dir[edof(f[0], f[2])] = 1;
      L.dir[edof(f[1], f[2])] = 1;
    }
  }
  L.dir_list.clear();
  for (int i = 0; i < n; ++i)
    if (L.dir[i]) L.dir_list.push_back(i);
  // pattern: the DoFs of the tets holding each DoF (found among the tets of
  // the DoF's vertex, or of its edge's lower vertex)
  std::vector<int32_t> ent_a(n), ent_b(n, -1);  // DoF -> its vertex (a) or edge (a, b)
  for (int v = 0; v < nv; ++v) {
    for (int f = 0; f < nb; ++f) ent_a[vdof(v) + f] = v;
    for (int32_t k = uptr[v]; k < uptr[v + 1]; ++k) {
      ent_a[edof_at(v, k)] = v;
      ent_b[edof_at(v, k)] = ucol[k];
    }
  }
  auto holds = [&](int e, int i) {  // local index of DoF i in tet e, or -1
    for (int li = 0; li < NL; ++li)
      if (L.tdof[NL * (size_t)e + li] == i) return li;
    return -1;
  };
  L.rowptr.assign(n + 1, 0);
  std::vector<std::vector<int32_t>> rows(n);
  std::vector<int32_t> buf;
  for (int i = 0; i < n; ++i) {
    buf.clear();
    const int a = ent_a[i];
    for (int k = vptr[a]; k < vptr[a + 1]; ++k) {
      const int e = vadj[k];
      if (holds(e, i) < 0) continue;
      buf.insert(buf.end(), &L.tdof[NL * (size_t)e], &L.tdof[NL * (size_t)e] + NL);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    rows[i] = buf;
    L.rowptr[i + 1] = L.rowptr[i] + (int32_t)buf.size();
  }
  L.col.resize(L.rowptr[n]);
  L.diag.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    std::copy(rows[i].begin(), rows[i].end(), L.col.begin() + L.rowptr[i]);
    L.diag[i] = find_in_row(L, i, i);
  }
  rows.clear();
  rows.shrink_to_fit();
  const int64_t nnz = L.col.size();
  L.nzflag.assign(nnz, 0);
  for (int i = 0; i < n; ++i)
    for (int q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
      const int j = L.col[q];
      if (L.dir[i]) L.nzflag[q] = (i == j) ? 1 : 2;
      else if (L.dir[j]) L.nzflag[q] = 2;
    }
  std::vector<int32_t> cnt(nnz + 1, 0);
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int32_t> fill;
    if (pass == 1) {
      L.cptr.assign(nnz + 1, 0);
      for (int64_t q = 0; q < nnz; ++q) L.cptr[q + 1] = L.cptr[q] + cnt[q];
      L.contrib.assign(L.cptr[nnz], 0);
      fill.assign(L.cptr.begin(), L.cptr.end() - 1);
    }
    for (int i = 0; i < n; ++i) {
      if (L.dir[i]) continue;
      const int a = ent_a[i];
      for (int k = vptr[a]; k < vptr[a + 1]; ++k) {  // ascending tet id
        const int e = vadj[k];
        const int li = holds(e, i);
        if (li < 0) continue;
        for (int lj = 0; lj < NL; ++lj) {
          const int32_t q = find_in_row(L, i, L.tdof[NL * (size_t)e + lj]);
          if (L.nzflag[q] != 0) continue;
          if (pass == 0) cnt[q]++;
          else L.contrib[fill[q]++] = e * NS + sym_slot(NL, li, lj);
        }
      }
    }
  }
  if (!smoothed) return "";
  // owners: a vertex's own; an edge's lower vertex's, if that id owns a
  // non-Dirichlet vertex, else its upper vertex's
  std::vector<char> is_id;
  {
    int32_t mx = 0;
    for (int v = 0; v < nv; ++v) mx = std::max(mx, vowner[v]);
    is_id.assign((size_t)mx + 1, 0);
    for (int v = 0; v < nv; ++v)
      if (!vdir[v] && vowner[v] >= 0) is_id[vowner[v]] = 1;
  }
  L.owner.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    if (ent_b[i] < 0) {
      L.owner[i] = vowner[ent_a[i]];
    } else {
      const int32_t oa = vowner[ent_a[i]], ob = vowner[ent_b[i]];
      L.owner[i] = (oa >= 0 && is_id[oa]) ? oa : ((ob >= 0 && is_id[ob]) ? ob : -1);
      if (L.owner[i] < 0 && !L.dir[i]) return "an edge DoF has no owning subdomain";
    }
  }
  if (delta < 1) return "P2 subdomains need delta >= 1";
  // subdomains: vertex layers over the tets from the vertices of each id,
  // then the vertex DoFs and the DoFs of edges with both ends inside
  std::vector<int32_t> ids;
  for (int v = 0; v < nv; ++v)
    if (!vdir[v]) ids.push_back(vowner[v]);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  L.nsub = (int)ids.size();
  std::vector<std::vector<int32_t>> by_id(L.nsub);
  for (int v = 0; v < nv; ++v) {
    auto it = std::lower_bound(ids.begin(), ids.end(), vowner[v]);
    if (it != ids.end() && *it == vowner[v]) by_id[it - ids.begin()].push_back(v);
  }
  std::vector<std::vector<int32_t>> dofs(L.nsub);
  std::vector<std::vector<uint8_t>> own(L.nsub);
  auto work = [&](int p0, int p1) {
    std::vector<int32_t> stamp(nv, -1), frontier, next, members;
    for (int p = p0; p < p1; ++p) {
      members = by_id[p];
      frontier = members;
      for (int v : members) stamp[v] = p;
      for (int layer = 0; layer < delta; ++layer) {
        next.clear();
        for (int v : frontier)
          for (int k = vptr[v]; k < vptr[v + 1]; ++k)
            for (int a = 0; a < 4; ++a) {
              const int w = L.tets[4 * (int64_t)vadj[k] + a];
              if (stamp[w] != p) {
                stamp[w] = p;
                members.push_back(w);
                next.push_back(w);
              }
            }
        frontier.swap(next);
      }
      std::vector<int32_t> d;
      for (int v : members) {
        for (int f = 0; f < nb; ++f)
          if (!L.dir[vdof(v) + f]) d.push_back(vdof(v) + f);
        for (int32_t k = uptr[v]; k < uptr[v + 1]; ++k)
          if (stamp[ucol[k]] == p && !L.dir[edof_at(v, k)]) d.push_back(edof_at(v, k));
      }
      std::sort(d.begin(), d.end());
      std::vector<uint8_t> o(d.size());
      for (size_t k = 0; k < d.size(); ++k) o[k] = (L.owner[d[k]] == ids[p]) ? 1 : 0;
      dofs[p] = std::move(d);
      own[p] = std::move(o);
    }
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  nth = std::min(nth, std::max(1, L.nsub));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)L.nsub * t / nth), (int)((int64_t)L.nsub * (t + 1) / nth));
  for (auto& t : th) t.join();
  L.sub_ptr.assign(L.nsub + 1, 0);
  for (int p = 0; p < L.nsub; ++p) L.sub_ptr[p + 1] = L.sub_ptr[p] + (int32_t)dofs[p].size();
  L.sub_dofs.resize(L.sub_ptr[L.nsub]);
  L.sub_own.resize(L.sub_ptr[L.nsub]);
  for (int p = 0; p < L.nsub; ++p) {
    std::copy(dofs[p].begin(), dofs[p].end(), L.sub_dofs.begin() + L.sub_ptr[p]);
    std::copy(own[p].begin(), own[p].end(), L.sub_own.begin() + L.sub_ptr[p]);
  }
  // every non-Dirichlet DoF owned exactly once
  std::vector<int> owned(n, 0);
  for (size_t k = 0; k < L.sub_dofs.size(); ++k) owned[L.sub_dofs[k]] += L.sub_own[k];
  for (int i = 0; i < n; ++i)
    if (!L.dir[i] && owned[i] != 1) return "internal: a P2 DoF is not owned exactly once";
  return "";
}

// P2 interpolation from C (coarse) to the DoFs of F: every non-Dirichlet
// fine DoF point is located in the coarse mesh by the rule of build_interp
// (the lowest containing tet id, else the tet whose smallest barycentric
// weight is largest) and its row holds the coarse tet's ten P2 basis
// functions there -- vertex a: l_a (2 l_a - 1), edge ab: 4 l_a l_b -- on the
// non-Dirichlet coarse DoFs, columns ascending, zero weights kept.  With the
// P2-P1 system the transfer is split by field (Section 2.1): rows of the P1
// field p hold the barycentric weights on the coarse p DoFs.
void build_interp_p2(const HostLevel& F, const HostLevel& C, HostLevel& out) {
  TetGrid g;
  build_grid(C, g);
  const int n = F.n;
  std::vector<int32_t> tet_of(n, -1);
  std::vector<double> lam_of(4 * (size_t)n, 0.0);
  auto work = [&](int f0, int f1) {
    for (int f = f0; f < f1; ++f) {
      if (F.dir[f]) continue;
      const double* x = &F.dofx[3 * (size_t)f];
      size_t c = (size_t)g.cell(x[0], 0) + (size_t)g.G * ((size_t)g.cell(x[1], 1) + (size_t)g.G * g.cell(x[2], 2));
      int best = -1;
      double lam[4];
      for (int k = g.ptr[c]; k < g.ptr[c + 1]; ++k) {
        bary(C, g.ids[k], x, lam);
        if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
          best = g.ids[k];
          break;
        }
      }
      if (best < 0) {
        double bm = -1e300, l2[4];
        for (int e = 0; e < C.m; ++e) {
          bary(C, e, x, l2);
          const double mn = std::min(std::min(l2[0], l2[1]), std::min(l2[2], l2[3]));
          if (mn > bm) {
            bm = mn;
            best = e;
            std::copy(l2, l2 + 4, lam);
          }
        }
      }
      tet_of[f] = best;
      std::copy(lam, lam + 4, &lam_of[4 * (size_t)f]);
    }
  };
  int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back(work, (int)((int64_t)n * t / nth), (int)((int64_t)n * (t + 1) / nth));
  for (auto& t : th) t.join();
  out.P_rowptr.assign(n + 1, 0);
  out.P_col.clear();
  out.P_val.clear();
  std::vector<std::pair<int32_t, double>> row;
  for (int f = 0; f < n; ++f) {
    if (tet_of[f] >= 0) {
      const double* l = &lam_of[4 * (size_t)f];
      const int32_t* td = &C.tdof[C.nloc * (size_t)tet_of[f]];
      row.clear();
      if (!F.pdof.empty() && F.pdof[f]) {  // the P1 field: its barycentric weights on the coarse p DoFs
        for (int a = 0; a < 4; ++a)
          if (!C.dir[td[10 + a]]) row.push_back({td[10 + a], l[a]});
      } else {
        for (int i = 0; i < 10; ++i) {
          if (C.dir[td[i]]) continue;
          const double w = i < 4 ? l[i] * (2.0 * l[i] - 1.0)
                                 : 4.0 * l[kP2EdgeEnd[i - 4][0]] * l[kP2EdgeEnd[i - 4][1]];
          row.push_back({td[i], w});
        }
      }
      std::sort(row.begin(), row.end());
      for (auto& pr : row) {
        out.P_col.push_back(pr.first);
        out.P_val.push_back(pr.second);
      }
    }
    out.P_rowptr[f + 1] = (int32_t)out.P_col.size();
  }
  out.PT_rowptr.assign(C.n + 1, 0);
  for (int32_t c : out.P_col) out.PT_rowptr[c + 1]++;
  for (int i = 0; i < C.n; ++i) out.PT_rowptr[i + 1] += out.PT_rowptr[i];
  out.PT_col.resize(out.P_col.size());
  out.PT_val.resize(out.P_col.size());
  std::vector<int32_t> fill(out.PT_rowptr.begin(), out.PT_rowptr.end() - 1);
  for (int f = 0; f < n; ++f)
    for (int q = out.P_rowptr[f]; q < out.P_rowptr[f + 1]; ++q) {
      const int32_t d = fill[out.P_col[q]]++;
      out.PT_col[d] = f;
      out.PT_val[d] = out.P_val[q];
    }
}

std::string check_level(const msp_level_desc& d, int l, bool need_owner) {
  if (d.n_nodes <= 0 || d.n_tets <= 0 || !d.xyz || !d.tets || !d.dirichlet)
    return "level " + std::to_string(l) + ": empty mesh or NULL array";
  if (need_owner && !d.owner) return "level " + std::to_string(l) + ": owner array required";
  for (int64_t k = 0; k < 4 * (int64_t)d.n_tets; ++k)
    if (d.tets[k] < 0 || d.tets[k] >= d.n_nodes)
      return "level " + std::to_string(l) + ": tet vertex out of range";
  for (int64_t k = 0; k < 3 * (int64_t)d.n_nodes; ++k)
    if (!std::isfinite(d.xyz[k])) return "level " + std::to_string(l) + ": non-finite coordinate";
  for (int e = 0; e < d.n_tets; ++e) {
    const int32_t* t = &d.tets[4 * (int64_t)e];
    const double* p0 = &d.xyz[3 * (int64_t)t[0]];
    double c[3][3];
    for (int a = 1; a < 4; ++a)
      for (int k = 0; k < 3; ++k) c[a - 1][k] = d.xyz[3 * (int64_t)t[a] + k] - p0[k];
    double D = det3(c[0], c[1], c[2]);
    double s = 0;
    for (int a = 0; a < 3; ++a) s = std::max(s, std::fabs(c[a][0]) + std::fabs(c[a][1]) + std::fabs(c[a][2]));
    if (!(std::fabs(D) > 1e-14 * s * s * s))
      return "level " + std::to_string(l) + ": degenerate tet " + std::to_string(e);
  }
  return "";
}

}  // namespace

std::string build_host_levels(const msp_level_desc* lv, int nlevels, const msp_options& o,
                              std::vector<HostLevel>& out) {
  if (nlevels < 1) return "nlevels must be >= 1";
  if (o.pde != MSP_PDE_POISSON && o.pde != MSP_PDE_ELASTICITY && o.pde != MSP_PDE_POISSON_P2 &&
      o.pde != MSP_PDE_P2P1)
    return "unknown pde";
  const bool elastic = o.pde == MSP_PDE_ELASTICITY;
  const bool p2 = o.pde == MSP_PDE_POISSON_P2 || o.pde == MSP_PDE_P2P1;
  if (o.pde == MSP_PDE_P2P1 && !(o.coupling > 0.0 && std::isfinite(o.coupling)))
    return "the P2-P1 system needs a coupling coefficient > 0";
  if (p2 && o.transfer != MSP_TRANSFER_BARY) return "P2 elements take the barycentric-rule transfers (P2 interpolation)";
  if (p2 && o.load_kind != MSP_F_ONE) return "P2 elements support the load f = 1 only";
  if (elastic && !(o.poisson_ratio > 0.0 && o.poisson_ratio < 0.5))
    return "linear elasticity needs a Poisson ratio in (0, 0.5)";
  if (elastic && o.transfer != MSP_TRANSFER_BARY)
    return "linear elasticity takes the barycentric transfers (field-split P)";
  out.assign(nlevels, HostLevel());
  for (int l = 0; l < nlevels; ++l) {
    const bool need_owner = l + 1 < nlevels || o.coarse_solver == MSP_COARSE_RAS;
    std::string e = check_level(lv[l], l, need_owner);
    if (!e.empty()) return e;
    HostLevel& L = out[l];
    L.n = L.nv = lv[l].n_nodes;
    L.m = lv[l].n_tets;
    L.xyz.assign(lv[l].xyz, lv[l].xyz + 3 * (size_t)L.n);
    L.tets.assign(lv[l].tets, lv[l].tets + 4 * (size_t)L.m);
    L.dir.resize(L.n);
    for (int i = 0; i < L.n; ++i) L.dir[i] = lv[l].dirichlet[i] ? 1 : 0;
    for (int i = 0; i < L.n; ++i)
      if (L.dir[i]) L.dir_list.push_back(i);
    if (need_owner) L.owner.assign(lv[l].owner, lv[l].owner + L.n);
    L.direct = (l + 1 == nlevels) && o.coarse_solver == MSP_COARSE_DIRECT;
    if (p2) {
      std::string e2 = build_p2_level(L, lv[l].owner, o.delta, !L.direct, o.pde == MSP_PDE_P2P1);
      if (!e2.empty()) return "level " + std::to_string(l) + ": " + e2;
      if (L.direct) build_coarsest_block(L);
      continue;
    }
    build_pattern_and_contribs(L);
    for (int i = 0; i < L.n; ++i)
      if (L.diag[i] < 0) return "level " + std::to_string(l) + ": node " + std::to_string(i) + " belongs to no tet";
    L.direct = (l + 1 == nlevels) && o.coarse_solver == MSP_COARSE_DIRECT;
    if (L.direct) build_coarsest_block(L);
    else build_subdomains(L, o.delta);
    if (L.sub_ptr[L.nsub] == 0 && L.direct && L.n > (int)L.dir_list.size())
      return "internal: empty coarsest block";
  }
  for (int l = 0; l + 1 < nlevels; ++l) {
    HostLevel& F = out[l];
    const HostLevel& C = out[l + 1];
    if (p2) {
      build_interp_p2(F, C, F);
    } else if (o.transfer == MSP_TRANSFER_MLS) {
      const double h = mls_unit(C);
      std::string e = build_mls(C, F, h, o.delta, false, F.P_rowptr, F.P_col, F.P_val);
      if (e.empty()) e = build_mls(F, C, h, o.delta, o.restrict_scaling != 0, F.PT_rowptr, F.PT_col, F.PT_val);
      if (!e.empty()) return "level " + std::to_string(l) + ": " + e;
    } else {
      build_interp(F, C, F);
    }
  }
  // DoF-level structures (several fields per vertex), then the subdomain
  // solvers' layouts on them
  for (int l = 0; l < nlevels; ++l) {
    HostLevel& L = out[l];
    if (elastic) {
      L.nslot = kElasticSlots;
      expand_fields(L);
      if (l + 1 < nlevels) {
        std::vector<int32_t> rp, cl;
        std::vector<double> vl;
        expand_csr(L.nv, L.P_rowptr, L.P_col, L.P_val, rp, cl, vl);
        L.P_rowptr.swap(rp);
        L.P_col.swap(cl);
        L.P_val.swap(vl);
        expand_csr(out[l + 1].nv, L.PT_rowptr, L.PT_col, L.PT_val, rp, cl, vl);
        L.PT_rowptr.swap(rp);
        L.PT_col.swap(cl);
        L.PT_val.swap(vl);
      }
    }
    const int fill = (l == 0) ? o.ilu_fill_fine : o.ilu_fill_coarse;
    if (!L.direct && fill >= 0) build_ilu(L, fill);
    build_factor_layout(L);
  }
  return "";
}

}  // namespace msp
