// Host-side set-up of a mesh hierarchy (done once, reused for every mu).
//
// Everything here is index bookkeeping and geometry that the paper treats as
// set-up (Algorithm 2, "construct the hierarchy"; Section 2.2 partition and
// overlap; the point location behind the interpolation weights):
//   * CSR pattern of J on every level and the element->nonzero map used by
//     the device assembly kernel,
//   * delta-overlapping subdomains and their dense extraction maps,
//   * barycentric interpolation P between consecutive levels and P^T.
#include <algorithm>
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
  for (int i = 0; i < C.n; ++i)
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
  out.assign(nlevels, HostLevel());
  for (int l = 0; l < nlevels; ++l) {
    std::string e = check_level(lv[l], l, l + 1 < nlevels);
    if (!e.empty()) return e;
    HostLevel& L = out[l];
    L.n = lv[l].n_nodes;
    L.m = lv[l].n_tets;
    L.xyz.assign(lv[l].xyz, lv[l].xyz + 3 * (size_t)L.n);
    L.tets.assign(lv[l].tets, lv[l].tets + 4 * (size_t)L.m);
    L.dir.resize(L.n);
    for (int i = 0; i < L.n; ++i) L.dir[i] = lv[l].dirichlet[i] ? 1 : 0;
    for (int i = 0; i < L.n; ++i)
      if (L.dir[i]) L.dir_list.push_back(i);
    if (l + 1 < nlevels) L.owner.assign(lv[l].owner, lv[l].owner + L.n);
    build_pattern_and_contribs(L);
    for (int i = 0; i < L.n; ++i)
      if (L.diag[i] < 0) return "level " + std::to_string(l) + ": node " + std::to_string(i) + " belongs to no tet";
    L.coarsest = (l + 1 == nlevels);
    if (L.coarsest) build_coarsest_block(L);
    else build_subdomains(L, o.delta);
    if (L.sub_ptr[L.nsub] == 0 && L.coarsest && L.n > (int)L.dir_list.size())
      return "internal: empty coarsest block";
    build_factor_layout(L);
  }
  for (int l = 0; l + 1 < nlevels; ++l) build_interp(out[l], out[l + 1], out[l]);
  return "";
}

}  // namespace msp
