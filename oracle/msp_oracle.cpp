// Oracle for the non-nested multilevel smoothed Schwarz method (arXiv 2412.08981).
//
// TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct FP64 CPU
// restatement of what the GPU library computes.  It shares no code with the
// library (no headers, helpers or tables) and is only ever loaded by the tests,
// by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.
//
// Every function follows the paper's statement step by step, in its order:
//   * discretisation J u = b of a linear PDE on a mesh (Section 2.1, Eq. 2-4),
//     realised as P1 finite elements for -div(k(x;mu) grad u) = f, or, as the
//     multi-field case of the mesh perspective (Section 2.1: DoF distribution
//     N = (3,0,0,0), three displacement fields per vertex), for linear
//     elasticity -div sigma(u) = f with sigma = k(x;mu) (2 mu_L eps(u) +
//     lambda_L tr(eps(u)) I), Lame parameters of a unit Young's modulus;
//   * one-level restricted additive Schwarz (Section 2.2, Eq. 6-8);
//   * the V-cycle of Algorithm 2 (Section 3.3), with the readings listed below;
//   * right-preconditioned (flexible) GMRES (Section 2.1, Eq. 5; Section 4).
// Readings where the paper is silent (shared with the library by specification,
// not by code):
//   * the transfers are either P (coarse->fine) and P^T (fine->coarse), P the
//     P1 barycentric interpolation of coarse fields at fine nodes, or the
//     overlapping MLS operators of Section 3.2 (Eq. 13-15, 24) in both
//     directions, with the readings stated at build_mls below;
//   * the coarsest level is solved directly, or (coarse_ras) smoothed like the
//     others as Algorithm 2 states: nu_pre RAS steps from z = 0; with a single
//     level that is the one-level RAS preconditioner;
//   * the smoothing loops of Algorithm 2 run exactly `its` times;
//   * subdomain solvers are unpivoted LU of each (SPD) subdomain block;
//   * Dirichlet rows are identity rows, Dirichlet columns are zeroed;
//   * k(x;mu) is evaluated at the tet centroid, f at the vertices (vertex rule);
//   * with several fields, DoF 3v + c is field c at vertex v; a Dirichlet
//     vertex fixes all its fields; the transfers are split by field (the
//     field-splitting interpolation I = sum_f R_f^T I_f R~_f of Section 2.1
//     with the scalar P for every field: P (x) I_3);
//   * with quadratic (P2) elements for the scalar problem, DoFs sit at the
//     vertices and at the edge midpoints (the DoF distribution N = (1,1,0,0)
//     of Section 2.1); see "P2 elements" below for their numbering, the
//     Dirichlet edges, the subdomains and the transfer between levels.
// Compiled with -O2 -ffp-contract=off, OpenMP over subdomains and rows only.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace {

struct Csr {
  std::vector<int> rowptr, col;
  std::vector<double> val;
};

struct Subdomain {
  std::vector<int> dofs;           // sorted global DoF ids (non-Dirichlet)
  std::vector<unsigned char> own;  // 1 where the DoF is owned (R^0 rows)
  std::vector<double> lu;          // dense n x n row-major, Doolittle LU in place
  Csr ilu;                         // ILU(p) instead: unit L below, U on and above the diagonal
  std::vector<int> udiag;          // position of the diagonal entry in each row of ilu
};

struct Level {
  int n = 0, m = 0;  // DoFs (fields x vertices, or vertices + edges with P2) and tets
  int nv = 0;        // vertices
  // P2 only: the edges (vertex pairs a < b, ascending), the global DoF of the
  // 10 local DoFs of every tet, the point of every DoF, the vertex owners
  std::vector<int> edges;
  std::vector<int> tdof;
  std::vector<double> dofx;
  std::vector<int> vowner;
  int nloc = 10;                // local DoFs per tet: 10 (P2), 14 (P2 u and P1 p)
  std::vector<unsigned char> pdof;  // P2-P1 only: 1 for the DoFs of the P1 field p
  std::vector<double> xyz;
  std::vector<int> tets;
  std::vector<unsigned char> vdir;  // per vertex
  std::vector<unsigned char> dir;   // per DoF
  std::vector<int> owner;           // per DoF (the owner of its vertex)
  Csr A;                  // assembled operator (pattern + values)
  std::vector<double> b;  // load vector
  std::vector<Subdomain> subs;
  Subdomain coarse;       // used on the coarsest level: all interior DoFs
  Csr P;                  // interpolation from level+1 (coarse) to this level
  Csr PT;                 // restriction to level+1: P^T, or the MLS operator
  int ilu_fill = -1;      // subdomain solver: dense LU (-1) or ILU(p), p = ilu_fill
};

struct Oracle {
  std::vector<Level> lv;
  int fields = 1;                     // DoFs per vertex: 1 (scalar) or 3 (elasticity)
  int p2 = 0;                         // 1: quadratic elements (DoFs on vertices and edges)
  int twofield = 0;                   // 1: the coupled system of a P2 field u and a P1 field p
  double sigma = 1.0;                 // its coupling coefficient
  double lame_l = 0.0, lame_m = 0.0;  // Lame parameters of the unit-modulus material
  int delta = 1, nu_pre = 2, nu_post = 2;
  int coef_kind = 0;  // 0: k = 1; 1: exp(s * sum_j mu_j * 0.5 * cos(pi a_j . x))
  int wave[24] = {0};
  double coef_scale = 1.0;
  int load_kind = 0;  // 0: f = 1; 1: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
  int transfer = 0;   // 0: P / P^T; 1: MLS both ways (Section 3.2)
  int restrict_scaling = 1;  // MLS restriction: 1 nodal-volume scaled, 0 plain
  int coarse_ras = 0;        // 1: the coarsest level is RAS-smoothed (Algorithm 2)
  std::vector<double> mu;
  std::string err;
};

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- geometry
// Barycentric gradients of a tet: lambda = J^{-1} (x - x0) with
// J = [x1-x0, x2-x0, x3-x0]; rows of J^{-1} are (e2 x e3, e3 x e1, e1 x e2)/det.
void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// grad[4][3], returns det (signed); volume = |det| / 6.
double tet_gradients(const double* x0, const double* x1, const double* x2, const double* x3,
                     double grad[4][3]) {
  double e1[3], e2[3], e3[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = x1[d] - x0[d];
    e2[d] = x2[d] - x0[d];
    e3[d] = x3[d] - x0[d];
  }
  double c23[3], c31[3], c12[3];
  cross(e2, e3, c23);
  cross(e3, e1, c31);
  cross(e1, e2, c12);
  double det = dot3(e1, c23);
  for (int d = 0; d < 3; ++d) {
    grad[1][d] = c23[d] / det;
    grad[2][d] = c31[d] / det;
    grad[3][d] = c12[d] / det;
    grad[0][d] = -(grad[1][d] + grad[2][d] + grad[3][d]);
  }
  return det;
}

// ------------------------------------------------------ coefficient and load
double coefficient(const Oracle& o, const double* x) {
  if (o.coef_kind == 0) return 1.0;
  double s = 0.0;
  for (int j = 0; j < 8; ++j) {
    double ax = o.wave[3 * j] * x[0] + o.wave[3 * j + 1] * x[1] + o.wave[3 * j + 2] * x[2];
    s += o.mu[j] * 0.5 * std::cos(kPi * ax);
  }
  return std::exp(o.coef_scale * s);
}

double load_f(const Oracle& o, const double* x) {
  if (o.load_kind == 0) return 1.0;
  return 3.0 * kPi * kPi * std::sin(kPi * x[0]) * std::sin(kPi * x[1]) * std::sin(kPi * x[2]);
}

// Body force of the elasticity problem, component c.  Load 0: unit force
// along -z.  Load 1: the force for which u = (s, s, s), s = sin(pi x)
// sin(pi y) sin(pi z), solves -div sigma(u) = f with k = 1:
// div sigma = mu_L lap u + (lambda_L + mu_L) grad div u, lap s = -3 pi^2 s,
// d_c d_c s = -pi^2 s, d_c d_d s = pi^2 cos(pi x_c) cos(pi x_d) sin(pi x_e).
double load_elastic(const Oracle& o, const double* x, int c) {
  if (o.load_kind == 0) return c == 2 ? -1.0 : 0.0;
  double S[3], Cs[3];
  for (int d = 0; d < 3; ++d) {
    S[d] = std::sin(kPi * x[d]);
    Cs[d] = std::cos(kPi * x[d]);
  }
  const double s = S[0] * S[1] * S[2];
  double graddiv = -kPi * kPi * s;  // d_c d_c s
  for (int d = 0; d < 3; ++d)
    if (d != c) {
      const int e = 3 - c - d;
      graddiv += kPi * kPi * Cs[c] * Cs[d] * S[e];
    }
  return 3.0 * kPi * kPi * o.lame_m * s - (o.lame_l + o.lame_m) * graddiv;
}

// Element stiffness of linear elasticity for P1 displacements (unit k):
// K[(a,i),(b,j)] = |T| (lambda g_a[i] g_b[j] + mu g_a[j] g_b[i] + mu delta_ij g_a.g_b),
// the bilinear form int 2 mu eps(u):eps(v) + lambda div u div v with u = phi_b e_j,
// v = phi_a e_i.  K12 is row-major 12 x 12, row 3a+i, column 3b+j.
void elastic_element(const double g[4][3], double vol, double lam, double mu, double* K12) {
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 4; ++b)
        for (int j = 0; j < 3; ++j) {
          double v = lam * g[a][i] * g[b][j] + mu * g[a][j] * g[b][i];
          if (i == j) v += mu * dot3(g[a], g[b]);
          K12[(3 * a + i) * 12 + 3 * b + j] = vol * v;
        }
}

// ------------------------------------------------------------ P2 elements
// Quadratic Lagrange elements for the scalar problem.  Local DoFs of a tet:
// its vertices 0..3, then its edges 01, 02, 03, 12, 13, 23.  Basis functions
// in barycentric coordinates: vertex a, lambda_a (2 lambda_a - 1); edge ab,
// 4 lambda_a lambda_b.  Element integrals by the 4-point rule that is exact
// for polynomials of degree 2 (the integrands grad phi_i . grad phi_j are of
// degree 2, phi_i of degree 2): barycentric points (A,B,B,B) and their
// permutations, A = (5 + 3 sqrt 5)/20, B = (5 - sqrt 5)/20, weights |T|/4.
const int kP2Edge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

double p2_phi(int i, const double lam[4]) {
  if (i < 4) return lam[i] * (2.0 * lam[i] - 1.0);
  const int a = kP2Edge[i - 4][0], b = kP2Edge[i - 4][1];
  return 4.0 * lam[a] * lam[b];
}

void p2_grad(int i, const double lam[4], const double g[4][3], double out[3]) {
  for (int d = 0; d < 3; ++d) {
    if (i < 4) {
      out[d] = (4.0 * lam[i] - 1.0) * g[i][d];
    } else {
      const int a = kP2Edge[i - 4][0], b = kP2Edge[i - 4][1];
      out[d] = 4.0 * (lam[a] * g[b][d] + lam[b] * g[a][d]);
    }
  }
}

// K10[i][j] = int_T grad phi_i . grad phi_j, m1[i] = int_T phi_i.
void p2_element(const double g[4][3], double vol, double* K10, double* m1) {
  const double A = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, B = (5.0 - std::sqrt(5.0)) / 20.0;
  for (int k = 0; k < 100; ++k) K10[k] = 0.0;
  for (int i = 0; i < 10; ++i) m1[i] = 0.0;
  for (int q = 0; q < 4; ++q) {
    double lam[4] = {B, B, B, B};
    lam[q] = A;
    double gr[10][3];
    for (int i = 0; i < 10; ++i) p2_grad(i, lam, g, gr[i]);
    for (int i = 0; i < 10; ++i) {
      m1[i] += vol / 4.0 * p2_phi(i, lam);
      for (int j = 0; j < 10; ++j) K10[i * 10 + j] += vol / 4.0 * dot3(gr[i], gr[j]);
    }
  }
}

// The coupled two-field element (u in P2, p in P1; unit k):
//   K_uu = int grad phi_i . grad phi_j + sigma int phi_i phi_j,
//   K_up = -sigma int phi_i lambda_b,
//   K_pp = int grad lambda_a . grad lambda_b + sigma int lambda_a lambda_b,
// local DoFs 0..9 the P2 ones (as p2_element), 10..13 the P1 ones; m1 = the
// integrals of the 14 basis functions.  Integrals by the collapsed (Duffy)
// map of the reference tet from the unit cube with 4 Gauss-Legendre points
// per direction, exact for these integrands (degree <= 4).
void coupled_element(const double g[4][3], double vol, double sigma, double* K14, double* m1) {
  const double gx[4] = {0.5 - 0.5 * 0.8611363115940526, 0.5 - 0.5 * 0.3399810435848563,
                        0.5 + 0.5 * 0.3399810435848563, 0.5 + 0.5 * 0.8611363115940526};
  const double gw[4] = {0.5 * 0.3478548451374538, 0.5 * 0.6521451548625461, 0.5 * 0.6521451548625461,
                        0.5 * 0.3478548451374538};
  for (int k = 0; k < 196; ++k) K14[k] = 0.0;
  for (int i = 0; i < 14; ++i) m1[i] = 0.0;
  for (int ia = 0; ia < 4; ++ia)
    for (int ib = 0; ib < 4; ++ib)
      for (int ic = 0; ic < 4; ++ic) {
        const double a = gx[ia], b = gx[ib], c = gx[ic];
        const double xi = a, eta = b * (1.0 - a), zeta = c * (1.0 - a) * (1.0 - b);
        const double w = 6.0 * vol * gw[ia] * gw[ib] * gw[ic] * (1.0 - a) * (1.0 - a) * (1.0 - b);
        const double lam[4] = {1.0 - xi - eta - zeta, xi, eta, zeta};
        double val[14], gr[14][3];
        for (int i = 0; i < 10; ++i) {
          val[i] = p2_phi(i, lam);
          p2_grad(i, lam, g, gr[i]);
        }
        for (int q = 0; q < 4; ++q) {
          val[10 + q] = lam[q];
          for (int d = 0; d < 3; ++d) gr[10 + q][d] = g[q][d];
        }
        for (int i = 0; i < 14; ++i) {
          m1[i] += w * val[i];
          for (int j = 0; j < 14; ++j) {
            const bool same = (i < 10) == (j < 10);
            const double v = same ? dot3(gr[i], gr[j]) + sigma * val[i] * val[j] : -sigma * val[i] * val[j];
            K14[i * 14 + j] += w * v;
          }
        }
      }
}

// The P2 DoFs of a level.  Edges: the distinct vertex pairs (a, b), a < b, of
// the tets, ascending.  Numbering: vertex 0, then the edges (0, b) in
// ascending b, then vertex 1 and its edges (1, b), b > 1, and so on (a DoF
// next to the DoFs of its neighbourhood, so subdomain blocks stay banded).
// An edge DoF sits at the edge's midpoint.  Dirichlet: a vertex as given; an
// edge when it lies on a boundary face (a face of exactly one tet) whose three
// vertices are Dirichlet.  Owner: a vertex's own; an edge takes the owner of
// its lower vertex if that id owns a non-Dirichlet vertex, else the owner of
// its upper vertex.  Returns false if an edge gets no owner.
// With the coupled system (twofield), each vertex also carries the DoF of the
// P1 field p, right after its P2 (u) DoF: vertex 0's u, vertex 0's p, the
// edges (0, b), vertex 1's u, ...; local DoFs 10..13 of a tet are the p DoFs
// of its vertices; a p DoF is Dirichlet and owned as its vertex.
bool p2_number(Level& L, const int* vowner, bool twofield = false) {
  std::vector<std::pair<int, int>> E;
  for (int e = 0; e < L.m; ++e)
    for (int k = 0; k < 6; ++k) {
      int a = L.tets[4 * e + kP2Edge[k][0]], b = L.tets[4 * e + kP2Edge[k][1]];
      E.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(E.begin(), E.end());
  E.erase(std::unique(E.begin(), E.end()), E.end());
  const int ne = (int)E.size();
  L.edges.assign(2 * (size_t)ne, 0);
  for (int k = 0; k < ne; ++k) {
    L.edges[2 * k] = E[k].first;
    L.edges[2 * k + 1] = E[k].second;
  }
  std::vector<int> vdof(L.nv), pdof(L.nv, -1), edof(ne);
  int cnt = 0, k = 0;
  for (int v = 0; v < L.nv; ++v) {
    vdof[v] = cnt++;
    if (twofield) pdof[v] = cnt++;
    while (k < ne && E[k].first == v) edof[k++] = cnt++;
  }
  L.n = cnt;
  const int NL = twofield ? 14 : 10;
  L.nloc = NL;
  L.tdof.assign(NL * (size_t)L.m, 0);
  for (int e = 0; e < L.m; ++e) {
    const int* t = &L.tets[4 * e];
    for (int a = 0; a < 4; ++a) L.tdof[NL * e + a] = vdof[t[a]];
    for (int q = 0; q < 6; ++q) {
      std::pair<int, int> key{std::min(t[kP2Edge[q][0]], t[kP2Edge[q][1]]),
                              std::max(t[kP2Edge[q][0]], t[kP2Edge[q][1]])};
      L.tdof[NL * e + 4 + q] = edof[std::lower_bound(E.begin(), E.end(), key) - E.begin()];
    }
    if (twofield)
      for (int a = 0; a < 4; ++a) L.tdof[NL * e + 10 + a] = pdof[t[a]];
  }
  L.dofx.assign(3 * (size_t)L.n, 0.0);
  L.dir.assign(L.n, 0);
  L.pdof.assign(L.n, 0);
  for (int v = 0; v < L.nv; ++v) {
    for (int d = 0; d < 3; ++d) L.dofx[3 * vdof[v] + d] = L.xyz[3 * v + d];
    L.dir[vdof[v]] = L.vdir[v];
    if (twofield) {
      for (int d = 0; d < 3; ++d) L.dofx[3 * pdof[v] + d] = L.xyz[3 * v + d];
      L.dir[pdof[v]] = L.vdir[v];
      L.pdof[pdof[v]] = 1;
    }
  }
  for (int q = 0; q < ne; ++q)
    for (int d = 0; d < 3; ++d)
      L.dofx[3 * edof[q] + d] = 0.5 * (L.xyz[3 * E[q].first + d] + L.xyz[3 * E[q].second + d]);
  std::map<std::array<int, 3>, int> faces;
  for (int e = 0; e < L.m; ++e)
    for (int skip = 0; skip < 4; ++skip) {
      std::array<int, 3> f;
      int c = 0;
      for (int a = 0; a < 4; ++a)
        if (a != skip) f[c++] = L.tets[4 * e + a];
      std::sort(f.begin(), f.end());
      faces[f]++;
    }
  for (const auto& fc : faces) {
    if (fc.second != 1) continue;
    const auto& f = fc.first;
    if (!(L.vdir[f[0]] && L.vdir[f[1]] && L.vdir[f[2]])) continue;
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b) {
        std::pair<int, int> key{std::min(f[a], f[b]), std::max(f[a], f[b])};
        L.dir[edof[std::lower_bound(E.begin(), E.end(), key) - E.begin()]] = 1;
      }
  }
  if (vowner) {
    L.vowner.assign(vowner, vowner + L.nv);
    std::set<int> ids;
    for (int v = 0; v < L.nv; ++v)
      if (!L.vdir[v]) ids.insert(vowner[v]);
    L.owner.assign(L.n, -1);
    for (int v = 0; v < L.nv; ++v) {
      L.owner[vdof[v]] = vowner[v];
      if (twofield) L.owner[pdof[v]] = vowner[v];
    }
    for (int q = 0; q < ne; ++q) {
      const int oa = vowner[E[q].first], ob = vowner[E[q].second];
      L.owner[edof[q]] = ids.count(oa) ? oa : (ids.count(ob) ? ob : -1);
      if (L.owner[edof[q]] < 0 && !L.dir[edof[q]]) return false;
    }
  }
  return true;
}

// Row i of the P2 pattern: the DoFs of the tets that hold DoF i, sorted.
void build_pattern_p2(Level& L) {
  const int NL = L.nloc;
  std::vector<std::set<int>> nb(L.n);
  for (int e = 0; e < L.m; ++e)
    for (int i = 0; i < NL; ++i)
      for (int j = 0; j < NL; ++j) nb[L.tdof[NL * e + i]].insert(L.tdof[NL * e + j]);
  L.A.rowptr.assign(L.n + 1, 0);
  L.A.col.clear();
  for (int i = 0; i < L.n; ++i) {
    for (int j : nb[i]) L.A.col.push_back(j);
    L.A.rowptr[i + 1] = (int)L.A.col.size();
  }
  L.A.val.assign(L.A.col.size(), 0.0);
}

// ------------------------------------------------------------- CSR pattern
// Row i: the sorted distinct vertices that share a tet with i (i included);
// with F fields, row F v + c holds the F DoFs of each of those vertices.
void build_pattern(Level& L, int F) {
  std::vector<std::set<int>> nb(L.nv);
  for (int e = 0; e < L.m; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) nb[L.tets[4 * e + a]].insert(L.tets[4 * e + b]);
  L.A.rowptr.assign(L.n + 1, 0);
  L.A.col.clear();
  for (int v = 0; v < L.nv; ++v)
    for (int c = 0; c < F; ++c) {
      for (int w : nb[v])
        for (int c2 = 0; c2 < F; ++c2) L.A.col.push_back(F * w + c2);
      L.A.rowptr[F * v + c + 1] = (int)L.A.col.size();
    }
  L.A.val.assign(L.A.col.size(), 0.0);
}

long csr_find(const Csr& A, int i, int j) {
  auto b = A.col.begin() + A.rowptr[i], e = A.col.begin() + A.rowptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return it - A.col.begin();
}

// --------------------------------------------------------------- assembly
// J(i,j) = sum over tets T (ascending id) of int_T k grad phi_j . grad phi_i
// (Eq. 4 for the P1 Galerkin scheme), k at the centroid; then Dirichlet rows
// become identity rows and Dirichlet columns are zeroed.
// b(a) = sum over tets T containing a of f(x_a) |T| / 4 (vertex rule), 0 on
// Dirichlet nodes.
int assemble_level(const Oracle& o, Level& L) {
  std::fill(L.A.val.begin(), L.A.val.end(), 0.0);
  L.b.assign(L.n, 0.0);
  for (int e = 0; e < L.m; ++e) {
    const int* t = &L.tets[4 * e];
    const double* x[4];
    for (int a = 0; a < 4; ++a) x[a] = &L.xyz[3 * t[a]];
    double g[4][3];
    double det = tet_gradients(x[0], x[1], x[2], x[3], g);
    double vol = std::fabs(det) / 6.0;
    if (!(vol > 0.0)) return -1;
    double xc[3];
    for (int d = 0; d < 3; ++d) xc[d] = (x[0][d] + x[1][d] + x[2][d] + x[3][d]) / 4.0;
    double k = coefficient(o, xc);
    if (o.p2) {  // quadratic elements: DoFs at the vertices and edge midpoints
      const int NL = L.nloc;
      double Ke[196], m1[14];
      if (o.twofield) coupled_element(g, vol, o.sigma, Ke, m1);
      else p2_element(g, vol, Ke, m1);
      const int* td = &L.tdof[NL * e];
      for (int i = 0; i < NL; ++i) {
        for (int j = 0; j < NL; ++j) {
          long nz = csr_find(L.A, td[i], td[j]);
          L.A.val[nz] += k * Ke[i * NL + j];
        }
        L.b[td[i]] += m1[i];  // f = 1 (for every field): b_i = int phi_i
      }
      continue;
    }
    if (o.fields == 3) {  // linear elasticity, three displacement fields
      double K12[144];
      elastic_element(g, vol, o.lame_l, o.lame_m, K12);
      for (int a = 0; a < 4; ++a) {
        for (int i = 0; i < 3; ++i)
          for (int b = 0; b < 4; ++b)
            for (int j = 0; j < 3; ++j) {
              long nz = csr_find(L.A, 3 * t[a] + i, 3 * t[b] + j);
              L.A.val[nz] += k * K12[(3 * a + i) * 12 + 3 * b + j];
            }
        for (int c = 0; c < 3; ++c) L.b[3 * t[a] + c] += load_elastic(o, x[a], c) * vol / 4.0;
      }
      continue;
    }
    for (int a = 0; a < 4; ++a) {
      for (int b = 0; b < 4; ++b) {
        long nz = csr_find(L.A, t[a], t[b]);
        L.A.val[nz] += k * vol * dot3(g[a], g[b]);
      }
      L.b[t[a]] += load_f(o, x[a]) * vol / 4.0;
    }
  }
  for (int i = 0; i < L.n; ++i) {
    for (int p = L.A.rowptr[i]; p < L.A.rowptr[i + 1]; ++p) {
      int j = L.A.col[p];
      if (L.dir[i]) L.A.val[p] = (i == j) ? 1.0 : 0.0;
      else if (L.dir[j]) L.A.val[p] = 0.0;
    }
    if (L.dir[i]) L.b[i] = 0.0;
  }
  return 0;
}

void spmv(const Csr& A, const double* x, double* y) {
  int n = (int)A.rowptr.size() - 1;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
    y[i] = s;
  }
}

// ------------------------------------------------------- subdomains (2.2)
// Owners come from the vertex partition; a subdomain exists for every owner id
// that owns at least one non-Dirichlet vertex, in ascending owner id.  The
// overlap adds delta layers: V^{k+1} = vertices of tets touching V^k.
void build_subdomains(const Oracle& o, Level& L) {
  L.subs.clear();
  std::set<int> ids;
  for (int i = 0; i < L.n; ++i)
    if (!L.dir[i]) ids.insert(L.owner[i]);
  for (int id : ids) {
    std::vector<unsigned char> in(L.n, 0);
    for (int i = 0; i < L.n; ++i)
      if (L.owner[i] == id) in[i] = 1;
    for (int layer = 0; layer < o.delta; ++layer) {
      std::vector<unsigned char> nxt = in;
      for (int i = 0; i < L.n; ++i)
        if (in[i])
          for (int p = L.A.rowptr[i]; p < L.A.rowptr[i + 1]; ++p) nxt[L.A.col[p]] = 1;
      in.swap(nxt);
    }
    Subdomain S;
    for (int i = 0; i < L.n; ++i)
      if (in[i] && !L.dir[i]) {
        S.dofs.push_back(i);
        S.own.push_back(L.owner[i] == id ? 1 : 0);
      }
    L.subs.push_back(std::move(S));
  }
}

// P2 subdomains: the vertex sets grow as for P1 (V^0 = the vertices with
// owner id, Dirichlet ones included; V^{k+1} = the vertices of the tets
// touching V^k, delta times); the subdomain holds the non-Dirichlet vertex
// DoFs of V^delta and the non-Dirichlet edge DoFs with both ends in V^delta,
// ascending; a DoF is owned where its owner is the subdomain's id.
void build_subdomains_p2(const Oracle& o, Level& L) {
  L.subs.clear();
  std::set<int> ids;
  for (int v = 0; v < L.nv; ++v)
    if (!L.vdir[v]) ids.insert(L.vowner[v]);
  std::vector<std::vector<int>> vt(L.nv);
  for (int e = 0; e < L.m; ++e)
    for (int a = 0; a < 4; ++a) vt[L.tets[4 * e + a]].push_back(e);
  for (int id : ids) {
    std::vector<unsigned char> in(L.nv, 0);
    for (int v = 0; v < L.nv; ++v)
      if (L.vowner[v] == id) in[v] = 1;
    for (int layer = 0; layer < o.delta; ++layer) {
      std::vector<unsigned char> nxt = in;
      for (int v = 0; v < L.nv; ++v)
        if (in[v])
          for (int e : vt[v])
            for (int a = 0; a < 4; ++a) nxt[L.tets[4 * e + a]] = 1;
      in.swap(nxt);
    }
    std::vector<unsigned char> take(L.n, 0);
    const int NL = L.nloc;
    for (int e = 0; e < L.m; ++e) {
      const int* t = &L.tets[4 * e];
      for (int a = 0; a < 4; ++a)
        if (in[t[a]]) {
          take[L.tdof[NL * e + a]] = 1;
          if (NL == 14) take[L.tdof[NL * e + 10 + a]] = 1;
        }
      for (int q = 0; q < 6; ++q)
        if (in[t[kP2Edge[q][0]]] && in[t[kP2Edge[q][1]]]) take[L.tdof[NL * e + 4 + q]] = 1;
    }
    Subdomain S;
    for (int i = 0; i < L.n; ++i)
      if (take[i] && !L.dir[i]) {
        S.dofs.push_back(i);
        S.own.push_back(L.owner[i] == id ? 1 : 0);
      }
    L.subs.push_back(std::move(S));
  }
}

void build_coarse(Level& L) {
  L.coarse = Subdomain();
  for (int i = 0; i < L.n; ++i)
    if (!L.dir[i]) {
      L.coarse.dofs.push_back(i);
      L.coarse.own.push_back(1);
    }
}

// ------------------------------------------------------------ dense LU
// Doolittle LU without pivoting, k-i-j order, in place (unit L below the
// diagonal, U on and above it).  Returns -1 on a zero pivot.
int lu_factor(int n, double* A) {
  for (int k = 0; k < n; ++k) {
    double piv = A[(size_t)k * n + k];
    if (piv == 0.0 || !std::isfinite(piv)) return -1;
    // rows are independent at fixed k (large blocks only; nested regions stay serial)
#pragma omp parallel for schedule(static) if (n > 1024)
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / piv;
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

void lu_solve(int n, const double* LU, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * x[j];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * x[j];
    x[i] = s / LU[(size_t)i * n + i];
  }
}

// A_p = R_p A R_p^T as a dense block (Eq. 6).
void extract_dense(const Csr& A, const Subdomain& S, std::vector<double>& D) {
  int n = (int)S.dofs.size();
  D.assign((size_t)n * n, 0.0);
  for (int li = 0; li < n; ++li) {
    int i = S.dofs[li];
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      auto it = std::lower_bound(S.dofs.begin(), S.dofs.end(), A.col[p]);
      if (it != S.dofs.end() && *it == A.col[p]) D[(size_t)li * n + (it - S.dofs.begin())] = A.val[p];
    }
  }
}

// ------------------------------------------------ ILU(p) (Section 4.4's solver)
// Incomplete LU of a subdomain block with the level-of-fill pattern: entries of
// A_p have level 0; eliminating with row k gives entry (i, j) the level
// lev(i,k) + lev(k,j) + 1, the smaller of its levels is kept, and entries of
// level > p are dropped.  The numbers then follow Gaussian elimination in IKJ
// order restricted to that pattern (the updates of dropped entries are lost).

// A_p as a local CSR (rows and columns in the sorted DoF order).
void local_block(const Csr& A, const Subdomain& S, Csr& B) {
  const int n = (int)S.dofs.size();
  B.rowptr.assign(n + 1, 0);
  B.col.clear();
  B.val.clear();
  for (int li = 0; li < n; ++li) {
    const int g = S.dofs[li];
    for (int q = A.rowptr[g]; q < A.rowptr[g + 1]; ++q) {
      auto it = std::lower_bound(S.dofs.begin(), S.dofs.end(), A.col[q]);
      if (it != S.dofs.end() && *it == A.col[q]) {
        B.col.push_back((int)(it - S.dofs.begin()));
        B.val.push_back(A.val[q]);
      }
    }
    B.rowptr[li + 1] = (int)B.col.size();
  }
}

// The ILU(p) pattern of B (sorted columns per row, diagonal included).
void ilu_symbolic(const Csr& B, int p, Csr& F) {
  const int n = (int)B.rowptr.size() - 1;
  std::vector<std::vector<int>> cols(n), levs(n);
  std::vector<int> lev(n, INT32_MAX);
  for (int i = 0; i < n; ++i) {
    std::set<int> row;
    for (int q = B.rowptr[i]; q < B.rowptr[i + 1]; ++q) {
      row.insert(B.col[q]);
      lev[B.col[q]] = 0;
    }
    row.insert(i);
    lev[i] = 0;
    for (auto it = row.begin(); it != row.end() && *it < i; ++it) {
      const int k = *it;
      if (lev[k] > p) continue;
      for (size_t t = 0; t < cols[k].size(); ++t) {
        const int j = cols[k][t];
        if (j <= k) continue;
        const int nl = lev[k] + levs[k][t] + 1;
        if (nl > p) continue;
        if (nl < lev[j]) lev[j] = nl;
        row.insert(j);  // std::set iterators stay valid; j > k, so the loop reaches it
      }
    }
    for (int j : row)
      if (lev[j] <= p) {
        cols[i].push_back(j);
        levs[i].push_back(lev[j]);
      }
    for (int j : row) lev[j] = INT32_MAX;
  }
  F.rowptr.assign(n + 1, 0);
  F.col.clear();
  for (int i = 0; i < n; ++i) {
    F.col.insert(F.col.end(), cols[i].begin(), cols[i].end());
    F.rowptr[i + 1] = (int)F.col.size();
  }
  F.val.assign(F.col.size(), 0.0);
}

// IKJ elimination on the pattern of F; returns -1 on a zero or non-finite pivot.
int ilu_numeric(const Csr& B, Csr& F, std::vector<int>& udiag) {
  const int n = (int)F.rowptr.size() - 1;
  udiag.assign(n, -1);
  std::vector<int> pos(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int q = F.rowptr[i]; q < F.rowptr[i + 1]; ++q) {
      pos[F.col[q]] = q;
      F.val[q] = 0.0;
      if (F.col[q] == i) udiag[i] = q;
    }
    for (int q = B.rowptr[i]; q < B.rowptr[i + 1]; ++q) F.val[pos[B.col[q]]] = B.val[q];
    for (int q = F.rowptr[i]; q < F.rowptr[i + 1] && F.col[q] < i; ++q) {
      const int k = F.col[q];
      const double piv = F.val[udiag[k]];
      if (piv == 0.0 || !std::isfinite(piv)) return -1;
      const double lik = F.val[q] / piv;
      F.val[q] = lik;
      for (int t = udiag[k] + 1; t < F.rowptr[k + 1]; ++t)
        if (pos[F.col[t]] >= 0) F.val[pos[F.col[t]]] -= lik * F.val[t];
    }
    for (int q = F.rowptr[i]; q < F.rowptr[i + 1]; ++q) pos[F.col[q]] = -1;
    if (udiag[i] < 0 || !(std::isfinite(F.val[udiag[i]])) || F.val[udiag[i]] == 0.0) return -1;
  }
  return 0;
}

// x <- (L U)^{-1} x with the unit lower L and upper U of F.
void ilu_solve(const Csr& F, const std::vector<int>& udiag, double* x) {
  const int n = (int)F.rowptr.size() - 1;
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int q = F.rowptr[i]; q < udiag[i]; ++q) s -= F.val[q] * x[F.col[q]];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int q = udiag[i] + 1; q < F.rowptr[i + 1]; ++q) s -= F.val[q] * x[F.col[q]];
    x[i] = s / F.val[udiag[i]];
  }
}

int factor_sub(const Csr& A, Subdomain& S, int ilu_fill = -1) {
  if (ilu_fill >= 0) {
    Csr B;
    local_block(A, S, B);
    if (S.ilu.rowptr.empty()) ilu_symbolic(B, ilu_fill, S.ilu);
    return ilu_numeric(B, S.ilu, S.udiag);
  }
  extract_dense(A, S, S.lu);
  return lu_factor((int)S.dofs.size(), S.lu.data());
}

void sub_solve(const Subdomain& S, double* t) {
  if (!S.ilu.rowptr.empty()) ilu_solve(S.ilu, S.udiag, t);
  else lu_solve((int)S.dofs.size(), S.lu.data(), t);
}

// ------------------------------------------------------------- RAS (2.2)
// z = sum_p (R^0_p)^T (A_p)^{-1} R^delta_p r  on non-Dirichlet DoFs, z_i = r_i
// on Dirichlet DoFs (identity rows).
void ras_apply(const Level& L, const double* r, double* z) {
  for (int i = 0; i < L.n; ++i) z[i] = L.dir[i] ? r[i] : 0.0;
  int np = (int)L.subs.size();
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < np; ++p) {
    const Subdomain& S = L.subs[p];
    int n = (int)S.dofs.size();
    std::vector<double> t(n);
    for (int li = 0; li < n; ++li) t[li] = r[S.dofs[li]];
    sub_solve(S, t.data());
    for (int li = 0; li < n; ++li)
      if (S.own[li]) z[S.dofs[li]] += t[li];  // each DoF is owned once: no race
  }
}

void coarse_solve(const Level& L, const double* r, double* z) {
  for (int i = 0; i < L.n; ++i) z[i] = L.dir[i] ? r[i] : 0.0;
  const Subdomain& S = L.coarse;
  int n = (int)S.dofs.size();
  std::vector<double> t(n);
  for (int li = 0; li < n; ++li) t[li] = r[S.dofs[li]];
  lu_solve(n, S.lu.data(), t.data());
  for (int li = 0; li < n; ++li) z[S.dofs[li]] = t[li];
}

// ---------------------------------------------------- interpolation P
// For each fine non-Dirichlet node x, the coarse tet that contains it (all
// barycentric coordinates >= -1e-12; the lowest tet id if several; the tet
// maximising the smallest coordinate if none) gives the row: the raw
// barycentric weights on that tet's vertices, columns sorted.  With
// drop_dirichlet the columns of Dirichlet coarse vertices are left out and the
// rows of Dirichlet fine nodes are empty.
void barycentric(const double* xyz, const int* t, const double* x, double lam[4]) {
  double g[4][3];
  tet_gradients(&xyz[3 * t[0]], &xyz[3 * t[1]], &xyz[3 * t[2]], &xyz[3 * t[3]], g);
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = x[k] - xyz[3 * t[0] + k];
  lam[1] = dot3(g[1], d);
  lam[2] = dot3(g[2], d);
  lam[3] = dot3(g[3], d);
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

void build_interp(int nc, const double* cxyz, int mc, const int* ctets, const unsigned char* cdir,
                  int nf, const double* fxyz, const unsigned char* fdir, int drop_dirichlet,
                  Csr& P) {
  // bucket grid over the coarse bounding box; each tet goes into every bucket
  // its (slightly enlarged) bounding box overlaps.  Candidates are then tested
  // exactly, so the grid only prunes.
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < nc; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], cxyz[3 * i + d]);
      hi[d] = std::max(hi[d], cxyz[3 * i + d]);
    }
  int G = std::max(1, (int)std::cbrt((double)mc / 6.0));
  double ext[3];
  for (int d = 0; d < 3; ++d) ext[d] = std::max(hi[d] - lo[d], 1e-300);
  auto cell = [&](double v, int d) {
    int c = (int)std::floor((v - lo[d]) / ext[d] * G);
    return std::min(std::max(c, 0), G - 1);
  };
  std::vector<std::vector<int>> bucket((size_t)G * G * G);
  for (int e = 0; e < mc; ++e) {
    double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) {
        blo[d] = std::min(blo[d], cxyz[3 * ctets[4 * e + a] + d]);
        bhi[d] = std::max(bhi[d], cxyz[3 * ctets[4 * e + a] + d]);
      }
    int c0[3], c1[3];
    for (int d = 0; d < 3; ++d) {
      double pad = 1e-9 * ext[d];
      c0[d] = cell(blo[d] - pad, d);
      c1[d] = cell(bhi[d] + pad, d);
    }
    for (int k = c0[2]; k <= c1[2]; ++k)
      for (int j = c0[1]; j <= c1[1]; ++j)
        for (int i = c0[0]; i <= c1[0]; ++i) bucket[(size_t)i + G * ((size_t)j + G * k)].push_back(e);
  }
  P.rowptr.assign(nf + 1, 0);
  P.col.clear();
  P.val.clear();
  for (int f = 0; f < nf; ++f) {
    if (!fdir[f] || !drop_dirichlet) {
      const double* x = &fxyz[3 * f];
      int best = -1;
      double lam_best[4];
      const auto& cand = bucket[(size_t)cell(x[0], 0) + G * ((size_t)cell(x[1], 1) + G * cell(x[2], 2))];
      for (int e : cand) {  // candidates are in ascending tet id
        double lam[4];
        barycentric(cxyz, &ctets[4 * e], x, lam);
        if (std::min(std::min(lam[0], lam[1]), std::min(lam[2], lam[3])) >= -1e-12) {
          best = e;
          std::copy(lam, lam + 4, lam_best);
          break;
        }
      }
      if (best < 0) {  // outside every tet: take the least-violating one (all tets)
        double bm = -1e300;
        for (int e = 0; e < mc; ++e) {
          double lam[4];
          barycentric(cxyz, &ctets[4 * e], x, lam);
          double mn = std::min(std::min(lam[0], lam[1]), std::min(lam[2], lam[3]));
          if (mn > bm) {
            bm = mn;
            best = e;
            std::copy(lam, lam + 4, lam_best);
          }
        }
      }
      std::vector<std::pair<int, double>> row;
      for (int a = 0; a < 4; ++a) {
        int c = ctets[4 * best + a];
        if (drop_dirichlet && cdir[c]) continue;
        row.push_back({c, lam_best[a]});
      }
      std::sort(row.begin(), row.end());
      for (auto& pr : row) {
        P.col.push_back(pr.first);
        P.val.push_back(pr.second);
      }
    }
    P.rowptr[f + 1] = (int)P.col.size();
  }
}

void transpose(const Csr& P, int ncols, Csr& T) {
  int nr = (int)P.rowptr.size() - 1;
  T.rowptr.assign(ncols + 1, 0);
  for (int c : P.col) T.rowptr[c + 1]++;
  for (int i = 0; i < ncols; ++i) T.rowptr[i + 1] += T.rowptr[i];
  T.col.assign(P.col.size(), 0);
  T.val.assign(P.col.size(), 0.0);
  std::vector<int> pos(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int i = 0; i < nr; ++i)  // rows visited in ascending order: columns of T sorted
    for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p) {
      int q = pos[P.col[p]]++;
      T.col[q] = i;
      T.val[q] = P.val[p];
    }
}

// P2 interpolation between non-nested levels: each non-Dirichlet fine DoF's
// point (a vertex or an edge midpoint) is located in the coarse mesh exactly
// as a P1 node is (build_interp's rule, run on the DoF points); its row holds
// the ten coarse P2 basis functions of that tet evaluated there, on the
// tet's non-Dirichlet coarse DoFs, columns ascending (zero weights kept).
// With the coupled system the interpolation is split by field (Section 2.1,
// I = sum_f R_f^T I_f R~_f): rows of the P2 field u as above, on the coarse u
// DoFs; rows of the P1 field p the barycentric weights on the coarse p DoFs.
void build_interp_p2(const Level& C, const Level& F, Csr& P) {
  // the containing tet and barycentric coordinates of every fine DoF point:
  // build_interp on the DoF points with every coarse vertex kept returns the
  // four raw weights in ascending vertex order, from which the tet follows
  std::vector<unsigned char> keep(C.nv, 0);
  Csr loc;
  build_interp(C.nv, C.xyz.data(), C.m, C.tets.data(), keep.data(), F.n, F.dofx.data(), F.dir.data(), 1, loc);
  // vertex set -> tet: the coarse tet with exactly those vertices, lowest id
  std::map<std::array<int, 4>, int> tet_of;
  for (int e = C.m - 1; e >= 0; --e) {
    std::array<int, 4> key{C.tets[4 * e], C.tets[4 * e + 1], C.tets[4 * e + 2], C.tets[4 * e + 3]};
    std::sort(key.begin(), key.end());
    tet_of[key] = e;
  }
  P.rowptr.assign(F.n + 1, 0);
  P.col.clear();
  P.val.clear();
  for (int f = 0; f < F.n; ++f) {
    if (loc.rowptr[f + 1] > loc.rowptr[f]) {
      std::array<int, 4> key;
      for (int a = 0; a < 4; ++a) key[a] = loc.col[loc.rowptr[f] + a];
      const int e = tet_of.at(key);
      const int* t = &C.tets[4 * e];
      double lam[4];
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 4; ++q)
          if (loc.col[loc.rowptr[f] + q] == t[a]) lam[a] = loc.val[loc.rowptr[f] + q];
      std::vector<std::pair<int, double>> row;
      const int NL = C.nloc;
      if (!F.pdof.empty() && F.pdof[f]) {  // the P1 field: barycentric weights on the coarse p DoFs
        for (int a = 0; a < 4; ++a) {
          const int c = C.tdof[NL * e + 10 + a];
          if (C.dir[c]) continue;
          row.push_back({c, lam[a]});
        }
      } else {
        for (int i = 0; i < 10; ++i) {
          const int c = C.tdof[NL * e + i];
          if (C.dir[c]) continue;
          row.push_back({c, p2_phi(i, lam)});
        }
      }
      std::sort(row.begin(), row.end());
      for (auto& pr : row) {
        P.col.push_back(pr.first);
        P.val.push_back(pr.second);
      }
    }
    P.rowptr[f + 1] = (int)P.col.size();
  }
}

// ------------------------------------- MLS transfer (Section 3.2, Eq. 13-15, 24)
// Overlapping moving-least-squares interpolation from a source mesh S to the
// nodes of a target mesh T.  For a target node x* with partition id q:
//   N(x*) = the source vertices of Omega^delta_q (the S-vertices owned by q,
//           Dirichlet ones included, grown by delta element layers as in
//           Section 2.2) at distance < rho from x*;
//   w     = 1 - 6 s^2 + 8 s^3 - 3 s^4, s = |x - x*| / rho        (Eq. 15);
//   P1    = sum_n w_n p(x_n) p(x_n)^T,  P2[:, n] = w_n p(x_n)   (Theorem 3.2);
//   row   = p(x*)^T P1^{-1} P2                                   (Eq. 24).
// Readings of what the paper leaves open:
//   * the polynomial space is linear, written in the basis
//     p(x) = [1, (x - x*)/rho] (p(x*) = e_1); the fitted value is the same in
//     every basis of the space;
//   * rho = c h, h = cbrt(6 |bounding box| / tets) of the coarser mesh of the
//     pair, c = 1.5 and then multiplied by 1.5 until rank(P) = 4, tested as:
//     at least 4 neighbours and every pivot of the unpivoted elimination of
//     P1 above 1e-9 P1[0][0];
//   * subdomain q of S is subdomain q of T when both meshes are partitioned
//     over the same set of ids (the paper keeps np subdomains on every level);
//     when either mesh has no partition (the coarsest level) or the id sets
//     differ, N(x*) is taken from all of S;
//   * Dirichlet source vertices take part in the fit; with drop_dirichlet
//     their columns are left out (the vectors transferred vanish there) and
//     Dirichlet target nodes get empty rows;
//   * with `scale` the row is multiplied by |w_t| / |w_n| (nodal volumes
//     |w_i| = sum of |T|/4 over the tets at i): the fine->coarse transfer of a
//     residual, whose entries are integrals, goes through the densities
//     r_i / |w_i| so that its scale matches the coarse operator.
double mls_weight(double s) { return 1.0 - 6.0 * s * s + 8.0 * s * s * s - 3.0 * s * s * s * s; }

double mesh_h(const Level& C) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < C.n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], C.xyz[3 * i + d]);
      hi[d] = std::max(hi[d], C.xyz[3 * i + d]);
    }
  double vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  return std::cbrt(6.0 * vol / C.m);
}

std::vector<double> nodal_volumes(const Level& L) {
  std::vector<double> v(L.n, 0.0);
  for (int e = 0; e < L.m; ++e) {
    const int* t = &L.tets[4 * e];
    double g[4][3];
    double det = tet_gradients(&L.xyz[3 * t[0]], &L.xyz[3 * t[1]], &L.xyz[3 * t[2]], &L.xyz[3 * t[3]], g);
    double vol = std::fabs(det) / 6.0;
    for (int a = 0; a < 4; ++a) v[t[a]] += vol / 4.0;
  }
  return v;
}

// Omega^delta_q on S, ascending vertex ids.
std::vector<int> overlap_vertices(const Level& S, int q, int delta) {
  std::vector<unsigned char> in(S.n, 0);
  for (int i = 0; i < S.n; ++i)
    if (S.owner[i] == q) in[i] = 1;
  for (int layer = 0; layer < delta; ++layer) {
    std::vector<unsigned char> nxt = in;
    for (int i = 0; i < S.n; ++i)
      if (in[i])
        for (int p = S.A.rowptr[i]; p < S.A.rowptr[i + 1]; ++p) nxt[S.A.col[p]] = 1;
    in.swap(nxt);
  }
  std::vector<int> v;
  for (int i = 0; i < S.n; ++i)
    if (in[i]) v.push_back(i);
  return v;
}

// One row of Eq. 24 at x* over the candidates (ascending ids); false when
// rank(P) < 4 for this rho.
bool mls_row(const double* xs, const std::vector<double>& sxyz, const std::vector<int>& cand,
             double rho, std::vector<std::pair<int, double>>& row) {
  std::vector<int> nb;
  std::vector<double> w, p;
  for (int n : cand) {
    double d0 = sxyz[3 * n] - xs[0], d1 = sxyz[3 * n + 1] - xs[1], d2 = sxyz[3 * n + 2] - xs[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 < rho * rho)) continue;
    nb.push_back(n);
    w.push_back(mls_weight(std::sqrt(r2) / rho));
    p.insert(p.end(), {1.0, d0 / rho, d1 / rho, d2 / rho});
  }
  const int N = (int)nb.size();
  if (N < 4) return false;
  double P1[16] = {0};
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) P1[4 * i + j] += w[k] * p[4 * k + i] * p[4 * k + j];
  double LU[16];
  std::copy(P1, P1 + 16, LU);
  if (lu_factor(4, LU)) return false;
  for (int i = 0; i < 4; ++i)
    if (!(LU[5 * i] > 1e-9 * P1[0])) return false;
  double y[4] = {1.0, 0.0, 0.0, 0.0};  // p(x*)
  lu_solve(4, LU, y);                  // y = P1^{-1} p(x*), i.e. y^T = p(x*)^T P1^{-1}
  row.clear();
  for (int k = 0; k < N; ++k) {
    double phi = 0.0;
    for (int i = 0; i < 4; ++i) phi += y[i] * (w[k] * p[4 * k + i]);  // (.. P2)_k
    row.push_back({nb[k], phi});
  }
  return true;
}

// The MLS operator from S to the nodes of T (rows: T nodes, columns: S nodes).
// Returns -1 if some row never reaches rank 4.
int build_mls(const Level& S, const Level& T, double h, int delta, int drop_dirichlet, int scale,
              Csr& R) {
  bool part = !S.owner.empty() && !T.owner.empty();
  if (part) {
    std::set<int> us(S.owner.begin(), S.owner.end()), ut(T.owner.begin(), T.owner.end());
    part = (us == ut);
  }
  std::vector<double> vs, vt;
  if (scale) {
    vs = nodal_volumes(S);
    vt = nodal_volumes(T);
  }
  std::vector<int> all(S.n);
  for (int i = 0; i < S.n; ++i) all[i] = i;
  std::vector<int> ids;
  if (part) {
    std::set<int> u(T.owner.begin(), T.owner.end());
    ids.assign(u.begin(), u.end());
  }
  std::vector<std::vector<int>> sets(ids.size());
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < (int)ids.size(); ++k) sets[k] = overlap_vertices(S, ids[k], delta);
  std::vector<std::vector<std::pair<int, double>>> rows(T.n);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
  for (int t = 0; t < T.n; ++t) {
    if (drop_dirichlet && T.dir[t]) continue;
    const std::vector<int>* cand = &all;
    if (part) cand = &sets[std::lower_bound(ids.begin(), ids.end(), T.owner[t]) - ids.begin()];
    double c = 1.5;
    bool ok = false;
    for (int it = 0; it < 16 && !ok; ++it, c *= 1.5) ok = mls_row(&T.xyz[3 * t], S.xyz, *cand, c * h, rows[t]);
    if (!ok) ++bad;
  }
  if (bad) return -1;
  R.rowptr.assign(T.n + 1, 0);
  R.col.clear();
  R.val.clear();
  for (int t = 0; t < T.n; ++t) {
    for (auto& e : rows[t]) {
      if (drop_dirichlet && S.dir[e.first]) continue;
      R.col.push_back(e.first);
      R.val.push_back(scale ? vt[t] * e.second / vs[e.first] : e.second);
    }
    R.rowptr[t + 1] = (int)R.col.size();
  }
  return 0;
}

// ------------------------------------------------------ V-cycle (Alg. 2)
void residual(const Level& L, const double* r, const double* z, double* t) {
  spmv(L.A, z, t);
  for (int i = 0; i < L.n; ++i) t[i] = r[i] - t[i];
}

// z += B^{-1} (r - A z), `its` times, starting from the given z.
void smooth(const Level& L, const double* r, double* z, int its) {
  std::vector<double> t(L.n), y(L.n);
  for (int s = 0; s < its; ++s) {
    residual(L, r, z, t.data());
    ras_apply(L, t.data(), y.data());
    for (int i = 0; i < L.n; ++i) z[i] += y[i];
  }
}

void vcycle(const Oracle& o, const double* r0, double* z0) {
  int Lc = (int)o.lv.size() - 1;
  std::vector<std::vector<double>> r(o.lv.size()), z(o.lv.size());
  for (int l = 0; l <= Lc; ++l) {
    r[l].assign(o.lv[l].n, 0.0);
    z[l].assign(o.lv[l].n, 0.0);
  }
  std::copy(r0, r0 + o.lv[0].n, r[0].begin());
  for (int l = 0; l < Lc; ++l) {  // down: pre-smooth from z = 0, restrict residual
    const Level& L = o.lv[l];
    smooth(L, r[l].data(), z[l].data(), o.nu_pre);
    std::vector<double> t(L.n);
    residual(L, r[l].data(), z[l].data(), t.data());
    spmv(L.PT, t.data(), r[l + 1].data());
  }
  if (o.coarse_ras) smooth(o.lv[Lc], r[Lc].data(), z[Lc].data(), o.nu_pre);  // from z = 0
  else coarse_solve(o.lv[Lc], r[Lc].data(), z[Lc].data());
  for (int l = Lc - 1; l >= 0; --l) {  // up: prolongate correction, post-smooth
    const Level& L = o.lv[l];
    std::vector<double> pz(L.n);
    spmv(L.P, z[l + 1].data(), pz.data());
    for (int i = 0; i < L.n; ++i) z[l][i] += pz[i];
    smooth(L, r[l].data(), z[l].data(), o.nu_post);
  }
  std::copy(z[0].begin(), z[0].end(), z0);
}

// ------------------------------------------------------------- FGMRES(m)
// Right-preconditioned flexible GMRES with modified Gram-Schmidt and Givens
// rotations; stops when the estimated residual |g_{j+1}| <= rtol ||b||, then
// confirms with the true residual at every restart.
double nrm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double a : v) s += a * a;
  return std::sqrt(s);
}
double dotv(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

int fgmres(const Oracle& o, const double* bptr, double* xptr, double rtol, int m, int maxit,
           int precond, int* iters_out, double* relres_out) {
  const Level& L = o.lv[0];
  int n = L.n;
  std::vector<double> b(bptr, bptr + n), x(n, 0.0), r(n), w(n);
  double bnorm = nrm2(b);
  *iters_out = 0;
  if (bnorm == 0.0) {
    std::copy(x.begin(), x.end(), xptr);
    *relres_out = 0.0;
    return 0;
  }
  int it = 0, status = -3;
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
  r = b;
  double rnorm = bnorm;
  while (true) {
    if (rnorm <= rtol * bnorm) {
      status = 0;
      break;
    }
    if (it >= maxit) break;
    for (int i = 0; i < n; ++i) V[0][i] = r[i] / rnorm;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = rnorm;
    int j = 0;
    bool breakdown = false;
    for (; j < m && it < maxit; ++j) {
      if (precond) vcycle(o, V[j].data(), Z[j].data());
      else Z[j] = V[j];
      spmv(L.A, Z[j].data(), w.data());
      for (int i = 0; i <= j; ++i) {
        double h = dotv(w, V[i]);
        H[(size_t)i * m + j] = h;
        for (int k = 0; k < n; ++k) w[k] -= h * V[i][k];
      }
      double hn = nrm2(w);
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {  // previous rotations
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      double den = std::hypot(a, c);
      cs[j] = (den == 0.0) ? 1.0 : a / den;
      sn[j] = (den == 0.0) ? 0.0 : c / den;
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
      for (int k = 0; k < n; ++k) V[j + 1][k] = w[k] / hn;
      if (std::fabs(g[j + 1]) <= rtol * bnorm) {
        ++j;
        break;
      }
    }
    // y = H(0:j,0:j)^{-1} g(0:j); x += Z y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < j; ++i)
      for (int k = 0; k < n; ++k) x[k] += y[i] * Z[i][k];
    spmv(L.A, x.data(), w.data());
    for (int k = 0; k < n; ++k) r[k] = b[k] - w[k];
    rnorm = nrm2(r);
    if (breakdown && rnorm > rtol * bnorm) break;
  }
  std::copy(x.begin(), x.end(), xptr);
  *iters_out = it;
  *relres_out = rnorm / bnorm;
  return (rnorm <= rtol * bnorm) ? 0 : status;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

typedef struct {
  int n_nodes;
  const double* xyz;
  int n_tets;
  const int* tets;
  const unsigned char* dirichlet;
  const int* owner;  // may be NULL on the coarsest level
} orc_level;

// pde: 0 scalar P1 (one field), 1 linear elasticity (three fields, Poisson
// ratio `poisson` in (0, 0.5), unit Young's modulus scaled by k(x;mu)), 2
// scalar P2 (DoFs on vertices and edges; barycentric transfers, f = 1, and
// delta >= 1 where a level is partitioned), 3 the coupled system of a P2
// field u and a P1 field p, -div(k grad u) + sigma k (u - p) = 1,
// -div(k grad p) + sigma k (p - u) = 1, sigma = `poisson` (> 0).
void* orc_create(const orc_level* lv, int nlevels, int delta, int nu_pre, int nu_post,
                 int coef_kind, const int* wave, double coef_scale, int load_kind, int transfer,
                 int restrict_scaling, int coarse_ras, int ilu_fine, int ilu_coarse, int pde,
                 double poisson) {
  if (nlevels < 1 || transfer < 0 || transfer > 1 || pde < 0 || pde > 3) return nullptr;
  if (pde == 1 && (transfer != 0 || !(poisson > 0.0 && poisson < 0.5))) return nullptr;
  if (pde >= 2 && (transfer != 0 || load_kind != 0 || delta < 1)) return nullptr;
  if (pde == 3 && !(poisson > 0.0)) return nullptr;
  Oracle* o = new Oracle();
  o->p2 = pde >= 2 ? 1 : 0;
  o->twofield = pde == 3 ? 1 : 0;
  if (pde == 3) o->sigma = poisson;  // the coupling coefficient of the two-field system
  if (pde == 1) {
    o->fields = 3;
    o->lame_l = poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson));
    o->lame_m = 1.0 / (2.0 * (1.0 + poisson));
  }
  const int NF = o->fields;
  o->coarse_ras = coarse_ras ? 1 : 0;
  o->transfer = transfer;
  o->restrict_scaling = restrict_scaling ? 1 : 0;
  o->delta = delta;
  o->nu_pre = nu_pre;
  o->nu_post = nu_post;
  o->coef_kind = coef_kind;
  if (wave) std::copy(wave, wave + 24, o->wave);
  o->coef_scale = coef_scale;
  o->load_kind = load_kind;
  o->lv.resize(nlevels);
  for (int l = 0; l < nlevels; ++l) {
    Level& L = o->lv[l];
    L.ilu_fill = (l == 0) ? ilu_fine : ilu_coarse;
    L.nv = lv[l].n_nodes;
    L.n = NF * L.nv;
    L.m = lv[l].n_tets;
    L.xyz.assign(lv[l].xyz, lv[l].xyz + 3 * (size_t)L.nv);
    L.tets.assign(lv[l].tets, lv[l].tets + 4 * (size_t)L.m);
    L.vdir.assign(lv[l].dirichlet, lv[l].dirichlet + L.nv);
    L.dir.resize(L.n);
    for (int i = 0; i < L.n; ++i) L.dir[i] = L.vdir[i / NF];
    if (o->p2) {
      if (!p2_number(L, lv[l].owner, o->twofield != 0)) {
        delete o;
        return nullptr;
      }
      build_pattern_p2(L);
      if (l + 1 < nlevels || o->coarse_ras) {
        if (!lv[l].owner) {
          delete o;
          return nullptr;
        }
        build_subdomains_p2(*o, L);
      } else {
        build_coarse(L);
      }
      continue;
    }
    if (lv[l].owner) {
      L.owner.resize(L.n);
      for (int i = 0; i < L.n; ++i) L.owner[i] = lv[l].owner[i / NF];
    }
    build_pattern(L, NF);
    if (l + 1 < nlevels || o->coarse_ras) {
      if (L.owner.empty()) {
        delete o;
        return nullptr;
      }
      build_subdomains(*o, L);
    } else {
      build_coarse(L);
    }
  }
  for (int l = 0; l + 1 < nlevels; ++l) {
    Level& F = o->lv[l];
    Level& C = o->lv[l + 1];
    if (o->transfer == 1) {
      double h = mesh_h(C);
      if (build_mls(C, F, h, o->delta, 1, 0, F.P) || build_mls(F, C, h, o->delta, 1, o->restrict_scaling, F.PT)) {
        delete o;
        return nullptr;
      }
    } else if (o->p2) {
      build_interp_p2(C, F, F.P);
      transpose(F.P, C.n, F.PT);
    } else {
      Csr Pv;  // the scalar interpolation between the vertex sets
      build_interp(C.nv, C.xyz.data(), C.m, C.tets.data(), C.vdir.data(), F.nv, F.xyz.data(),
                   F.vdir.data(), 1, Pv);
      // one copy per field: P = Pv (x) I_F in the interleaved DoF numbering
      const int nf = o->fields;
      F.P = Csr();
      F.P.rowptr.assign(F.n + 1, 0);
      for (int i = 0; i < F.nv; ++i)
        for (int c = 0; c < nf; ++c) {
          for (int q = Pv.rowptr[i]; q < Pv.rowptr[i + 1]; ++q) {
            F.P.col.push_back(nf * Pv.col[q] + c);
            F.P.val.push_back(Pv.val[q]);
          }
          F.P.rowptr[nf * i + c + 1] = (int)F.P.col.size();
        }
      transpose(F.P, C.n, F.PT);
    }
  }
  return o;
}

void orc_destroy(void* h) { delete static_cast<Oracle*>(h); }

int orc_assemble(void* h, const double* mu) {
  Oracle* o = static_cast<Oracle*>(h);
  o->mu.assign(mu, mu + 8);
  for (auto& L : o->lv)
    if (assemble_level(*o, L)) return -1;
  return 0;
}

int orc_factor(void* h) {
  Oracle* o = static_cast<Oracle*>(h);
  int bad = 0;
  for (size_t l = 0; l < o->lv.size(); ++l) {
    Level& L = o->lv[l];
    if (l + 1 < o->lv.size() || o->coarse_ras) {
      int np = (int)L.subs.size();
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
      for (int p = 0; p < np; ++p) bad += factor_sub(L.A, L.subs[p], L.ilu_fill) ? 1 : 0;
    } else {
      bad += factor_sub(L.A, L.coarse) ? 1 : 0;
    }
  }
  return bad ? -1 : 0;
}

// Factor only the coarsest block.
int orc_factor_coarsest(void* h) {
  Oracle* o = static_cast<Oracle*>(h);
  if (o->coarse_ras) return -1;
  Level& L = o->lv.back();
  return factor_sub(L.A, L.coarse) ? -1 : 0;
}

// Factor only the subdomains [p0, p1) of one level (used to time a sample).
int orc_factor_range(void* h, int level, int p0, int p1) {
  Oracle* o = static_cast<Oracle*>(h);
  Level& L = o->lv[level];
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (int p = p0; p < p1; ++p) bad += factor_sub(L.A, L.subs[p], L.ilu_fill) ? 1 : 0;
  return bad ? -1 : 0;
}

int orc_spmv(void* h, int level, const double* x, double* y) {
  spmv(static_cast<Oracle*>(h)->lv[level].A, x, y);
  return 0;
}
int orc_interp(void* h, int level, const double* xc, double* yf) {  // y_l = P x_{l+1}
  spmv(static_cast<Oracle*>(h)->lv[level].P, xc, yf);
  return 0;
}
int orc_restrict(void* h, int level, const double* yf, double* xc) {  // x_{l+1} = R y_l
  spmv(static_cast<Oracle*>(h)->lv[level].PT, yf, xc);
  return 0;
}
int orc_ras_apply(void* h, int level, const double* r, double* z) {
  ras_apply(static_cast<Oracle*>(h)->lv[level], r, z);
  return 0;
}
// RAS contributions of the subdomains [p0, p1) only: z[owned] = A_p^{-1} r
// (used to time a sample of the subdomain solves).
int orc_ras_apply_range(void* h, int level, int p0, int p1, const double* r, double* z) {
  Oracle* o = static_cast<Oracle*>(h);
  const Level& L = o->lv[level];
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = p0; p < p1; ++p) {
    const Subdomain& S = L.subs[p];
    int n = (int)S.dofs.size();
    std::vector<double> t(n);
    for (int li = 0; li < n; ++li) t[li] = r[S.dofs[li]];
    sub_solve(S, t.data());
    for (int li = 0; li < n; ++li)
      if (S.own[li]) z[S.dofs[li]] = t[li];
  }
  return 0;
}

int orc_coarse_solve(void* h, const double* r, double* z) {
  Oracle* o = static_cast<Oracle*>(h);
  if (o->coarse_ras) return -1;
  coarse_solve(o->lv.back(), r, z);
  return 0;
}
// Solve one subdomain block: y = A_p^{-1} r[V_p] (level `level`, subdomain p;
// p = -1 for the coarsest block).  y has n_p entries.
int orc_sub_solve(void* h, int level, int p, const double* r, double* y) {
  Oracle* o = static_cast<Oracle*>(h);
  const Level& L = o->lv[level];
  const Subdomain& S = (p < 0) ? L.coarse : L.subs[p];
  int n = (int)S.dofs.size();
  if (S.lu.size() != (size_t)n * n && S.ilu.rowptr.empty()) return -1;
  for (int li = 0; li < n; ++li) y[li] = r[S.dofs[li]];
  sub_solve(S, y);
  return 0;
}

int orc_vcycle(void* h, const double* r, double* z) {
  vcycle(*static_cast<Oracle*>(h), r, z);
  return 0;
}
int orc_fgmres(void* h, const double* b, double* x, double rtol, int restart, int maxit,
               int precond, int* iters, double* relres) {
  return fgmres(*static_cast<Oracle*>(h), b, x, rtol, restart, maxit, precond, iters, relres);
}

// Accessors into the oracle's state; they return the element count and set *ptr.
long orc_get(void* h, const char* what, int level, int sub, const void** ptr) {
  Oracle* o = static_cast<Oracle*>(h);
  if (level < 0 || level >= (int)o->lv.size()) return -1;
  Level& L = o->lv[level];
  std::string w(what);
  auto ret = [&](const auto& v) {
    *ptr = v.data();
    return (long)v.size();
  };
  if (w == "rowptr") return ret(L.A.rowptr);
  if (w == "col") return ret(L.A.col);
  if (w == "val") return ret(L.A.val);
  if (w == "b") return ret(L.b);
  if (w == "P_rowptr") return ret(L.P.rowptr);
  if (w == "P_col") return ret(L.P.col);
  if (w == "P_val") return ret(L.P.val);
  if (w == "PT_rowptr") return ret(L.PT.rowptr);
  if (w == "PT_col") return ret(L.PT.col);
  if (w == "PT_val") return ret(L.PT.val);
  if (w == "dofdir") return ret(L.dir);
  if (w == "pdof") return ret(L.pdof);
  if (w == "dofx") return ret(L.dofx);
  if (w == "n_subs") {
    *ptr = nullptr;
    return (long)L.subs.size();
  }
  const Subdomain* S = nullptr;
  if (sub < 0) S = &L.coarse;
  else if (sub < (int)L.subs.size()) S = &L.subs[sub];
  if (!S) return -1;
  if (w == "sub_ilu_ptr") return ret(S->ilu.rowptr);
  if (w == "sub_ilu_col") return ret(S->ilu.col);
  if (w == "sub_ilu_val") return ret(S->ilu.val);
  if (w == "sub_dofs") return ret(S->dofs);
  if (w == "sub_own") return ret(S->own);
  if (w == "sub_lu") return ret(S->lu);
  return -1;
}

// DoFs of a level.
int orc_ndofs(void* h, int level) {
  Oracle* o = static_cast<Oracle*>(h);
  if (level < 0 || level >= (int)o->lv.size()) return -1;
  return o->lv[level].n;
}

// ---- standalone pieces used by the pins ----
// The P2 element of a tet (local DoFs: vertices 0..3, edges 01 02 03 12 13 23):
// K100 row-major = k int grad phi_i . grad phi_j, m10 = int phi_i; returns |T|.
// The coupled two-field element (P2 u, P1 p): K196 row-major 14 x 14 times k,
// m14 = int of the 14 basis functions; returns |T|.
double orc_tet_p2p1(const double* x4, double k, double sigma, double* K196, double* m14) {
  double g[4][3];
  double det = tet_gradients(&x4[0], &x4[3], &x4[6], &x4[9], g);
  double vol = std::fabs(det) / 6.0;
  coupled_element(g, vol, sigma, K196, m14);
  for (int i = 0; i < 196; ++i) K196[i] *= k;
  return vol;
}

double orc_tet_p2(const double* x4, double k, double* K100, double* m10) {
  double g[4][3];
  double det = tet_gradients(&x4[0], &x4[3], &x4[6], &x4[9], g);
  double vol = std::fabs(det) / 6.0;
  p2_element(g, vol, K100, m10);
  for (int i = 0; i < 100; ++i) K100[i] *= k;
  return vol;
}

double orc_tet_stiffness(const double* x4, double k, double* K16) {
  double g[4][3];
  double det = tet_gradients(&x4[0], &x4[3], &x4[6], &x4[9], g);
  double vol = std::fabs(det) / 6.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) K16[4 * a + b] = k * vol * dot3(g[a], g[b]);
  return vol;
}

// Element stiffness of linear elasticity (12 x 12, row-major, row 3a+i,
// column 3b+j) for Lame parameters lam, mu and coefficient k; returns |T|.
double orc_tet_elasticity(const double* x4, double k, double lam, double mu, double* K144) {
  double g[4][3];
  double det = tet_gradients(&x4[0], &x4[3], &x4[6], &x4[9], g);
  double vol = std::fabs(det) / 6.0;
  elastic_element(g, vol, lam, mu, K144);
  for (int e = 0; e < 144; ++e) K144[e] *= k;
  return vol;
}

int orc_lu_factor(int n, double* A) { return lu_factor(n, A); }
void orc_lu_solve(int n, const double* LU, double* x) { lu_solve(n, LU, x); }

// Interpolation between two arbitrary meshes (returns nnz; arrays are
// allocated by the oracle and freed with orc_free_csr).
long orc_build_interp(int nc, const double* cxyz, int mc, const int* ctets, const unsigned char* cdir,
                      int nf, const double* fxyz, const unsigned char* fdir, int drop_dirichlet,
                      int** rowptr, int** col, double** val) {
  Csr P;
  build_interp(nc, cxyz, mc, ctets, cdir, nf, fxyz, fdir, drop_dirichlet, P);
  *rowptr = new int[P.rowptr.size()];
  *col = new int[P.col.size() + 1];
  *val = new double[P.val.size() + 1];
  std::copy(P.rowptr.begin(), P.rowptr.end(), *rowptr);
  std::copy(P.col.begin(), P.col.end(), *col);
  std::copy(P.val.begin(), P.val.end(), *val);
  return (long)P.col.size();
}
// MLS operator from mesh S to the nodes of mesh T (see build_mls).  owner may
// be NULL on either mesh (no partition).  h <= 0 takes h from the coarser
// (fewer tets) of the two.  Returns nnz, or -1 if a row never reaches rank 4.
long orc_build_mls(const orc_level* src, const orc_level* dst, double h, int delta, int drop_dirichlet,
                   int scale, int** rowptr, int** col, double** val) {
  Level M[2];
  const orc_level* d[2] = {src, dst};
  for (int k = 0; k < 2; ++k) {
    M[k].n = M[k].nv = d[k]->n_nodes;
    M[k].m = d[k]->n_tets;
    M[k].xyz.assign(d[k]->xyz, d[k]->xyz + 3 * (size_t)M[k].n);
    M[k].tets.assign(d[k]->tets, d[k]->tets + 4 * (size_t)M[k].m);
    M[k].dir.assign(d[k]->dirichlet, d[k]->dirichlet + M[k].n);
    M[k].vdir = M[k].dir;
    if (d[k]->owner) M[k].owner.assign(d[k]->owner, d[k]->owner + M[k].n);
    build_pattern(M[k], 1);
  }
  if (!(h > 0)) h = mesh_h(M[0].m <= M[1].m ? M[0] : M[1]);
  Csr R;
  if (build_mls(M[0], M[1], h, delta, drop_dirichlet, scale, R)) return -1;
  *rowptr = new int[R.rowptr.size()];
  *col = new int[R.col.size() + 1];
  *val = new double[R.val.size() + 1];
  std::copy(R.rowptr.begin(), R.rowptr.end(), *rowptr);
  std::copy(R.col.begin(), R.col.end(), *col);
  std::copy(R.val.begin(), R.val.end(), *val);
  return (long)R.col.size();
}

// ILU(p) of an n x n CSR matrix (sorted columns): returns the nnz of the
// factor (unit L below the diagonal, U on and above it, one CSR), -1 on a
// zero pivot.  Arrays are freed with orc_free_csr.
long orc_ilu_factor(int n, const int* rowptr, const int* col, const double* val, int p, int** fptr,
                    int** fcol, double** fval) {
  Csr B, F;
  B.rowptr.assign(rowptr, rowptr + n + 1);
  B.col.assign(col, col + rowptr[n]);
  B.val.assign(val, val + rowptr[n]);
  ilu_symbolic(B, p, F);
  std::vector<int> ud;
  if (ilu_numeric(B, F, ud)) return -1;
  *fptr = new int[F.rowptr.size()];
  *fcol = new int[F.col.size() + 1];
  *fval = new double[F.val.size() + 1];
  std::copy(F.rowptr.begin(), F.rowptr.end(), *fptr);
  std::copy(F.col.begin(), F.col.end(), *fcol);
  std::copy(F.val.begin(), F.val.end(), *fval);
  return (long)F.col.size();
}

double orc_mesh_h(const orc_level* c) {
  Level L;
  L.n = c->n_nodes;
  L.m = c->n_tets;
  L.xyz.assign(c->xyz, c->xyz + 3 * (size_t)L.n);
  return mesh_h(L);
}

void orc_free_csr(int* rowptr, int* col, double* val) {
  delete[] rowptr;
  delete[] col;
  delete[] val;
}

}  // extern "C"
