"""Pins for the oracle's quadratic (P2) elements: DoFs on the vertices and on
the edge midpoints, the DoF distribution N = (1,1,0,0) of the mesh perspective
(Section 2.1), and the P2 transfer between non-nested levels.

* The element matrix against exact rational integration (sympy) of the P2
  Lagrange basis on a tet with rational vertices, the basis itself by its
  nodal property.
* The DoF numbering and the Dirichlet edges against an independent numpy
  construction and the lattice geometry of the synthetic meshes.
* The assembled operator by the patch test: for a quadratic u with constant
  Laplacian and k = 1, rows away from the boundary satisfy
  (J u_I)_i = -lap(u) int phi_i exactly.
* The transfer by exact reproduction of quadratic fields.
* Subdomains: partition of unity and the stated overlap rule; RAS with one
  subdomain is the exact inverse; FGMRES against a direct solve.
CPU only.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as syn
from _common import make_oracle, workload

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def test_p2_element_against_exact_integration(orc):
    sp = pytest.importorskip("sympy")
    X = [sp.Matrix([0, 0, 0]), sp.Matrix([sp.Rational(3, 2), sp.Rational(1, 5), 0]),
         sp.Matrix([sp.Rational(1, 3), sp.Rational(5, 4), sp.Rational(1, 7)]),
         sp.Matrix([sp.Rational(-1, 4), sp.Rational(1, 3), sp.Rational(6, 5)])]
    x, y, z = sp.symbols("x y z")
    # barycentric coordinates: the affine functions equal to 1 at one vertex, 0 at the others
    M = sp.Matrix([[1, *X[a]] for a in range(4)])
    coef = M.inv()  # column a: coefficients of lambda_a in (1, x, y, z)
    lam = [coef[0, a] + coef[1, a] * x + coef[2, a] * y + coef[3, a] * z for a in range(4)]
    phi = [lam[a] * (2 * lam[a] - 1) for a in range(4)] + [4 * lam[a] * lam[b] for a, b in EDGES]
    # the nodal (Lagrange) property at the vertices and edge midpoints
    nodes = list(X) + [(X[a] + X[b]) / 2 for a, b in EDGES]
    for i, f in enumerate(phi):
        for j, p in enumerate(nodes):
            assert f.subs({x: p[0], y: p[1], z: p[2]}) == (1 if i == j else 0)
    # exact integrals over the tet through the reference tet map
    s, t, u = sp.symbols("s t u")
    J = sp.Matrix.hstack(X[1] - X[0], X[2] - X[0], X[3] - X[0])
    detJ = abs(J.det())
    mp = X[0] + J * sp.Matrix([s, t, u])

    def integrate(expr):
        e = sp.expand(expr.subs({x: mp[0], y: mp[1], z: mp[2]}))
        return detJ * sp.integrate(e, (u, 0, 1 - s - t), (t, 0, 1 - s), (s, 0, 1))

    grads = [[sp.diff(f, v) for v in (x, y, z)] for f in phi]
    K_exact = np.zeros((10, 10))
    for i in range(10):
        for j in range(i, 10):
            val = integrate(sum(grads[i][d] * grads[j][d] for d in range(3)))
            K_exact[i, j] = K_exact[j, i] = float(val)
    m_exact = np.array([float(integrate(f)) for f in phi])
    x4 = np.array([[float(c) for c in p] for p in X])
    K, m, vol = orc.tet_p2(x4, k=2.5)
    assert abs(vol - float(detJ) / 6) <= 1e-15
    assert np.max(np.abs(K - 2.5 * K_exact)) <= 1e-13 * np.max(np.abs(K))
    assert np.max(np.abs(m - m_exact)) <= 1e-15


def _edges_of(levels_lv):
    t = levels_lv.tets
    E = np.concatenate([np.sort(t[:, [a, b]], axis=1) for a, b in EDGES])
    return np.unique(E, axis=0)


def test_p2_numbering_points_and_dirichlet_edges(orc):
    levels, w = workload("p2cube6_3lvl")
    o = make_oracle(levels, w, orc)
    for l, lv in enumerate(levels):
        E = _edges_of(lv)
        nv = lv.n_nodes
        assert o.n[l] == nv + len(E) == (2 * lv.n + 1) ** 3
        # vertex v, then its edges (v, b) in ascending b
        order = sorted([(v, -1) for v in range(nv)] + [(int(a), int(b)) for a, b in E])
        pts = np.array([lv.xyz[v] if b < 0 else 0.5 * (lv.xyz[v] + lv.xyz[b]) for v, b in order])
        np.testing.assert_array_equal(o.get("dofx", l).reshape(-1, 3), pts)
        # Dirichlet: vertices as given; an edge when its midpoint lies on the boundary of the
        # lattice cube (both ends on one face), from the lattice coordinates
        lat = lv.lattice
        d = []
        for v, b in order:
            if b < 0:
                d.append(lv.dirichlet[v])
            else:
                on = np.any(((lat[v] == 0) & (lat[b] == 0)) | ((lat[v] == lv.n) & (lat[b] == lv.n)))
                d.append(1 if on else 0)
        np.testing.assert_array_equal(o.get("dofdir", l), np.array(d, np.uint8))


def test_p2_patch_test(orc):
    levels, w = workload("p2cube6_3lvl")
    w = dict(w, coef="const")
    o = make_oracle(levels, w, orc)
    o.assemble(np.zeros(8))
    A = o.csr(0).tocsr()
    b = o.get("b", 0)
    X = o.get("dofx", 0).reshape(-1, 3)
    dirv = o.get("dofdir", 0)
    # u = x^2 + 2 y^2 - z^2 + xy - yz + 3 x - 1: lap u = 2 + 4 - 2 = 4
    u = X[:, 0] ** 2 + 2 * X[:, 1] ** 2 - X[:, 2] ** 2 + X[:, 0] * X[:, 1] - X[:, 1] * X[:, 2] + 3 * X[:, 0] - 1
    Au = A @ u
    away = np.array([not dirv[i] and not np.any(dirv[A.indices[A.indptr[i]:A.indptr[i + 1]]])
                     for i in range(A.shape[0])])
    assert away.sum() > 100
    assert np.max(np.abs(Au[away] - (-4.0) * b[away])) <= 1e-12 * np.max(np.abs(Au[away]))
    # symmetric, and constants are in the kernel of the unconstrained rows
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    assert np.max(np.abs((A @ np.ones(A.shape[0]))[away])) <= 1e-13 * abs(A).max()


def test_p2_transfer_reproduces_quadratics(orc):
    levels, w = workload("p2cube6_3lvl")
    # a coarse level without Dirichlet nodes: no column is dropped from P
    coarse = levels[1]
    levels = [levels[0], syn.Level(n=coarse.n, xyz=coarse.xyz, tets=coarse.tets,
                                   dirichlet=np.zeros_like(coarse.dirichlet), owner=coarse.owner,
                                   lattice=coarse.lattice), levels[2]]
    o = make_oracle(levels, w, orc)
    P = o.csr(0, "P")
    Xf = o.get("dofx", 0).reshape(-1, 3)
    Xc = o.get("dofx", 1).reshape(-1, 3)
    dirf = o.get("dofdir", 0)

    def q(X):
        return 1 + X[:, 0] - 2 * X[:, 1] + 0.5 * X[:, 2] + X[:, 0] ** 2 - X[:, 1] * X[:, 2] + 3 * X[:, 2] ** 2

    y = P @ q(Xc)
    fine = dirf == 0
    assert np.max(np.abs(y[fine] - q(Xf)[fine])) <= 1e-12
    assert np.all(np.diff(P.indptr)[~fine] == 0)  # Dirichlet fine DoFs have empty rows
    PT = o.csr(0, "PT")
    assert abs(PT - P.T).max() == 0


def test_p2_subdomains(orc):
    levels, w = workload("p2cube6_3lvl")
    o = make_oracle(levels, w, orc)
    lv = levels[0]
    dirv = o.get("dofdir", 0)
    X = o.get("dofx", 0).reshape(-1, 3)
    owned = np.zeros(o.n[0], int)
    subs = o.subdomains(0)
    assert len(subs) == 8
    # vertex DoF of every vertex, edge DoF of every edge, by their points
    key = {tuple(p): i for i, p in enumerate(X)}
    vd = np.array([key[tuple(p)] for p in lv.xyz])
    E = _edges_of(lv)
    ed = np.array([key[tuple(0.5 * (lv.xyz[a] + lv.xyz[b]))] for a, b in E])
    ids = sorted(set(lv.owner[lv.dirichlet == 0]))
    for p, (dofs, own) in enumerate(subs):
        owned[dofs[own == 1]] += 1
        # the stated rule: delta = 1 vertex layer, then vertices + edges with both ends inside
        inside = lv.owner == ids[p]
        grow = inside.copy()
        for t in lv.tets:
            if inside[t].any():
                grow[t] = True
        want = set(vd[grow]) | set(ed[grow[E[:, 0]] & grow[E[:, 1]]])
        want = sorted(i for i in want if not dirv[i])
        np.testing.assert_array_equal(dofs, want)
    assert np.all(owned[dirv == 0] == 1) and np.all(owned[dirv == 1] == 0)


def test_p2_solves(orc):
    levels, w = workload("p2cube6_3lvl")
    mu = syn.mu_draw(3)
    # one subdomain with the whole level: RAS = the exact inverse
    one = [syn.Level(n=lv.n, xyz=lv.xyz, tets=lv.tets, dirichlet=lv.dirichlet,
                     owner=np.zeros_like(lv.owner) if lv.owner is not None else None, lattice=lv.lattice)
           for lv in levels]
    o1 = make_oracle(one, w, orc)
    o1.assemble(mu)
    o1.factor()
    A = o1.csr(0).tocsc()
    r = np.random.default_rng(2).normal(size=o1.n[0])
    z = o1.ras_apply(r, 0)
    assert np.linalg.norm(A @ z - r) <= 1e-11 * np.linalg.norm(r)
    # FGMRES with the three-level V-cycle against a direct solve
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    x, st = o.fgmres(rtol=1e-11)
    A = o.csr(0).tocsc()
    xd = spla.spsolve(A, o.get("b", 0))
    assert st["status"] == 0 and st["iters"] <= 8
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


# ---------------------------------------------------------------------------
# The coupled two-field system: a P2 field u and a P1 field p (DoFs of u on
# the vertices and edges, of p on the vertices), -div(k grad u) + s k (u - p)
# = 1, -div(k grad p) + s k (p - u) = 1; the transfers split by field (the
# P2 interpolation for u, the P1 one for p).

def test_p2p1_element_against_exact_integration(orc):
    sp = pytest.importorskip("sympy")
    X = [sp.Matrix([0, 0, 0]), sp.Matrix([sp.Rational(5, 4), sp.Rational(1, 3), 0]),
         sp.Matrix([sp.Rational(1, 5), sp.Rational(4, 3), sp.Rational(1, 6)]),
         sp.Matrix([sp.Rational(-1, 3), sp.Rational(1, 4), sp.Rational(7, 5)])]
    x, y, z = sp.symbols("x y z")
    M = sp.Matrix([[1, *X[a]] for a in range(4)])
    coef = M.inv()
    lam = [coef[0, a] + coef[1, a] * x + coef[2, a] * y + coef[3, a] * z for a in range(4)]
    phi = [lam[a] * (2 * lam[a] - 1) for a in range(4)] + [4 * lam[a] * lam[b] for a, b in EDGES] + lam
    s_, t_, u_ = sp.symbols("s t u")
    J = sp.Matrix.hstack(X[1] - X[0], X[2] - X[0], X[3] - X[0])
    detJ = abs(J.det())
    mp = X[0] + J * sp.Matrix([s_, t_, u_])

    def integrate(expr):
        e = sp.expand(expr.subs({x: mp[0], y: mp[1], z: mp[2]}))
        return detJ * sp.integrate(e, (u_, 0, 1 - s_ - t_), (t_, 0, 1 - s_), (s_, 0, 1))

    sigma, k = sp.Rational(7, 10), 1.3
    grads = [[sp.diff(f, v) for v in (x, y, z)] for f in phi]
    K_exact = np.zeros((14, 14))
    for i in range(14):
        for j in range(i, 14):
            mass = integrate(phi[i] * phi[j])
            if (i < 10) == (j < 10):
                val = integrate(sum(grads[i][d] * grads[j][d] for d in range(3))) + sigma * mass
            else:
                val = -sigma * mass
            K_exact[i, j] = K_exact[j, i] = float(val)
    m_exact = np.array([float(integrate(f)) for f in phi])
    x4 = np.array([[float(c) for c in p] for p in X])
    K, m, vol = orc.tet_p2p1(x4, k=k, sigma=0.7)
    assert np.max(np.abs(K - k * K_exact)) <= 1e-13 * np.max(np.abs(K))
    assert np.max(np.abs(m - m_exact)) <= 1e-15
    # positive semi-definite with one zero mode: u = p = constant (no gradient, no coupling)
    ev = np.linalg.eigvalsh(K)
    assert ev[0] >= -1e-14 * ev[-1] and abs(ev[0]) <= 1e-14 * ev[-1] and ev[1] > 1e-3 * ev[-1]
    assert np.max(np.abs(K @ np.ones(14))) <= 1e-14 * ev[-1]


def _p2p1(orc, name="p2p1cube6_3lvl", **kw):
    levels, w = workload(name)
    return levels, w, make_oracle(levels, w, orc, **kw)


def test_p2p1_numbering_and_equal_fields(orc):
    """DoFs: every vertex's u, then its p, then its edges' u; u = p = an affine
    field makes the coupling vanish, so rows away from the boundary of J x are
    zero (k = 1)."""
    levels, w, o = _p2p1(orc, coef="const")
    lv = levels[0]
    E = _edges_of(lv)
    assert o.n[0] == 2 * lv.n_nodes + len(E)
    pd = o.get("pdof", 0)
    X = o.get("dofx", 0).reshape(-1, 3)
    order = sorted([(v, -2) for v in range(lv.n_nodes)] + [(v, -1) for v in range(lv.n_nodes)] +
                   [(int(a), int(b)) for a, b in E])
    np.testing.assert_array_equal(pd, np.array([1 if b == -1 else 0 for _, b in order], np.uint8))
    o.assemble(np.zeros(8))
    A = o.csr(0).tocsr()
    dirv = o.get("dofdir", 0)
    aff = 0.3 + X[:, 0] - 2 * X[:, 1] + 0.7 * X[:, 2]
    Ax = A @ aff
    away = np.array([not dirv[i] and not np.any(dirv[A.indices[A.indptr[i]:A.indptr[i + 1]]])
                     for i in range(A.shape[0])])
    assert away.sum() > 50
    assert np.max(np.abs(Ax[away])) <= 1e-13 * abs(A).max()
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()


def test_p2p1_transfer_splits_by_field(orc):
    levels, w = workload("p2p1cube6_3lvl")
    coarse = levels[1]
    levels = [levels[0], syn.Level(n=coarse.n, xyz=coarse.xyz, tets=coarse.tets,
                                   dirichlet=np.zeros_like(coarse.dirichlet), owner=coarse.owner,
                                   lattice=coarse.lattice), levels[2]]
    o = make_oracle(levels, w, orc)
    P = o.csr(0, "P").tocsr()
    Xf, Xc = o.get("dofx", 0).reshape(-1, 3), o.get("dofx", 1).reshape(-1, 3)
    pf, pc = o.get("pdof", 0).astype(bool), o.get("pdof", 1).astype(bool)
    dirf = o.get("dofdir", 0)
    # rows of u only reference coarse u DoFs, rows of p only coarse p DoFs
    for f in range(P.shape[0]):
        cols = P.indices[P.indptr[f]:P.indptr[f + 1]]
        assert np.all(pc[cols] == pf[f])
    # u reproduces quadratics (P2), p reproduces affine fields (P1) exactly
    q = 1 + Xc[:, 0] - Xc[:, 1] * Xc[:, 2] + 2 * Xc[:, 2] ** 2
    a = 0.5 - Xc[:, 0] + 3 * Xc[:, 1] + Xc[:, 2]
    xc = np.where(pc, a, q)
    y = P @ xc
    qf = 1 + Xf[:, 0] - Xf[:, 1] * Xf[:, 2] + 2 * Xf[:, 2] ** 2
    af = 0.5 - Xf[:, 0] + 3 * Xf[:, 1] + Xf[:, 2]
    want = np.where(pf, af, qf)
    fine = dirf == 0
    assert np.max(np.abs(y[fine] - want[fine])) <= 1e-12


def test_p2p1_subdomains_and_solve(orc):
    levels, w, o = _p2p1(orc)
    dirv = o.get("dofdir", 0)
    owned = np.zeros(o.n[0], int)
    for dofs, own in o.subdomains(0):
        owned[dofs[own == 1]] += 1
    assert np.all(owned[dirv == 0] == 1) and np.all(owned[dirv == 1] == 0)
    o.assemble(syn.mu_draw(4))
    o.factor()
    x, st = o.fgmres(rtol=1e-11)
    xd = spla.spsolve(o.csr(0).tocsc(), o.get("b", 0))
    assert st["status"] == 0 and st["iters"] <= 8
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
