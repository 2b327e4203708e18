"""Pins for the FP64 oracle: each checks it against something other than itself.

The oracle restates the method of arXiv 2412.08981 (Sections 2.1-2.3 and
Algorithm 2, with the P / P^T transfer and coarsest direct solve readings).
These tests pin it to closed forms, invariants, special cases that reduce to a
library routine, and brute force on tiny meshes.  CPU only.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla
from scipy.spatial import ConvexHull

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ----------------------------------------------------------------- helpers
def pattern_numpy(tets, n):
    """Independent CSR pattern: all vertex pairs that share a tet."""
    a = np.repeat(tets, 4, axis=1).ravel()
    b = np.tile(tets, (1, 4)).ravel()
    M = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def mk_oracle(orc, levels, **kw):
    o = orc.Oracle(levels, **kw)
    return o


def random_tet(rng):
    while True:
        x = rng.normal(size=(4, 3))
        if abs(np.linalg.det(x[1:] - x[0])) > 0.2:
            return x


# ------------------------------------------------------- element stiffness
def test_reference_tet_closed_form(orc):
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    K, vol = orc.tet_stiffness(x)
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    np.testing.assert_allclose(K, ref, atol=1e-15)
    assert vol == pytest.approx(1.0 / 6.0, abs=1e-16)
    # scaling by h multiplies the 3-D stiffness by h; rigid motions leave it unchanged
    Q, _ = np.linalg.qr(np.random.default_rng(0).normal(size=(3, 3)))
    for h in (0.5, 3.0):
        Kh, _ = orc.tet_stiffness(h * x @ Q.T + np.array([0.3, -2.0, 1.0]), k=2.5)
        np.testing.assert_allclose(Kh, 2.5 * h * ref, atol=1e-13)
    # vertex order reversal (negative orientation) gives the permuted matrix
    perm = [0, 2, 1, 3]
    Kp, _ = orc.tet_stiffness(x[perm])
    np.testing.assert_allclose(Kp, ref[np.ix_(perm, perm)], atol=1e-15)


def test_element_patch_and_energy(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = random_tet(rng)
        k = float(rng.uniform(0.1, 10))
        K, vol = orc.tet_stiffness(x, k)
        assert vol == pytest.approx(ConvexHull(x).volume, rel=1e-12)
        np.testing.assert_allclose(K, K.T, atol=1e-14 * abs(K).max())
        np.testing.assert_allclose(K @ np.ones(4), 0, atol=1e-13 * abs(K).max())
        g = rng.normal(size=3)
        u = x @ g + 0.7
        # energy of an affine field: k |T| |grad u|^2
        assert u @ K @ u == pytest.approx(k * vol * g @ g, rel=1e-11)
        assert np.linalg.matrix_rank(K, tol=1e-10 * abs(K).max()) == 3


# ------------------------------------------------------ pattern, assembly
@pytest.mark.parametrize("n", [3, 6])
def test_csr_pattern_independent(orc, n):
    lv = syn.cube_level(n, 11)
    o = mk_oracle(orc, [lv])
    M = pattern_numpy(lv.tets, lv.n_nodes)
    np.testing.assert_array_equal(o.get("rowptr"), M.indptr)
    np.testing.assert_array_equal(o.get("col"), M.indices)


def interior_rows_away_from_dirichlet(lv, A):
    dirn = lv.dirichlet.astype(bool)
    M = pattern_numpy(lv.tets, lv.n_nodes)
    touch = (M @ dirn.astype(float)) > 0
    return np.where(~dirn & ~touch)[0]


@pytest.mark.parametrize("coef", ["const", "cosexp"])
def test_assembly_symmetry_rowsum_patch(orc, coef):
    lv = syn.cube_level(8, 21)
    o = mk_oracle(orc, [lv], coef=coef, wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(3))
    A = o.csr(0)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    rows = interior_rows_away_from_dirichlet(lv, A)
    assert rows.size > 0
    one = np.ones(lv.n_nodes)
    np.testing.assert_allclose((A @ one)[rows], 0, atol=1e-13 * abs(A).max())
    if coef == "const":  # patch test: affine fields are discrete-harmonic for constant k
        g = np.array([0.3, -1.2, 2.0])
        aff = lv.xyz @ g + 0.5
        np.testing.assert_allclose((A @ aff)[rows], 0, atol=1e-12 * abs(A).max())
    # Dirichlet rows are identity rows, Dirichlet columns are zero elsewhere
    d = np.where(lv.dirichlet)[0]
    Ad = A[d].toarray()
    np.testing.assert_array_equal(Ad, np.eye(lv.n_nodes)[d])
    nd = np.where(lv.dirichlet == 0)[0]
    assert abs(A[nd][:, d]).max() == 0.0
    # SPD on the interior
    Aii = A[nd][:, nd].toarray()
    assert np.linalg.eigvalsh(Aii).min() > 0


def test_unjittered_grid_is_7_point_stencil(orc):
    n = 6
    lv = syn.cube_level(n, 5, jitter=0.0)
    o = mk_oracle(orc, [lv])
    o.assemble()
    A = o.csr(0).tocsr()
    h = 1.0 / n
    lat = lv.lattice
    N = n + 1
    for i in np.where(np.all((lat >= 2) & (lat <= n - 2), axis=1))[0]:
        row = A.getrow(i)
        entries = dict(zip(row.indices, row.data))
        assert entries[i] == pytest.approx(6 * h, rel=1e-13)
        for d, s in itertools.product(range(3), (-1, 1)):
            off = [0, 0, 0]
            off[d] = s
            j = i + off[0] + N * (off[1] + N * off[2])
            assert entries[j] == pytest.approx(-h, rel=1e-13)
        others = [v for j, v in entries.items()
                  if j != i and abs(j - i) not in (1, N, N * N)]
        assert max(abs(v) for v in others) < 1e-15


def _gauss_integral_of_k(wave, mu, npts=24):
    xg, wg = np.polynomial.legendre.leggauss(npts)
    xg = 0.5 * (xg + 1)
    wg = 0.5 * wg
    X, Y, Z = np.meshgrid(xg, xg, xg, indexing="ij")
    W = wg[:, None, None] * wg[None, :, None] * wg[None, None, :]
    s = np.zeros_like(X)
    for j in range(8):
        s += mu[j] * 0.5 * np.cos(np.pi * (wave[j, 0] * X + wave[j, 1] * Y + wave[j, 2] * Z))
    return float((np.exp(s) * W).sum())


def test_coefficient_energy_matches_quadrature(orc):
    """u^T A u of an affine u on a Neumann mesh = |g|^2 * int k, up to O(h^2)."""
    wave = syn.wave_vectors()
    mu = syn.mu_draw(5)
    exact = _gauss_integral_of_k(wave, mu)
    g = np.array([1.0, -0.5, 0.25])
    errs = []
    for n in (8, 16, 32):
        lv = syn.cube_level(n, 77, jitter=0.0)  # uniform: the centroid-rule error is O(h^2)
        lv.dirichlet = np.zeros_like(lv.dirichlet)  # pure Neumann operator
        o = mk_oracle(orc, [lv], coef="cosexp", wave=wave)
        o.assemble(mu)
        A = o.csr(0)
        u = lv.xyz @ g
        errs.append(abs(u @ (A @ u) / (g @ g) - exact) / exact)
    assert errs[-1] < 2e-3, errs
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5  # ~4 per halving


def test_manufactured_solution_converges_h2(orc):
    """P1 Poisson, k = 1, u = sin sin sin: L2 error O(h^2) (direct solve)."""
    errs, hs = [], []
    for n in (8, 16, 32):
        lv = syn.cube_level(n, 1000 + n)
        o = mk_oracle(orc, [lv], load="sines")
        o.assemble()
        A = o.csr(0).tocsc()
        b = o.get("b")
        u = spla.spsolve(A, b)
        ue = np.prod(np.sin(np.pi * lv.xyz), axis=1)
        # lumped mass from an independent volume computation
        x = lv.xyz[lv.tets]
        vol = np.abs(np.linalg.det(x[:, 1:] - x[:, :1])) / 6.0
        m = np.bincount(lv.tets.ravel(), weights=np.repeat(vol / 4, 4), minlength=lv.n_nodes)
        errs.append(np.sqrt(np.sum(m * (u - ue) ** 2)))
        hs.append(1.0 / n)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - 2.0) <= 0.2, (slope, errs)
    assert np.allclose(spla.spsolve(A, b)[lv.dirichlet == 1], 0)


# --------------------------------------------------------------- subdomains
@pytest.mark.parametrize("delta,parts", [(1, (2, 2, 2)), (2, (3, 2, 2)), (2, (4, 4, 4))])
def test_partition_of_unity_and_overlap(orc, delta, parts):
    n = 8
    lv = syn.cube_level(n, 31, parts=parts)
    coarse = syn.cube_level(4, 32)
    o = mk_oracle(orc, [lv, coarse], delta=delta)
    subs = o.subdomains(0)
    dirn = lv.dirichlet.astype(bool)
    ids = sorted(set(lv.owner[~dirn].tolist()))
    assert len(subs) == len(ids)
    count = np.zeros(lv.n_nodes, int)
    G = pattern_numpy(lv.tets, lv.n_nodes)
    G.setdiag(0)
    G.eliminate_zeros()
    for (dofs, own), sid in zip(subs, ids):
        assert np.all(np.diff(dofs) > 0)
        assert not dirn[dofs].any()
        count[dofs[own == 1]] += 1
        np.testing.assert_array_equal(own, (lv.owner[dofs] == sid).astype(np.uint8))
        src = np.where(lv.owner == sid)[0]
        dist = csg.shortest_path(G, unweighted=True, indices=src, directed=False).min(axis=0)
        expect = np.where((dist <= delta) & ~dirn)[0]
        np.testing.assert_array_equal(dofs, expect)
    np.testing.assert_array_equal(count, (~dirn).astype(int))  # R0 sum = I off Dirichlet


# ----------------------------------------------------------------------- LU
def test_lu_reconstructs_and_solves(orc):
    rng = np.random.default_rng(2)
    for n in (1, 5, 64, 131):
        B = rng.normal(size=(n, n))
        A = B @ B.T + n * np.eye(n)
        LU = orc.lu_factor(A)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        assert np.linalg.norm(L @ U - A) / np.linalg.norm(A) <= 1e-14
        b = rng.normal(size=n)
        np.testing.assert_allclose(orc.lu_solve(LU, b), sla.solve(A, b), rtol=1e-12, atol=1e-14)
    with pytest.raises(ValueError):
        orc.lu_factor(np.zeros((3, 3)))


# ---------------------------------------------------------------------- RAS
def _two_level(n=6, nc=3, parts=(2, 2, 2), delta=1, seed=40):
    lv = syn.cube_level(n, seed, parts=parts)
    return lv, syn.cube_level(nc, seed + 1)


def test_ras_single_subdomain_is_exact(orc):
    lv, co = _two_level()
    lv.owner = np.zeros_like(lv.owner)
    o = mk_oracle(orc, [lv, co], delta=1, coef="cosexp", wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(1))
    o.factor()
    A = o.csr(0).tocsc()
    r = np.random.default_rng(3).normal(size=lv.n_nodes)
    np.testing.assert_allclose(o.ras_apply(r), spla.spsolve(A, r), rtol=1e-11, atol=1e-13)
    # the whole V-cycle then equals A^{-1}, and FGMRES needs one iteration
    np.testing.assert_allclose(o.vcycle(r), spla.spsolve(A, r), rtol=1e-10, atol=1e-12)
    x, st = o.fgmres(rtol=1e-10)
    assert st["status"] == 0 and st["iters"] == 1


def test_ras_full_overlap_is_exact(orc):
    lv, co = _two_level()
    o = mk_oracle(orc, [lv, co], delta=20)
    o.assemble()
    o.factor()
    A = o.csr(0).tocsc()
    r = np.random.default_rng(4).normal(size=lv.n_nodes)
    np.testing.assert_allclose(o.ras_apply(r), spla.spsolve(A, r), rtol=1e-11, atol=1e-13)


def _dense_ras(lv, A, subs):
    n = lv.n_nodes
    B = np.diag(lv.dirichlet.astype(float))
    for dofs, own in subs:
        R = np.zeros((dofs.size, n))
        R[np.arange(dofs.size), dofs] = 1.0
        R0 = R * own[:, None]
        B += R0.T @ np.linalg.inv(R @ A @ R.T) @ R
    return B


def test_ras_matches_dense_formula(orc):
    lv, co = _two_level(parts=(3, 2, 2))
    o = mk_oracle(orc, [lv, co], delta=1, coef="cosexp", wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(2))
    o.factor()
    A = o.csr(0).toarray()
    B = _dense_ras(lv, A, o.subdomains(0))
    I = np.eye(lv.n_nodes)
    Bo = np.stack([o.ras_apply(I[:, j]) for j in range(lv.n_nodes)], axis=1)
    np.testing.assert_allclose(Bo, B, atol=1e-11 * abs(B).max())


# ------------------------------------------------------------ interpolation
def test_interp_reproduces_affine_fields(orc):
    fine = syn.cube_level(9, 51)
    coarse = syn.cube_level(4, 52)
    P = orc.build_interp(coarse, fine.xyz, fine.dirichlet, drop_dirichlet=False)
    assert np.all(np.diff(P.indptr) == 4)
    np.testing.assert_allclose(P @ np.ones(coarse.n_nodes), 1.0, atol=1e-14)
    rng = np.random.default_rng(6)
    for _ in range(3):
        g, c = rng.normal(size=3), rng.normal()
        np.testing.assert_allclose(P @ (coarse.xyz @ g + c), fine.xyz @ g + c, atol=1e-13)
    assert P.data.min() >= -1e-12  # the domains coincide: every point is inside
    # the containing tet: every barycentric weight in [-eps, 1+eps]
    assert P.data.max() <= 1 + 1e-12
    # dropping Dirichlet columns keeps exactly the non-Dirichlet columns of each row
    Pd = orc.build_interp(coarse, fine.xyz, fine.dirichlet, drop_dirichlet=True)
    keep = (fine.dirichlet == 0)
    Pm = P[keep][:, coarse.dirichlet == 0]
    np.testing.assert_allclose(Pd[keep][:, coarse.dirichlet == 0].toarray(), Pm.toarray(), atol=0)
    assert Pd[~keep].nnz == 0 and Pd[:, coarse.dirichlet == 1].nnz == 0


def test_interp_identity_on_equal_meshes(orc):
    m = syn.cube_level(5, 61)
    P = orc.build_interp(m, m.xyz, m.dirichlet, drop_dirichlet=False)
    np.testing.assert_allclose(P.toarray(), np.eye(m.n_nodes), atol=1e-14)


def test_interp_picks_lowest_containing_tet(orc):
    """Brute force over all coarse tets on a tiny mesh."""
    fine = syn.cube_level(5, 71)
    coarse = syn.cube_level(2, 72, jitter=0.0)  # unjittered: many shared faces
    P = orc.build_interp(coarse, fine.xyz, fine.dirichlet, drop_dirichlet=False)
    X = coarse.xyz[coarse.tets]
    for f in range(fine.n_nodes):
        x = fine.xyz[f]
        best = None
        for e in range(coarse.n_tets):
            lam1 = np.linalg.solve((X[e, 1:] - X[e, 0]).T, x - X[e, 0])
            lam = np.r_[1 - lam1.sum(), lam1]
            if lam.min() >= -1e-12:
                best = (e, lam)
                break
        e, lam = best
        row = P.getrow(f)
        order = np.argsort(coarse.tets[e])
        np.testing.assert_array_equal(row.indices, coarse.tets[e][order])
        np.testing.assert_allclose(row.data, lam[order], atol=1e-13)


# ------------------------------------------------------------------ V-cycle
def _dense_vcycle(levels, As, Bs, Ps, nu_pre, nu_post, r, l=0):
    if l == len(levels) - 1:
        return np.linalg.solve(As[l], r)
    A, B = As[l], Bs[l]
    z = np.zeros_like(r)
    for _ in range(nu_pre):
        z = z + B @ (r - A @ z)
    rc = Ps[l].T @ (r - A @ z)
    z = z + Ps[l] @ _dense_vcycle(levels, As, Bs, Ps, nu_pre, nu_post, rc, l + 1)
    for _ in range(nu_post):
        z = z + B @ (r - A @ z)
    return z


@pytest.mark.parametrize("nu", [(2, 2), (1, 3)])
def test_vcycle_matches_dense_composition(orc, nu):
    levels = [syn.cube_level(6, 81, parts=(2, 2, 1)), syn.cube_level(4, 82, parts=(2, 1, 1)),
              syn.cube_level(2, 83)]
    wave = syn.wave_vectors()
    o = mk_oracle(orc, levels, delta=1, nu_pre=nu[0], nu_post=nu[1], coef="cosexp", wave=wave)
    mu = syn.mu_draw(9)
    o.assemble(mu)
    o.factor()
    As = [o.csr(l).toarray() for l in range(3)]
    Bs = [_dense_ras(levels[l], As[l], o.subdomains(l)) for l in range(2)]
    # P from an independent barycentric solve on the coarse tet the oracle chose
    Ps = []
    for l in range(2):
        P = o.csr(l, "P").toarray()
        f, c = levels[l], levels[l + 1]
        for i in np.where(f.dirichlet == 0)[0]:
            cols = np.nonzero(P[i])[0]
            # the row must reproduce the fine node position from the coarse ones
            if np.all(c.dirichlet[cols] == 0) and cols.size == 4:
                np.testing.assert_allclose(P[i, cols] @ c.xyz[cols], f.xyz[i], atol=1e-13)
        Ps.append(P)
    rng = np.random.default_rng(10)
    for _ in range(3):
        r = rng.normal(size=levels[0].n_nodes)
        zd = _dense_vcycle(levels, As, Bs, Ps, nu[0], nu[1], r)
        np.testing.assert_allclose(o.vcycle(r), zd, rtol=1e-10, atol=1e-12 * abs(zd).max())


# ------------------------------------------------------------------- FGMRES
def test_gmres_identity_preconditioner_is_krylov_optimal(orc):
    lv, co = _two_level(n=5, nc=2)
    o = mk_oracle(orc, [lv, co], delta=1, coef="cosexp", wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(4))
    A = o.csr(0).toarray()
    b = o.get("b")
    for k in (1, 2, 4, 7):
        x, st = o.fgmres(b, rtol=1e-30, restart=50, maxit=k, precond=False)
        assert st["iters"] == k
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        np.testing.assert_allclose(x, Q @ y, rtol=1e-8, atol=1e-10 * abs(x).max())


@pytest.mark.parametrize("name", ["cube8_2lvl", "cube16_3lvl"])
def test_fgmres_matches_direct_solve(orc, name):
    levels, w = syn.workload(name)
    o = mk_oracle(orc, levels, delta=w["delta"], coef=w["coef"], wave=syn.wave_vectors(),
                  load=w["load"], scale=w["scale"])
    o.assemble(syn.mu_draw(0))
    o.factor()
    x, st = o.fgmres(rtol=1e-12, restart=30)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    A = o.csr(0).tocsc()
    b = o.get("b")
    xe = spla.spsolve(A, b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-10
    # restarting with a tiny restart length still converges to the same solution
    x2, st2 = o.fgmres(rtol=1e-12, restart=2)
    assert st2["status"] == 0
    assert np.linalg.norm(x2 - xe) / np.linalg.norm(xe) <= 1e-10


def test_multilevel_beats_single_level_iterations(orc):
    """Qualitative claim of the paper (Section 4): far fewer iterations with levels."""
    levels, w = syn.workload("cube16_3lvl")
    kw = dict(delta=w["delta"], coef="cosexp", wave=syn.wave_vectors(), load="one")
    o3 = mk_oracle(orc, levels, **kw)
    o3.assemble(syn.mu_draw(0))
    o3.factor()
    _, s3 = o3.fgmres(rtol=1e-8)
    # one RAS level + a direct solve on a tiny 2^3 mesh that contributes nothing
    o1 = mk_oracle(orc, [levels[0], syn.cube_level(2, 5)], **kw)
    o1.assemble(syn.mu_draw(0))
    o1.factor()
    _, s1 = o1.fgmres(rtol=1e-8)
    assert s3["status"] == 0 and s1["status"] == 0
    assert s3["iters"] < s1["iters"]


def test_zero_rhs_gives_zero(orc):
    lv, co = _two_level()
    o = mk_oracle(orc, [lv, co])
    o.assemble()
    o.factor()
    x, st = o.fgmres(np.zeros(lv.n_nodes))
    assert st["status"] == 0 and st["iters"] == 0 and not x.any()
