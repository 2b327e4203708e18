"""Pins for the oracle's overlapping MLS transfer (Section 3.2, Eq. 13-15, 24).

Each row of the oracle's operator is checked against a brute-force restatement
that shares none of its steps: the neighbourhood from a sparse-matrix
breadth-first search and a numpy distance test, the radius grown until numpy's
SVD rank of the monomial basis [1, x, y, z] is 4, the weights of Eq. 15, and
the fitted value from the SVD pseudo-inverse of the weighted least-squares
system in that monomial basis.  Further pins: exact reproduction of affine
fields (MLS reproduces its polynomial space, Theorem 3.2), the Dirichlet
handling, the nodal-volume scaling of the restriction, and the V-cycle built on
the MLS transfers against a dense composition.  CPU only.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ----------------------------------------------------------------- helpers
def _graph(lv):
    a = np.repeat(lv.tets, 4, axis=1).ravel()
    b = np.tile(lv.tets, (1, 4)).ravel()
    G = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(lv.n_nodes,) * 2).tocsr()
    G.data[:] = 1.0
    return G


def _overlap(lv, q, delta, G):
    """Vertices within delta graph hops of the vertices owned by q."""
    reach = (lv.owner == q).astype(float)
    for _ in range(delta):
        reach = np.minimum(reach + G @ reach, 1.0)
    return np.nonzero(reach)[0]


def _h(lv):
    ext = lv.xyz.max(axis=0) - lv.xyz.min(axis=0)
    return np.cbrt(6.0 * np.prod(ext) / lv.tets.shape[0])


def _brute_row(src, dst, t, h, delta, G):
    x = dst.xyz[t]
    cand = np.arange(src.n_nodes)
    if (src.owner is not None and dst.owner is not None
            and set(np.unique(src.owner)) == set(np.unique(dst.owner))):
        cand = _overlap(src, dst.owner[t], delta, G)
    d = np.linalg.norm(src.xyz[cand] - x, axis=1)
    c = 1.5
    for _ in range(16):
        rho = c * h
        nb = cand[d < rho]
        Pm = np.c_[np.ones(nb.size), src.xyz[nb]]
        if nb.size >= 4 and np.linalg.matrix_rank(Pm) == 4:
            break
        c *= 1.5
    else:
        raise AssertionError("no rank-4 neighbourhood")
    s = np.linalg.norm(src.xyz[nb] - x, axis=1) / rho
    w = 1 - 6 * s**2 + 8 * s**3 - 3 * s**4
    sw = np.sqrt(w)
    phi = (np.r_[1.0, x] @ np.linalg.pinv(sw[:, None] * Pm)) * sw
    return nb, phi


def _nodal_volumes(lv):
    x = lv.xyz[lv.tets]
    v = np.abs(np.linalg.det(x[:, 1:] - x[:, :1])) / 6.0
    out = np.zeros(lv.n_nodes)
    np.add.at(out, lv.tets.ravel(), np.repeat(v / 4.0, 4))
    return out


def _pair(nf=8, nc=4, pf=(2, 2, 2), pc=(2, 2, 2), seed=300):
    f = syn.cube_level(nf, seed, parts=pf)
    c = syn.cube_level(nc, seed + 1, parts=pc)
    return f, c


# -------------------------------------------------------------------- rows
@pytest.mark.parametrize("direction", ["prolong", "restrict"])
@pytest.mark.parametrize("delta", [1, 2])
def test_mls_rows_match_weighted_least_squares(orc, direction, delta):
    f, c = _pair()
    src, dst = (c, f) if direction == "prolong" else (f, c)
    h = _h(c)
    M = orc.build_mls(src, dst, h=h, delta=delta, drop_dirichlet=False)
    G = _graph(src)
    for t in range(dst.n_nodes):
        nb, phi = _brute_row(src, dst, t, h, delta, G)
        row = M.getrow(t)
        np.testing.assert_array_equal(row.indices, nb)
        np.testing.assert_allclose(row.data, phi, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("cparts", [None, (2, 1, 1)])
def test_mls_unmatched_partitions_use_whole_mesh(orc, cparts):
    """No partition on the source (a coarsest level), or partitions over
    different id sets: the neighbourhood comes from the whole source mesh."""
    f, _ = _pair()
    c = syn.cube_level(3, 77, parts=cparts)
    h = _h(c)
    M = orc.build_mls(c, f, h=h, delta=2, drop_dirichlet=False)
    Mall = orc.build_mls(syn.cube_level(3, 77), f, h=h, delta=2, drop_dirichlet=False)
    np.testing.assert_array_equal(abs(M - Mall).max(), 0.0)
    G = _graph(c)
    for t in range(0, f.n_nodes, 7):
        nb, phi = _brute_row(c, f, t, h, 2, G)
        np.testing.assert_array_equal(M.getrow(t).indices, nb)
        np.testing.assert_allclose(M.getrow(t).data, phi, rtol=1e-9, atol=1e-11)


def test_mls_overlap_limits_the_neighbourhood(orc):
    """With delta = 0 the fit near a subdomain face uses one side only, so the
    operator differs from the whole-mesh one there, and every column lies in
    the target's own source subdomain."""
    f, c = _pair(nf=8, nc=8, pf=(2, 2, 2), pc=(2, 2, 2), seed=310)
    h = _h(c)
    M0 = orc.build_mls(c, f, h=h, delta=0, drop_dirichlet=False)
    c_np = syn.cube_level(8, 311)  # same mesh, no partition
    Mall = orc.build_mls(c_np, f, h=h, delta=0, drop_dirichlet=False)
    assert abs(M0 - Mall).max() > 1e-3
    for t in range(f.n_nodes):
        cols = M0.getrow(t).indices
        assert np.all(c.owner[cols] == f.owner[t])


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", ["cube8_2lvl", "cube16_3lvl"])
def test_mls_reproduces_affine_fields(orc, name):
    levels, w = syn.workload(name)
    rng = np.random.default_rng(5)
    for l in range(len(levels) - 1):
        f, c = levels[l], levels[l + 1]
        h = _h(c)
        for src, dst in ((c, f), (f, c)):
            M = orc.build_mls(src, dst, h=h, delta=w["delta"], drop_dirichlet=False)
            for _ in range(3):
                a = rng.normal(size=4)
                u = lambda x: a[0] + x @ a[1:]
                np.testing.assert_allclose(M @ u(src.xyz), u(dst.xyz), atol=1e-12)
            np.testing.assert_allclose(np.asarray(M.sum(axis=1)).ravel(), 1.0, atol=1e-13)


def test_mls_dirichlet_handling(orc):
    f, c = _pair()
    h = _h(c)
    full = orc.build_mls(c, f, h=h, delta=1, drop_dirichlet=False).tolil()
    drop = orc.build_mls(c, f, h=h, delta=1, drop_dirichlet=True)
    expect = full.copy()
    expect[np.nonzero(f.dirichlet)[0], :] = 0
    expect[:, np.nonzero(c.dirichlet)[0]] = 0
    expect = expect.tocsr()
    expect.eliminate_zeros()
    assert np.all(np.diff(drop.indptr)[f.dirichlet == 1] == 0)
    assert not np.isin(drop.indices, np.nonzero(c.dirichlet)[0]).any()
    np.testing.assert_array_equal(abs(drop - expect).max(), 0.0)


def test_mls_restriction_scaling(orc):
    f, c = _pair()
    h = _h(c)
    R = orc.build_mls(f, c, h=h, delta=1, drop_dirichlet=True, scale=False)
    Rs = orc.build_mls(f, c, h=h, delta=1, drop_dirichlet=True, scale=True)
    vf, vc = _nodal_volumes(f), _nodal_volumes(c)
    expect = sp.diags(vc) @ R @ sp.diags(1.0 / vf)
    np.testing.assert_allclose(Rs.toarray(), expect.toarray(), rtol=1e-13, atol=0)
    # on these uniform-density meshes the scale is about (H/h)^3 = 8
    ratio = Rs.sum() / R.sum()
    assert 6.0 < ratio < 10.0


def test_mls_radius_unit(orc):
    assert orc.mesh_h(syn.cube_level(4, 1)) == pytest.approx(0.25, rel=1e-14)
    assert orc.mesh_h(syn.cube_level(10, 2)) == pytest.approx(0.1, rel=1e-14)


# ------------------------------------------------------------------ V-cycle
def _dense_ras(lv, A, subs):
    B = np.zeros_like(A)
    for dofs, own in subs:
        inv = np.linalg.inv(A[np.ix_(dofs, dofs)])
        rows = dofs[own.astype(bool)]
        B[np.ix_(rows, dofs)] = inv[own.astype(bool)]
    d = np.nonzero(lv.dirichlet)[0]
    B[d, d] = 1.0
    return B


def _dense_vcycle(As, Bs, Ps, Rs, nu_pre, nu_post, r, l=0):
    if l == len(As) - 1:
        return np.linalg.solve(As[l], r)
    A, B = As[l], Bs[l]
    z = np.zeros_like(r)
    for _ in range(nu_pre):
        z = z + B @ (r - A @ z)
    z = z + Ps[l] @ _dense_vcycle(As, Bs, Ps, Rs, nu_pre, nu_post, Rs[l] @ (r - A @ z), l + 1)
    for _ in range(nu_post):
        z = z + B @ (r - A @ z)
    return z


@pytest.mark.parametrize("scaling", [True, False])
def test_vcycle_with_mls_matches_dense_composition(orc, scaling):
    levels = [syn.cube_level(6, 81, parts=(2, 2, 1)), syn.cube_level(4, 82, parts=(2, 1, 1)),
              syn.cube_level(2, 83)]
    o = orc.Oracle(levels, delta=1, coef="cosexp", wave=syn.wave_vectors(), transfer="mls",
                   restrict_scaling=scaling)
    o.assemble(syn.mu_draw(9))
    o.factor()
    As = [o.csr(l).toarray() for l in range(3)]
    Bs = [_dense_ras(levels[l], As[l], o.subdomains(l)) for l in range(2)]
    Ps, Rs = [], []
    for l in range(2):
        f, c = levels[l], levels[l + 1]
        P = orc.build_mls(c, f, h=orc.mesh_h(c), delta=1, drop_dirichlet=True)
        R = orc.build_mls(f, c, h=orc.mesh_h(c), delta=1, drop_dirichlet=True, scale=scaling)
        np.testing.assert_array_equal(abs(o.csr(l, "P") - P).max(), 0.0)
        np.testing.assert_array_equal(abs(o.csr(l, "PT") - R).max(), 0.0)
        Ps.append(P.toarray())
        Rs.append(R.toarray())
    rng = np.random.default_rng(10)
    for _ in range(3):
        r = rng.normal(size=levels[0].n_nodes)
        zd = _dense_vcycle(As, Bs, Ps, Rs, 2, 2, r)
        np.testing.assert_allclose(o.vcycle(r), zd, rtol=1e-10, atol=1e-12 * abs(zd).max())


def test_mls_multilevel_converges_and_beats_single_level(orc):
    levels, w = syn.workload("cube16_3lvl")
    kw = dict(delta=w["delta"], coef="cosexp", wave=syn.wave_vectors(), load="one")
    om = orc.Oracle(levels, transfer="mls", **kw)
    om.assemble(syn.mu_draw(0))
    om.factor()
    x, sm = om.fgmres(rtol=1e-10)
    A = om.csr(0)
    b = om.get("b")
    assert sm["status"] == 0
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.01
    its = {}
    for tag, o in (("mls", om),
                   ("plain", orc.Oracle(levels, transfer="mls", restrict_scaling=False, **kw)),
                   ("one", orc.Oracle([levels[0], syn.cube_level(2, 5)], **kw))):
        o.assemble(syn.mu_draw(0))
        o.factor()
        _, st = o.fgmres(rtol=1e-8)
        assert st["status"] == 0
        its[tag] = st["iters"]
    # the scaled restriction matches the coarse operator's scale: fewer
    # iterations than the plain interpolated residual, and than one level
    assert its["mls"] < its["plain"] <= its["one"]
