"""Pins for the oracle's multi-field case: linear elasticity with three P1
displacement fields per vertex (the DoF distribution N = (3,0,0,0) of the
mesh perspective, Section 2.1) and the field-split transfers P (x) I_3.

The element stiffness is checked against an independent Voigt-notation
construction (B^T D B with engineering shear strains), rigid-body modes, its
rank and the closed-form energy of linear fields; the assembled operator by
the patch test, rigid modes and O(h^2) convergence to a manufactured
solution; the transfers by exact reproduction of affine vector fields; RAS,
the V-cycle and FGMRES by the same dense compositions as the scalar case.
CPU only.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

NU = 0.3


def _random_tet(rng):
    while True:
        x = rng.normal(size=(4, 3))
        if abs(np.linalg.det(x[1:] - x[0])) > 0.2:
            return x


def _rigid_modes(x):
    """6 rigid-body displacements of the points x (n x 3), interleaved 3n."""
    n = x.shape[0]
    modes = []
    for c in range(3):
        u = np.zeros((n, 3))
        u[:, c] = 1.0
        modes.append(u.ravel())
    for w in np.eye(3):
        modes.append(np.cross(w, x).ravel())
    return np.stack(modes, axis=1)


def _voigt_stiffness(x, lam, mu):
    """|T| B^T D B: strains (e_xx, e_yy, e_zz, g_yz, g_xz, g_xy), g = 2 e."""
    T = np.hstack([np.ones((4, 1)), x])
    G = np.linalg.inv(T)[1:].T  # gradients of the barycentric functions, 4 x 3
    vol = abs(np.linalg.det(x[1:] - x[0])) / 6.0
    B = np.zeros((6, 12))
    for a in range(4):
        gx, gy, gz = G[a]
        B[0, 3 * a] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1], B[3, 3 * a + 2] = gz, gy
        B[4, 3 * a], B[4, 3 * a + 2] = gz, gx
        B[5, 3 * a], B[5, 3 * a + 1] = gy, gx
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return vol * B.T @ D @ B, vol


def test_element_matches_voigt_construction(orc):
    lam, mu = orc.lame(NU)
    rng = np.random.default_rng(1)
    for _ in range(4):
        x = _random_tet(rng)
        k = rng.uniform(0.5, 2.0)
        K, vol = orc.tet_elasticity(x, k=k, poisson=NU)
        Kv, volv = _voigt_stiffness(x, lam, mu)
        assert abs(vol - volv) <= 1e-14 * volv
        np.testing.assert_allclose(K, k * Kv, rtol=0, atol=1e-13 * abs(Kv).max())


def test_element_rigid_modes_rank_and_linear_energy(orc):
    lam, mu = orc.lame(NU)
    rng = np.random.default_rng(2)
    x = _random_tet(rng)
    K, vol = orc.tet_elasticity(x, poisson=NU)
    np.testing.assert_allclose(K, K.T, atol=1e-14 * abs(K).max())
    R = _rigid_modes(x)
    assert abs(K @ R).max() <= 1e-13 * abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) <= 1e-12 * ev.max()) == 6 and ev.min() > -1e-12 * ev.max()
    for _ in range(3):  # linear u = G x: energy = |T| (2 mu eps:eps + lam tr(eps)^2)
        Gm = rng.normal(size=(3, 3))
        u = (x @ Gm.T).ravel()
        eps = 0.5 * (Gm + Gm.T)
        e = vol * (2 * mu * np.sum(eps * eps) + lam * np.trace(eps) ** 2)
        assert abs(u @ K @ u - e) <= 1e-12 * e


def _free_level(n, seed, parts=None):
    lv = syn.cube_level(n, seed, parts=parts)
    lv.dirichlet = np.zeros_like(lv.dirichlet)
    return lv


def test_global_patch_test_and_rigid_modes(orc):
    """No Dirichlet nodes, k constant: rigid motions are in the kernel of the
    assembled operator, and a linear field has zero nodal force at every
    vertex off the boundary (constant stress is in equilibrium)."""
    lv = _free_level(4, 11)
    o = orc.Oracle([lv], pde="elasticity", poisson=NU)
    o.assemble()
    A = o.csr(0)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    R = _rigid_modes(lv.xyz)
    assert abs(A @ R).max() <= 1e-12 * abs(A).max()
    bnd = np.any((lv.xyz <= 1e-12) | (lv.xyz >= 1 - 1e-12), axis=1)
    rng = np.random.default_rng(3)
    for _ in range(2):
        Gm, c = rng.normal(size=(3, 3)), rng.normal(size=3)
        f = (A @ (lv.xyz @ Gm.T + c).ravel()).reshape(-1, 3)
        assert abs(f[~bnd]).max() <= 1e-12 * abs(f[bnd]).max()
        assert abs(f[bnd]).max() > 1e-6


def test_dirichlet_rows_and_load(orc):
    lv = syn.cube_level(4, 12)
    o = orc.Oracle([lv], pde="elasticity", poisson=NU)
    o.assemble()
    A = o.csr(0).toarray()
    b = o.get("b")
    d = np.repeat(lv.dirichlet.astype(bool), 3)
    np.testing.assert_array_equal(A[d][:, d], np.eye(d.sum()))
    assert not A[d][:, ~d].any() and not A[~d][:, d].any()
    assert not b[d].any()
    # unit body force along -z: b_z = -sum_{T ni v} |T| / 4, x and y zero
    x = lv.xyz[lv.tets]
    vol = np.abs(np.linalg.det(x[:, 1:] - x[:, :1])) / 6.0
    m = np.bincount(lv.tets.ravel(), weights=np.repeat(vol / 4, 4), minlength=lv.n_nodes)
    bb = b.reshape(-1, 3)
    np.testing.assert_allclose(bb[:, 2], np.where(lv.dirichlet == 1, 0.0, -m), atol=1e-15)
    assert not bb[:, :2].any()
    np.linalg.cholesky(A[~d][:, ~d])  # SPD on the free DoFs


def test_manufactured_solution_converges_h2(orc):
    """k = 1, u = (s, s, s) with s = sin sin sin: nodal L2 error O(h^2)."""
    errs, hs = [], []
    for n in (6, 12, 24):
        lv = syn.cube_level(n, 2000 + n)
        o = orc.Oracle([lv], pde="elasticity", poisson=NU, load="sines")
        o.assemble()
        u = spla.spsolve(o.csr(0).tocsc(), o.get("b")).reshape(-1, 3)
        ue = np.prod(np.sin(np.pi * lv.xyz), axis=1)
        x = lv.xyz[lv.tets]
        vol = np.abs(np.linalg.det(x[:, 1:] - x[:, :1])) / 6.0
        m = np.bincount(lv.tets.ravel(), weights=np.repeat(vol / 4, 4), minlength=lv.n_nodes)
        errs.append(np.sqrt(np.sum(m[:, None] * (u - ue[:, None]) ** 2)))
        hs.append(1.0 / n)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - 2.0) <= 0.25, (slope, errs)


def test_field_split_transfer_reproduces_affine_vector_fields(orc):
    fine = _free_level(7, 21, parts=(1, 1, 1))
    coarse = _free_level(3, 22)
    o = orc.Oracle([fine, coarse], pde="elasticity", poisson=NU)
    P = o.csr(0, "P")
    assert P.shape == (3 * fine.n_nodes, 3 * coarse.n_nodes)
    rng = np.random.default_rng(5)
    for _ in range(3):
        Gm, c = rng.normal(size=(3, 3)), rng.normal(size=3)
        uc = (coarse.xyz @ Gm.T + c).ravel()
        uf = (fine.xyz @ Gm.T + c).ravel()
        np.testing.assert_allclose(P @ uc, uf, atol=1e-12)
    # fields never mix, and each field's block is the scalar interpolation
    Ps = orc.build_interp(coarse, fine.xyz, fine.dirichlet, drop_dirichlet=True)
    for c in range(3):
        for c2 in range(3):
            blk = P[c::3][:, c2::3]
            if c == c2:
                np.testing.assert_allclose(blk.toarray(), Ps.toarray(), atol=0)
            else:
                assert blk.nnz == 0 or not blk.toarray().any()
    np.testing.assert_allclose(o.csr(0, "PT").toarray(), P.T.toarray(), atol=0)


def _dense_ras(lv, A, subs):
    B = np.zeros_like(A)
    for dofs, own in subs:
        inv = np.linalg.inv(A[np.ix_(dofs, dofs)])
        ow = own.astype(bool)
        B[np.ix_(dofs[ow], dofs)] = inv[ow]
    d = np.nonzero(np.repeat(lv.dirichlet, 3))[0]
    B[d, d] = 1.0
    return B


def test_ras_one_subdomain_is_exact_and_dense_formula(orc):
    lv = syn.cube_level(4, 31, parts=(1, 1, 1))
    co = syn.cube_level(2, 32)
    o = orc.Oracle([lv, co], delta=1, pde="elasticity", poisson=NU, coef="cosexp",
                   wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(1))
    o.factor()
    A = o.csr(0).toarray()
    r = np.random.default_rng(7).normal(size=A.shape[0])
    np.testing.assert_allclose(o.ras_apply(r, 0), np.linalg.solve(A, r), rtol=1e-9, atol=1e-12)
    lv2 = syn.cube_level(5, 33, parts=(2, 2, 1))
    o2 = orc.Oracle([lv2, co], delta=1, pde="elasticity", poisson=NU, coef="cosexp",
                    wave=syn.wave_vectors())
    o2.assemble(syn.mu_draw(2))
    o2.factor()
    subs = o2.subdomains(0)
    for dofs, _ in subs:  # all three fields of a vertex together
        assert np.all(dofs.reshape(-1, 3) == 3 * (dofs[::3] // 3)[:, None] + np.arange(3))
    A2 = o2.csr(0).toarray()
    B = _dense_ras(lv2, A2, subs)
    r2 = np.random.default_rng(8).normal(size=A2.shape[0])
    np.testing.assert_allclose(o2.ras_apply(r2, 0), B @ r2, rtol=1e-10, atol=1e-12)


def _dense_vcycle(As, Bs, Ps, nu_pre, nu_post, r, l=0):
    if l == len(As) - 1:
        return np.linalg.solve(As[l], r)
    A, B = As[l], Bs[l]
    z = np.zeros_like(r)
    for _ in range(nu_pre):
        z = z + B @ (r - A @ z)
    z = z + Ps[l] @ _dense_vcycle(As, Bs, Ps, nu_pre, nu_post, Ps[l].T @ (r - A @ z), l + 1)
    for _ in range(nu_post):
        z = z + B @ (r - A @ z)
    return z


def test_vcycle_matches_dense_composition(orc):
    levels = [syn.cube_level(5, 41, parts=(2, 2, 1)), syn.cube_level(3, 42, parts=(2, 1, 1)),
              syn.cube_level(2, 43)]
    o = orc.Oracle(levels, delta=1, nu_pre=2, nu_post=1, pde="elasticity", poisson=NU, coef="cosexp",
                   wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(3))
    o.factor()
    As = [o.csr(l).toarray() for l in range(3)]
    Bs = [_dense_ras(levels[l], As[l], o.subdomains(l)) for l in range(2)]
    Ps = [o.csr(l, "P").toarray() for l in range(2)]
    rng = np.random.default_rng(9)
    for _ in range(2):
        r = rng.normal(size=As[0].shape[0])
        zd = _dense_vcycle(As, Bs, Ps, 2, 1, r)
        np.testing.assert_allclose(o.vcycle(r), zd, rtol=1e-10, atol=1e-12 * abs(zd).max())


def test_fgmres_solves_and_levels_help(orc):
    levels = syn.hierarchy((12, 6, 3), ((2, 2, 2), (2, 2, 2)))
    kw = dict(delta=1, pde="elasticity", poisson=NU, coef="cosexp", wave=syn.wave_vectors())
    o = orc.Oracle(levels, **kw)
    o.assemble(syn.mu_draw(0))
    o.factor()
    x, st = o.fgmres(rtol=1e-10)
    assert st["status"] == 0
    xe = spla.spsolve(o.csr(0).tocsc(), o.get("b"))
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-8
    o1 = orc.Oracle([levels[0], syn.cube_level(2, 5)], **kw)
    o1.assemble(syn.mu_draw(0))
    o1.factor()
    _, s1 = o1.fgmres(rtol=1e-10)
    assert s1["status"] == 0 and st["iters"] < s1["iters"]


def test_elasticity_rejects_mls_and_bad_poisson(orc):
    levels = [syn.cube_level(4, 51, parts=(2, 1, 1)), syn.cube_level(2, 52)]
    with pytest.raises(ValueError):
        orc.Oracle(levels, pde="elasticity", transfer="mls")
    with pytest.raises(ValueError):
        orc.Oracle(levels, pde="elasticity", poisson=0.5)
