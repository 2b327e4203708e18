"""Pins for the oracle's paper-literal Algorithm 2 options: the coarsest level
RAS-smoothed like the others (nu_pre steps from z = 0) instead of solved, and
with it the one-level RAS preconditioner.  Each is checked against a dense
numpy composition of independently computed operators.  CPU only.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _dense_ras(lv, A, subs):
    """B = sum_p (R0_p)^T (R_p A R_p^T)^{-1} R_p (Eq. 7), identity on Dirichlet rows."""
    B = np.zeros_like(A)
    for dofs, own in subs:
        inv = np.linalg.inv(A[np.ix_(dofs, dofs)])
        o = own.astype(bool)
        B[np.ix_(dofs[o], dofs)] = inv[o]
    d = np.nonzero(lv.dirichlet)[0]
    B[d, d] = 1.0
    return B


def _smooth(A, B, r, z, its):
    for _ in range(its):
        z = z + B @ (r - A @ z)
    return z


def _dense_vcycle_all_smoothed(As, Bs, Ps, Rs, nu_pre, nu_post, r, l=0):
    z = _smooth(As[l], Bs[l], r, np.zeros_like(r), nu_pre)
    if l == len(As) - 1:
        return z
    rc = Rs[l] @ (r - As[l] @ z)
    z = z + Ps[l] @ _dense_vcycle_all_smoothed(As, Bs, Ps, Rs, nu_pre, nu_post, rc, l + 1)
    return _smooth(As[l], Bs[l], r, z, nu_post)


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_one_level_ras_preconditioner(orc, nu):
    """A single level with the coarsest smoothed: nu RAS sweeps from zero; with
    nu = 1 exactly the one-level RAS preconditioner B of Eq. 7."""
    lv = syn.cube_level(7, 61, parts=(2, 2, 2))
    o = orc.Oracle([lv], delta=1, nu_pre=nu, nu_post=0, coef="cosexp", wave=syn.wave_vectors(),
                   coarse="ras")
    o.assemble(syn.mu_draw(3))
    o.factor()
    A = o.csr(0).toarray()
    B = _dense_ras(lv, A, o.subdomains(0))
    rng = np.random.default_rng(11)
    for _ in range(2):
        r = rng.normal(size=lv.n_nodes)
        zd = _smooth(A, B, r, np.zeros_like(r), nu)
        if nu == 1:
            np.testing.assert_allclose(zd, B @ r)
        np.testing.assert_allclose(o.vcycle(r), zd, rtol=1e-10, atol=1e-12 * abs(zd).max())


@pytest.mark.parametrize("transfer,scaling", [("bary", True), ("mls", False), ("mls", True)])
def test_vcycle_with_smoothed_coarsest_matches_dense_composition(orc, transfer, scaling):
    levels = [syn.cube_level(6, 91, parts=(2, 2, 1)), syn.cube_level(4, 92, parts=(2, 2, 1)),
              syn.cube_level(3, 93, parts=(2, 2, 1))]
    o = orc.Oracle(levels, delta=1, nu_pre=3, nu_post=2, coef="cosexp", wave=syn.wave_vectors(),
                   transfer=transfer, restrict_scaling=scaling, coarse="ras")
    o.assemble(syn.mu_draw(12))
    o.factor()
    As = [o.csr(l).toarray() for l in range(3)]
    Bs = [_dense_ras(levels[l], As[l], o.subdomains(l)) for l in range(3)]
    Ps, Rs = [], []
    for l in range(2):
        f, c = levels[l], levels[l + 1]
        if transfer == "mls":
            h = orc.mesh_h(c)
            P = orc.build_mls(c, f, h=h, delta=1).toarray()
            R = orc.build_mls(f, c, h=h, delta=1, scale=scaling).toarray()
        else:
            P = orc.build_interp(c, f.xyz, f.dirichlet).toarray()
            R = P.T
        Ps.append(P)
        Rs.append(R)
    rng = np.random.default_rng(13)
    for _ in range(2):
        r = rng.normal(size=levels[0].n_nodes)
        zd = _dense_vcycle_all_smoothed(As, Bs, Ps, Rs, 3, 2, r)
        np.testing.assert_allclose(o.vcycle(r), zd, rtol=1e-10, atol=1e-12 * abs(zd).max())


def test_paper_literal_multilevel_beats_one_level_ras(orc):
    """Section 4's qualitative claim with Algorithm 2 taken literally (MLS both
    ways, interpolated residual, every level RAS-smoothed, its = 3, delta = 1):
    far fewer FGMRES iterations than one-level RAS with delta = 1."""
    levels = syn.hierarchy((16, 8, 4), ((4, 4, 4), (4, 4, 4), (2, 2, 2)))
    kw = dict(coef="cosexp", wave=syn.wave_vectors(), load="one", delta=1)
    its = {}
    for tag, lv, extra in (("one", levels[:1], dict(nu_pre=1, nu_post=0)),
                           ("three", levels, dict(nu_pre=3, nu_post=3, transfer="mls",
                                                  restrict_scaling=False))):
        o = orc.Oracle(lv, coarse="ras", **extra, **kw)
        o.assemble(syn.mu_draw(0))
        o.factor()
        x, st = o.fgmres(rtol=1e-8)
        assert st["status"] == 0
        its[tag] = st["iters"]
    assert 2 * its["three"] < its["one"]


def test_smoothed_coarsest_needs_a_partition(orc):
    levels = [syn.cube_level(4, 1, parts=(2, 1, 1)), syn.cube_level(2, 2)]
    with pytest.raises(ValueError):
        orc.Oracle(levels, coarse="ras")
