"""Parity at the measured size: cube64_3lvl (274,625 fine nodes, 512
subdomains per smoothed level), built with the options `bench.py` times.

The oracle cannot run the whole 64^3 hierarchy in seconds, so the checks are
the outputs it computes one by one at this size and properties that hold at
any size:
  * level-0 CSR pattern (bit for bit), values and load vector, subdomain DoF
    lists and owned flags (bit for bit) -- the oracle builds level 0 alone,
    with a tiny coarse level so that its own transfers stay cheap;
  * the factors L, D and the RAS rows of three sampled subdomains (the
    oracle factors just those);
  * J x against the oracle's CSR; P reproduces affine fields and P^T is its
    adjoint; the coarsest direct solve leaves a residual at rounding level;
  * the FGMRES solution meets rtol on the oracle's operator, and the FP32
    factor path reaches the same solution.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, make_oracle, rel, relmax, workload

pytestmark = pytest.mark.gpu

SAMPLED = (0, 255, 511)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def P():
    from paper_2412_08981_gb300 import build as b
    b.build()
    import paper_2412_08981_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def full(P, orc, torch):
    levels, w = workload("cube64_3lvl")
    mu = syn.mu_draw(0)
    h = make_hierarchy(levels, w, P)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    o0 = make_oracle([levels[0], syn.cube_level(2, 5)], w, orc)
    o0.assemble(mu)
    for p in SAMPLED:
        assert o0.factor_range(0, p, p + 1) == 0
    return dict(levels=levels, w=w, mu=mu, h=h, inst=inst, o0=o0)


def _dev(torch, a):
    return torch.tensor(np.asarray(a, np.float64), device="cuda")


def test_full_assembly_pattern_and_load(full):
    h, inst, o0 = full["h"], full["inst"], full["o0"]
    np.testing.assert_array_equal(h.array(0, "rowptr"), o0.get("rowptr", 0))
    np.testing.assert_array_equal(h.array(0, "col"), o0.get("col", 0))
    vo = o0.get("val", 0)
    assert np.max(np.abs(inst.array(0, "val") - vo)) <= 1e-13 * np.max(np.abs(vo))
    assert rel(h.array(0, "load"), o0.get("b", 0)) <= 1e-14


def test_full_subdomains_bit_exact(full):
    h, o0 = full["h"], full["o0"]
    subs = o0.subdomains(0)
    sp, sd, so = h.array(0, "sub_ptr"), h.array(0, "sub_dofs"), h.array(0, "sub_own")
    assert sp.size - 1 == len(subs) == 512
    for p, (d, ow) in enumerate(subs):
        np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)
        np.testing.assert_array_equal(so[sp[p]:sp[p + 1]], ow)


def test_full_spmv(full, P, torch):
    inst, o0 = full["inst"], full["o0"]
    A = o0.csr(0)
    x = np.random.default_rng(1).normal(size=A.shape[0])
    y = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    inst.apply_op(P.msp.MSP_OP_SPMV, 0, _dev(torch, x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), A @ x) <= 1e-14


def test_full_transfers_reproduce_affine_fields_and_are_adjoint(full, P, torch):
    h, inst, levels = full["h"], full["inst"], full["levels"]
    m = P.msp
    for l in range(2):
        f, c = levels[l], levels[l + 1]
        rp = h.array(l, "P_rowptr")
        full_rows = (np.diff(rp) == 4) & (f.dirichlet == 0)  # no Dirichlet column dropped
        assert full_rows.mean() > 0.5
        rng = np.random.default_rng(2 + l)
        g, c0 = rng.normal(size=3), rng.normal()
        yf = torch.zeros(f.n_nodes, dtype=torch.float64, device="cuda")
        inst.apply_op(m.MSP_OP_INTERP, l, _dev(torch, c.xyz @ g + c0), yf)
        torch.cuda.synchronize()
        yv = yf.cpu().numpy()
        want = f.xyz @ g + c0
        assert np.max(np.abs(yv[full_rows] - want[full_rows])) <= 1e-12 * np.max(np.abs(want))
        assert not yv[f.dirichlet == 1].any()
        xc, xf = rng.normal(size=c.n_nodes), rng.normal(size=f.n_nodes)
        yc = torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")
        inst.apply_op(m.MSP_OP_INTERP, l, _dev(torch, xc), yf)
        inst.apply_op(m.MSP_OP_RESTRICT, l, _dev(torch, xf), yc)
        torch.cuda.synchronize()
        a, b = float(yf.cpu().numpy() @ xf), float(xc @ yc.cpu().numpy())
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


def test_full_sampled_factors_and_ras_rows(full, P, torch):
    h, inst, o0 = full["h"], full["inst"], full["o0"]
    for p in SAMPLED:
        dofs = o0.get("sub_dofs", 0, p)
        n = dofs.size
        LU = o0.get("sub_lu", 0, p).reshape(n, n)
        Lo, do = np.tril(LU, -1) + np.eye(n), np.diag(LU)
        Lg, dg = P.msp.unpack_factor(inst.array(0, "factor", p), n, P.msp.tile_first_of(h, 0, p))
        assert np.max(np.abs(Lg - Lo)) <= 1e-10 * max(1.0, np.max(np.abs(Lo)))
        assert rel(dg, do) <= 1e-12
    r = np.random.default_rng(4).normal(size=o0.n[0])
    z = torch.zeros(o0.n[0], dtype=torch.float64, device="cuda")
    inst.apply_op(P.msp.MSP_OP_RAS, 0, _dev(torch, r), z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy()
    for p in SAMPLED:
        zo = o0.ras_apply_range(r, 0, p, p + 1)
        dofs, own = o0.get("sub_dofs", 0, p), o0.get("sub_own", 0, p).astype(bool)
        assert rel(zg[dofs[own]], zo[dofs[own]]) <= 1e-12


def test_full_coarsest_solve_residual(full, P, orc, torch):
    levels, w, inst = full["levels"], full["w"], full["inst"]
    oc = make_oracle([levels[2]], w, orc)
    oc.assemble(full["mu"])
    Ac = oc.csr(0)
    import scipy.sparse.linalg as spla
    lu = spla.splu(Ac.tocsc())
    rng = np.random.default_rng(5)
    # repeated applications: the cluster sweeps exchange every tile row, so an
    # ordering fault would show as an occasional wrong row, not a constant one
    for _ in range(12):
        r = rng.normal(size=Ac.shape[0])
        z = torch.zeros(Ac.shape[0], dtype=torch.float64, device="cuda")
        inst.apply_op(P.msp.MSP_OP_COARSE, 2, _dev(torch, r), z)
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
        assert rel(Ac @ zg, r) <= 1e-11
        assert relmax(zg, lu.solve(r)) <= 1e-11


def test_full_solution_meets_rtol_in_fp64_and_fp32(full, P, torch):
    levels, w, inst, o0 = full["levels"], full["w"], full["inst"], full["o0"]
    A, b = o0.csr(0), o0.get("b", 0)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    xg = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(b - A @ xg) <= 1.01e-10 * np.linalg.norm(b)
    h32 = make_hierarchy(levels, w, P, precision="f32")
    i32 = h32.assemble(full["mu"], stream=torch.cuda.current_stream())
    i32.factor()
    x32 = torch.zeros_like(x)
    s32 = i32.solve(x32, rtol=1e-10)
    assert s32["status"] == 0 and s32["iterations"] <= st["iterations"] + 3
    assert rel(x32.cpu().numpy(), xg) <= 1e-8
