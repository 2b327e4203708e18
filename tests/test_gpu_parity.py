"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every operator of the hot path is compared element by element on the same
seeded inputs: assembly, load vector, SpMV, the transfers (P and P^T, or the
MLS operators), subdomain factors, the
RAS application, the coarsest solve, the whole V-cycle and the FGMRES
solution.  Tolerances: FP64 operators <= 1e-12 relative (the per operator
bound of the method's FP64 path), solution <= 1e-7 relative at rtol 1e-10;
vectors are held to each bound both norm-wise (||a - b|| / ||b||) and
element-wise (max |a - b| / max |b|).
"""
import numpy as np
import pytest

import synthetic as syn
from _common import PARITY, close, make_hierarchy, make_oracle, rel, workload

pytestmark = pytest.mark.gpu

OP_TOL = 1e-12


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


class Case:
    def __init__(self, name, P, orc, torch, mu_req=0, transfer="bary", **kw):
        self.levels, self.w = workload(name)
        self.mu = syn.mu_draw(mu_req)
        self.o = make_oracle(self.levels, self.w, orc, transfer=transfer)
        self.o.assemble(self.mu)
        self.o.factor()
        self.h = make_hierarchy(self.levels, self.w, P, transfer=transfer, **kw)
        self.inst = self.h.assemble(self.mu, stream=torch.cuda.current_stream())
        self.inst.factor()
        self.torch = torch
        self.n = list(self.o.n)  # DoFs per level (fields x vertices, or vertices + edges)
        self.dir0 = self.o.get("dofdir", 0)

    def dev(self, x):
        return self.torch.tensor(np.asarray(x, np.float64), device="cuda")

    def zeros(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64, device="cuda")

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.cpu().numpy()


# every parity workload with P / P^T, two with the MLS transfers of Section
# 3.2 (cube20m pairs the subdomains of the two RAS levels), the multi-field
# case (linear elasticity, three fields per vertex, field-split P), the
# quadratic elements (DoFs on vertices and edges, the P2 interpolation) and
# the coupled pair of a P2 and a P1 field (the transfer split by field with a
# different interpolation per field)
CASES = ([(n, "bary") for n in PARITY] + [("cube16_3lvl", "mls"), ("cube20m_3lvl", "mls")] +
         [("elast12_3lvl", "bary"), ("p2cube12_3lvl", "bary"), ("p2p1cube12_3lvl", "bary")])


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def case(request, P, orc, torch):
    name, transfer = request.param
    return Case(name, P, orc, torch, transfer=transfer)


def test_assembly_and_load(case):
    for l in range(len(case.levels)):
        vg = case.inst.array(l, "val")
        vo = case.o.get("val", l)
        assert np.max(np.abs(vg - vo)) <= 1e-13 * np.max(np.abs(vo))
    bg = case.h.array(0, "load")
    assert close(bg, case.o.get("b", 0), 1e-14)


def test_spmv_and_transfers(case, P):
    rng = np.random.default_rng(1)
    m = P.msp
    for l in range(len(case.levels)):
        x = rng.normal(size=case.n[l])
        y = case.zeros(case.n[l])
        case.inst.apply_op(m.MSP_OP_SPMV, l, case.dev(x), y)
        assert close(case.host(y), case.o.spmv(x, l), 1e-14)
        # residual form: y = r - A x
        r = rng.normal(size=case.n[l])
        yr = case.dev(r)
        case.inst.apply_op(m.MSP_OP_RESIDUAL, l, case.dev(x), yr)
        assert close(case.host(yr), r - case.o.spmv(x, l), 1e-13)
    for l in range(len(case.levels) - 1):
        xc = rng.normal(size=case.n[l + 1])
        yf = case.zeros(case.n[l])
        case.inst.apply_op(m.MSP_OP_INTERP, l, case.dev(xc), yf)
        assert close(case.host(yf), case.o.interp(xc, l), 1e-14)
        xf = rng.normal(size=case.n[l])
        yc = case.zeros(case.n[l + 1])
        case.inst.apply_op(m.MSP_OP_RESTRICT, l, case.dev(xf), yc)
        assert close(case.host(yc), case.o.restrict(xf, l), 1e-14)


def test_subdomain_factors(case, P):
    """L and D of sampled blocks vs the oracle's Doolittle LU (U = D L^T)."""
    for l in range(len(case.levels)):
        coarse = l == len(case.levels) - 1
        ns = 1 if coarse else case.o.get("n_subs", l)
        for p in sorted(set([0, ns // 2, ns - 1])):
            sub = -1 if coarse else p
            dofs = case.o.get("sub_dofs", l, sub)
            n = dofs.size
            LU = case.o.get("sub_lu", l, sub).reshape(n, n)
            Lo = np.tril(LU, -1) + np.eye(n)
            do = np.diag(LU)
            Lg, dg = P.msp.unpack_factor(case.inst.array(l, "factor", sub), n,
                                         P.msp.tile_first_of(case.h, l, sub))
            assert np.max(np.abs(Lg - Lo)) <= 1e-10 * max(1.0, np.max(np.abs(Lo)))
            assert close(dg, do, 1e-12)
            # the symmetric factors reproduce the block: L D L^T = A_p
            A = case.o.csr(l).toarray()[np.ix_(dofs, dofs)]
            assert np.linalg.norm(Lg @ np.diag(dg) @ Lg.T - A) <= 1e-13 * np.linalg.norm(A)


def test_diagonal_tiles_hold_the_inverse(case, P):
    """Every diagonal tile of sampled blocks of every level stores X^T above
    its diagonal, X the inverse of the tile's unit lower factor (the solves
    multiply by it): X L_II = I.  On the tile-step levels (the coarsest
    block, and levels with few blocks) X's diagonal 16 x 16 blocks come from
    the diagonal kernel and the rest from the fill launch after the steps."""
    T = P.msp.MSP_TILE
    for l in range(len(case.levels)):
        coarse = l == len(case.levels) - 1
        ns = 1 if coarse else case.o.get("n_subs", l)
        for p in sorted(set([0, ns - 1])):
            sub = -1 if coarse else p
            flat = case.inst.array(l, "factor", sub)
            first = P.msp.tile_first_of(case.h, l, sub)
            t = 0
            for I in range(len(first)):
                t += I - int(first[I])  # the tiles left of the diagonal
                tile = flat[t * T * T:(t + 1) * T * T].reshape(T, T)
                t += 1
                Lii = np.tril(tile, -1) + np.eye(T)
                X = np.triu(tile, 1).T + np.eye(T)
                err = np.max(np.abs(X @ Lii - np.eye(T)))
                assert err <= 1e-12 * max(1.0, np.max(np.abs(X))) * max(1.0, np.max(np.abs(Lii))), (l, p, I, err)
            assert t * T * T == flat.size


def test_ras_and_coarse_solve(case, P):
    rng = np.random.default_rng(2)
    m = P.msp
    L = len(case.levels)
    for l in range(L - 1):
        r = rng.normal(size=case.n[l])
        z = case.zeros(case.n[l])
        case.inst.apply_op(m.MSP_OP_RAS, l, case.dev(r), z)
        assert close(case.host(z), case.o.ras_apply(r, l), OP_TOL)
    r = rng.normal(size=case.n[-1])
    z = case.zeros(case.n[-1])
    case.inst.apply_op(m.MSP_OP_COARSE, L - 1, case.dev(r), z)
    assert close(case.host(z), case.o.coarse_solve(r), OP_TOL)


def test_vcycle(case):
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.normal(size=case.n[0])
        z = case.zeros(case.n[0])
        case.inst.apply(case.dev(r), z)
        assert close(case.host(z), case.o.vcycle(r), OP_TOL)


def test_fgmres_solution(case):
    rtol = 1e-10
    xo, so = case.o.fgmres(rtol=rtol, restart=case.w["restart"])
    x = case.zeros(case.n[0])
    st = case.inst.solve(x, rtol=rtol)
    assert st["status"] == 0 and st["rel_residual"] <= rtol
    assert abs(st["iterations"] - so["iters"]) <= 1
    assert close(case.host(x), xo, 1e-7)
    # user right-hand side through the same call
    b = np.random.default_rng(4).normal(size=case.n[0])
    b[case.dir0 == 1] = 0.0
    xb = case.zeros(case.n[0])
    st = case.inst.solve(xb, b=case.dev(b), rtol=rtol)
    xob, _ = case.o.fgmres(b, rtol=rtol, restart=case.w["restart"])
    assert st["status"] == 0 and rel(case.host(xb), xob) <= 1e-7


def test_solve_host_end_to_end(case):
    """The host-buffer entry point: re-assemble, factor, solve, copy back."""
    x = np.zeros(case.n[0])
    mu2 = syn.mu_draw(17)
    st = case.inst.solve_host(mu2, x, rtol=1e-10)
    case.o.assemble(mu2)
    case.o.factor()
    xo, _ = case.o.fgmres(rtol=1e-10, restart=case.w["restart"])
    assert st["status"] == 0 and rel(x, xo) <= 1e-7
    # back to the fixture's parameter for the other tests of this module
    case.o.assemble(case.mu)
    case.o.factor()
    case.inst.reassemble(case.mu)
    case.inst.factor()


def test_elasticity_fp32_factors(P, orc, torch):
    """Three displacement fields per vertex with FP32 subdomain factors under
    the FP64 outer loop: the FP64 oracle's solution, at most 3 more
    iterations; the load is the unit body force along -z."""
    levels, w = workload("elast12_3lvl")
    mu = syn.mu_draw(5)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10, restart=w["restart"])
    h = make_hierarchy(levels, w, P, precision="f32")
    assert h.n_dofs(0) == 3 * levels[0].n_nodes
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= so["iters"] + 3
    b = h.array(0, "load").reshape(-1, 3)
    assert not b[:, :2].any() and (b[:, 2] <= 0).all() and (b[:, 2] < 0).any()


# ------------------------------------------------------------- edge cases
def test_p2_fp32_factors(P, orc, torch):
    """Quadratic elements with FP32 subdomain factors under the FP64 outer
    loop: the FP64 oracle's solution at rtol 1e-10, at most 3 more iterations."""
    levels, w = workload("p2cube12_3lvl")
    mu = syn.mu_draw(6)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10, restart=w["restart"])
    h = make_hierarchy(levels, w, P, precision="f32")
    assert h.n_dofs(0) == o.n[0] == (2 * levels[0].n + 1) ** 3
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(o.n[0], dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and st["iterations"] <= so["iters"] + 3
    assert close(x.cpu().numpy(), xo, 1e-7)


def test_single_level_is_a_direct_solve(P, orc, torch):
    lv = syn.cube_level(6, 9)
    w = dict(delta=1, nu=2, coef="cosexp", scale=1.0, load="one", restart=30)
    h = make_hierarchy([lv], w, P)
    mu = syn.mu_draw(3)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(lv.n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-12)
    assert st["iterations"] == 1
    o = make_oracle([lv], w, orc)
    o.assemble(mu)
    o.factor()
    xo, _ = o.fgmres(rtol=1e-12)
    assert close(x.cpu().numpy(), xo, 1e-10)


@pytest.mark.parametrize("delta,nu_pre,nu_post", [(0, 1, 1), (1, 0, 2), (3, 3, 1)])
def test_overlap_and_smoothing_variants(P, orc, torch, delta, nu_pre, nu_post):
    """No overlap (block Jacobi smoother), no pre-smoothing, asymmetric counts."""
    levels = syn.hierarchy((10, 5), ((3, 2, 2),))
    w = dict(delta=delta, nu=1, coef="cosexp", scale=1.0, load="one", restart=20)
    o = orc.Oracle(levels, delta=delta, nu_pre=nu_pre, nu_post=nu_post, coef="cosexp",
                   wave=syn.wave_vectors(), load="one")
    mu = syn.mu_draw(8)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, w, P, nu_pre=nu_pre, nu_post=nu_post)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    r = np.random.default_rng(5).normal(size=levels[0].n_nodes)
    z = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    inst.apply(torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), o.vcycle(r), OP_TOL)
    x = torch.zeros_like(z)
    st = inst.solve(x, rtol=1e-10)
    xo, so = o.fgmres(rtol=1e-10, restart=20)
    assert st["status"] == 0 and so["status"] == 0
    assert close(x.cpu().numpy(), xo, 1e-7)


def test_zero_rhs_and_bad_inputs(P, torch):
    levels, w = workload("cube8_2lvl")
    h = make_hierarchy(levels, w, P)
    inst = h.assemble(np.zeros(8), stream=torch.cuda.current_stream())
    n = levels[0].n_nodes
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.MspError):  # not factored yet
        inst.solve(x)
    inst.factor()
    st = inst.solve(x, b=torch.zeros_like(x))
    assert st["status"] == 0 and st["iterations"] == 0 and not x.any()
    h2 = make_hierarchy(*workload("cube16_3lvl"), P)
    with pytest.raises(P.MspError) as e:
        h2.assemble(np.array([np.nan] + [0.0] * 7), stream=torch.cuda.current_stream())
    assert e.value.code == P.msp.MSP_ERR_INVALID
    with pytest.raises(P.MspError):  # aliasing input and output
        inst.apply(x, x)


def test_memory_budget_refuses_instances(P, torch):
    levels, w = workload("cube8_2lvl")
    h = make_hierarchy(levels, w, P, budget_bytes=1)
    with pytest.raises(P.MspError) as e:
        h.assemble(np.zeros(8), stream=torch.cuda.current_stream())
    assert e.value.code == P.msp.MSP_ERR_OOM


def test_not_converged_reports_partial_stats(P, torch):
    levels, w = workload("cube16_3lvl")
    h = make_hierarchy(levels, w, P, max_it=2)
    inst = h.assemble(syn.mu_draw(1), stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-14, raise_on_fail=False)
    assert st["status"] == P.msp.MSP_ERR_NOT_CONVERGED and st["iterations"] == 2
    assert 0 < st["rel_residual"] < 1


def test_fp32_factors_reach_fp64_accuracy(P, orc, torch):
    """FP32 subdomain factors under the FP64 outer loop: same tolerance on x."""
    levels, w = workload("cube16_3lvl")
    mu = syn.mu_draw(2)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10)
    h = make_hierarchy(levels, w, P, precision="f32")
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= so["iters"] + 3
    # the smoother really runs in FP32: one RAS application differs from the
    # FP64 one at single-precision level, not at double-precision level
    r = np.random.default_rng(6).normal(size=levels[0].n_nodes)
    z = torch.zeros_like(x)
    inst.apply_op(P.msp.MSP_OP_RAS, 0, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    d = rel(z.cpu().numpy(), o.ras_apply(r, 0))
    assert 1e-10 < d < 1e-4, d
    fac = inst.array(0, "factor", 0, dtype=np.float32)
    Lg, dg = P.msp.unpack_factor(fac.astype(np.float64), o.get("sub_dofs", 0, 0).size,
                                 P.msp.tile_first_of(h, 0, 0))
    n0 = o.get("sub_dofs", 0, 0).size
    do = np.diag(o.get("sub_lu", 0, 0).reshape(n0, n0))
    assert 1e-12 < rel(dg, do) < 1e-5


@pytest.mark.parametrize("scaling", [True, False])
def test_mls_with_fp32_factors(P, orc, torch, scaling):
    """MLS transfers (both restriction scalings) with FP32 subdomain factors:
    the FP64 outer loop still reaches the FP64 oracle's solution."""
    levels, w = workload("cube20m_3lvl")
    mu = syn.mu_draw(6)
    o = make_oracle(levels, w, orc, transfer="mls", restrict_scaling=scaling)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10)
    h = make_hierarchy(levels, w, P, precision="f32", transfer="mls", restrict_scaling=scaling)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= so["iters"] + 3


def _bf16_rne(f32):
    """Round float32 to BF16 (nearest, ties to even) as uint16, numpy only."""
    u = np.ascontiguousarray(f32, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def test_bf16_factors(P, orc, torch):
    """BF16 factor storage (factored in FP32, rounded to nearest even), FP32
    accumulation in the solves, FP64 outer loop: the solution still matches
    the FP64 oracle's; the stored factors are exactly the rounded FP32 ones."""
    levels, w = workload("cube16_3lvl")
    mu = syn.mu_draw(2)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10)
    h = make_hierarchy(levels, w, P, precision="bf16")
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= 4 * so["iters"] + 4
    # the stored factor of every sampled block = RNE(FP32 factor)
    h32 = make_hierarchy(levels, w, P, precision="f32")
    i32 = h32.assemble(mu, stream=torch.cuda.current_stream())
    i32.factor()
    for l in range(len(levels) - 1):
        ns = o.get("n_subs", l)
        for p in sorted({0, ns // 2, ns - 1}):
            f32 = i32.array(l, "factor", p, dtype=np.float32)
            b16 = inst.array(l, "factor", p, dtype=np.uint16)
            np.testing.assert_array_equal(b16, _bf16_rne(f32))
    # the smoother really runs on BF16 data
    r = np.random.default_rng(6).normal(size=levels[0].n_nodes)
    z = torch.zeros_like(x)
    inst.apply_op(P.msp.MSP_OP_RAS, 0, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    d = rel(z.cpu().numpy(), o.ras_apply(r, 0))
    assert 1e-6 < d < 0.5, d


def test_bf16_tensor_core_factorisation(P, orc, torch):
    """Levels with many blocks factor BF16 hierarchies in the persistent kernel
    whose trailing updates run on the tensor cores (BF16 operands, FP32
    accumulation): factors within BF16 accuracy of the blocks, close to the
    rounded FP32 factors, and the FP64 outer loop reaches the oracle's x."""
    levels = syn.hierarchy((20, 10, 5), ((5, 5, 4), (5, 5, 4)))
    w = dict(delta=2, nu=2, coef="cosexp", scale=1.0, load="one", restart=30)
    mu = syn.mu_draw(7)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, so = o.fgmres(rtol=1e-10)
    h = make_hierarchy(levels, w, P, precision="bf16")
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.profile_enable(P.msp.KERNEL_CLASSES)
    inst.factor()
    prof = inst.profile()
    assert prof["ldlt_blocks"]["launches"] == 2  # both smoothed levels, one launch each
    h32 = make_hierarchy(levels, w, P, precision="f32")
    i32 = h32.assemble(mu, stream=torch.cuda.current_stream())
    i32.factor()
    for l in range(2):
        ns = o.get("n_subs", l)
        assert ns >= 76  # at least half the SMs: the persistent path
        for p in sorted({0, ns // 3, ns - 1}):
            dofs = o.get("sub_dofs", l, p)
            n = dofs.size
            first = P.msp.tile_first_of(h, l, p)
            Lg, dg = P.msp.unpack_factor(inst.array(l, "factor", p, dtype="bf16").astype(np.float64),
                                         n, first)
            A = o.csr(l).toarray()[np.ix_(dofs, dofs)]
            err = np.linalg.norm(Lg @ np.diag(dg) @ Lg.T - A) / np.linalg.norm(A)
            assert err < 3e-2, err
            L32, d32 = P.msp.unpack_factor(i32.array(l, "factor", p, dtype=np.float32).astype(np.float64),
                                           n, first)
            assert rel(dg, d32) < 3e-2
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= so["iters"] + 3


# ------------------------------------------------------- ILU(p) subdomains
@pytest.mark.parametrize("name,ilu", [("cube16_3lvl", (2, 0)), ("cube20_3lvl", (1, 1)),
                                      ("cube20m_3lvl", (0, 2)), ("cube16_3lvl", (3, 0))])
def test_ilu_subdomain_solver(P, orc, torch, name, ilu):
    """ILU(p) subdomain factors (Section 4.4): L and D of every block, the RAS
    application, the V-cycle and the FGMRES solution against the oracle.
    ILU(3) on the 16^3 mesh has rows of up to 51 strictly-lower entries, past
    the 32 of the lane-per-entry factorisation: it covers the other form."""
    levels, w = workload(name)
    mu = syn.mu_draw(4)
    o = make_oracle(levels, w, orc, ilu=ilu)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, w, P, ilu=ilu)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    m = P.msp
    rng = np.random.default_rng(8)
    for l in range(len(levels) - 1):
        ptr, sptr = h.array(l, "ilu_ptr"), h.array(l, "sub_ptr")
        Lg, Dg = inst.array(l, "ilu_val"), inst.array(l, "ilu_d")
        ns = o.get("n_subs", l)
        for p in sorted({0, ns // 2, ns - 1}):
            fp, fc, fv = (o.get(k, l, p) for k in ("sub_ilu_ptr", "sub_ilu_col", "sub_ilu_val"))
            for i in range(fp.size - 1):
                sel = fc[fp[i]:fp[i + 1]] < i
                lo = fv[fp[i]:fp[i + 1]][sel]
                R = sptr[p] + i
                lg = Lg[ptr[R]:ptr[R + 1]]
                assert np.max(np.abs(lg - lo), initial=0.0) <= 1e-12 * max(1.0, np.max(np.abs(lo), initial=0.0))
                di = fv[fp[i]:fp[i + 1]][fc[fp[i]:fp[i + 1]] == i][0]
                assert abs(Dg[R] - di) <= 1e-12 * abs(di)
        r = rng.normal(size=levels[l].n_nodes)
        z = torch.zeros(levels[l].n_nodes, dtype=torch.float64, device="cuda")
        inst.apply_op(m.MSP_OP_RAS, l, torch.tensor(r, device="cuda"), z)
        torch.cuda.synchronize()
        assert close(z.cpu().numpy(), o.ras_apply(r, l), OP_TOL)
    r = rng.normal(size=levels[0].n_nodes)
    z = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    inst.apply(torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), o.vcycle(r), OP_TOL)
    x = torch.zeros_like(z)
    st = inst.solve(x, rtol=1e-10)
    xo, so = o.fgmres(rtol=1e-10, restart=w["restart"])
    assert st["status"] == 0 and so["status"] == 0
    assert abs(st["iterations"] - so["iters"]) <= 1
    assert close(x.cpu().numpy(), xo, 1e-7)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_ilu_fp32_factors(P, orc, torch, precision):
    """ILU(2)/ILU(0) factors computed and applied in FP32 (both reduced
    precisions store ILU levels in FP32) under the FP64 outer loop: the
    factors agree with the oracle's FP64 ILU at single-precision level, one
    RAS application too, and FGMRES reaches the FP64 oracle's solution."""
    levels, w = workload("cube16_3lvl")
    ilu = (2, 0)
    mu = syn.mu_draw(9)
    o = make_oracle(levels, w, orc, ilu=ilu)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, w, P, ilu=ilu, precision=precision)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    ptr, sptr = h.array(0, "ilu_ptr"), h.array(0, "sub_ptr")
    Lg = inst.array(0, "ilu_val", dtype=np.float32).astype(np.float64)
    Dg = inst.array(0, "ilu_d", dtype=np.float32).astype(np.float64)
    assert Lg.size == ptr[-1] and Dg.size == sptr[-1]
    for p in (0, o.get("n_subs", 0) - 1):
        fp, fc, fv = (o.get(k, 0, p) for k in ("sub_ilu_ptr", "sub_ilu_col", "sub_ilu_val"))
        lo, lg, do, dg = [], [], [], []
        for i in range(fp.size - 1):
            c, v = fc[fp[i]:fp[i + 1]], fv[fp[i]:fp[i + 1]]
            R = sptr[p] + i
            lo.append(v[c < i])
            lg.append(Lg[ptr[R]:ptr[R + 1]])
            do.append(v[c == i][0])
            dg.append(Dg[R])
        lo, lg = np.concatenate(lo), np.concatenate(lg)
        assert 1e-12 < rel(lg, lo) < 1e-4
        assert rel(np.array(dg), np.array(do)) < 1e-5
    r = np.random.default_rng(12).normal(size=levels[0].n_nodes)
    z = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    inst.apply_op(P.msp.MSP_OP_RAS, 0, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    d = rel(z.cpu().numpy(), o.ras_apply(r, 0))
    assert 1e-10 < d < 1e-4, d
    xo, so = o.fgmres(rtol=1e-10, restart=w["restart"])
    x = torch.zeros_like(z)
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0 and st["rel_residual"] <= 1e-10
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert st["iterations"] <= so["iters"] + 3


# ------------------------------------------- paper-literal Algorithm 2 options
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_paper_literal_algorithm2(P, orc, torch, precision):
    """Every level RAS-smoothed (the coarsest too, its = 3), MLS both ways with
    the interpolated residual, delta = 1: V-cycle and solution vs the oracle."""
    levels = syn.hierarchy((16, 8, 4), ((4, 4, 4), (4, 4, 4), (2, 2, 2)))
    kw = dict(delta=1, nu_pre=3, nu_post=3, coef="cosexp", wave=syn.wave_vectors(), load="one",
              transfer="mls", restrict_scaling=False, coarse="ras")
    mu = syn.mu_draw(21)
    o = orc.Oracle(levels, **kw)
    o.assemble(mu)
    o.factor()
    h = P.Hierarchy(levels, precision=precision, **kw)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    n = levels[0].n_nodes
    if precision == "f64":
        r = np.random.default_rng(22).normal(size=n)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        inst.apply(torch.tensor(r, device="cuda"), z)
        torch.cuda.synchronize()
        assert close(z.cpu().numpy(), o.vcycle(r), OP_TOL)
        # the coarsest level is a RAS level now: its smoother matches the oracle's
        rc = np.random.default_rng(23).normal(size=levels[2].n_nodes)
        zc = torch.zeros(levels[2].n_nodes, dtype=torch.float64, device="cuda")
        inst.apply_op(P.msp.MSP_OP_RAS, 2, torch.tensor(rc, device="cuda"), zc)
        torch.cuda.synchronize()
        assert close(zc.cpu().numpy(), o.ras_apply(rc, 2), OP_TOL)
        with pytest.raises(P.MspError):
            inst.apply_op(P.msp.MSP_OP_COARSE, 2, torch.tensor(rc, device="cuda"), zc)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    xo, so = o.fgmres(rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert close(x.cpu().numpy(), xo, 1e-7)
    assert abs(st["iterations"] - so["iters"]) <= (1 if precision == "f64" else 3)


def test_one_level_ras(P, orc, torch):
    """A single level with the coarsest smoothed once: one-level RAS (Eq. 7)."""
    lv = syn.cube_level(16, 31, parts=(4, 4, 4))
    kw = dict(delta=1, nu_pre=1, nu_post=0, coef="cosexp", wave=syn.wave_vectors(), load="one",
              coarse="ras")
    mu = syn.mu_draw(24)
    o = orc.Oracle([lv], **kw)
    o.assemble(mu)
    o.factor()
    h = P.Hierarchy([lv], **kw)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    r = np.random.default_rng(25).normal(size=lv.n_nodes)
    z = torch.zeros(lv.n_nodes, dtype=torch.float64, device="cuda")
    inst.apply(torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), o.ras_apply(r, 0), OP_TOL)
    x = torch.zeros_like(z)
    st = inst.solve(x, rtol=1e-10)
    xo, so = o.fgmres(rtol=1e-10)
    assert st["status"] == 0 and rel(x.cpu().numpy(), xo) <= 1e-7
    assert abs(st["iterations"] - so["iters"]) <= 1


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_factorisation_graph_replay_is_bitwise_the_same(P, torch, precision):
    """From its second call on the factorisation replays a captured CUDA graph
    (while no kernel class is timed): same factors bit for bit, same launch
    counts per factorisation."""
    levels = syn.hierarchy((16, 8, 4), ((4, 4, 4), (2, 2, 2)))
    w = dict(delta=2, nu=2, coef="cosexp", scale=1.0, load="one", restart=30)
    h = make_hierarchy(levels, w, P, precision=precision)
    inst = h.assemble(syn.mu_draw(3), stream=torch.cuda.current_stream())
    facs, counts = [], []
    for call in range(3):  # direct, capture + replay, replay
        inst.profile_reset()
        inst.factor()
        prof = inst.profile()
        counts.append({k: v["launches"] for k, v in prof.items()})
        dt = np.uint16 if precision == "bf16" else (np.float32 if precision == "f32" else np.float64)
        facs.append([inst.array(l, "factor", -1 if l == 2 else 0, dtype=dt if l < 2 else np.float64)
                     for l in range(3)])
    for call in (1, 2):
        assert counts[call] == counts[0]
        for a, b in zip(facs[0], facs[call]):
            np.testing.assert_array_equal(a, b)
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    assert inst.solve(x, rtol=1e-10)["status"] == 0


def test_spmv_schedules_are_tuned_and_stable(P, torch):
    """The SpMV lanes-per-row schedule of every operator is picked on the device
    at load time; a second load of the same meshes gets the same choices."""
    levels, w = workload("cube16_3lvl")
    h1 = make_hierarchy(levels, w, P)
    h2 = make_hierarchy(levels, w, P)
    for l in range(len(levels)):
        a, b = h1.info(l)["spmv_lanes"], h2.info(l)["spmv_lanes"]
        assert a == b
        assert a[0] in (1, 2, 4, 8, 16, 32)  # J: the four-entry form does not apply
        if l + 1 < len(levels):
            assert a[1] in (1, 2, 4, 8, 16, 32, 64) and a[2] in (1, 2, 4, 8, 16, 32)


@pytest.mark.parametrize("lanes", [1, 2, 4, 32, 64])
def test_every_spmv_schedule_matches_the_oracle(P, orc, torch, lanes, monkeypatch):
    """Each SpMV schedule, fixed through MSP_SPMV_LANES, on J, P and P^T of
    every level (1: one lane per row over shared-memory row blocks; 64: one
    thread per row of P's four-entry form), and a whole solve with it."""
    monkeypatch.setenv("MSP_SPMV_LANES", str(lanes))
    levels, w = workload("cube16_3lvl")
    mu = syn.mu_draw(7)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, w, P)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    m = P.msp
    rng = np.random.default_rng(31)
    dev = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    for l in range(len(levels)):
        lv = h.info(l)["spmv_lanes"]
        if lanes == 64:  # the four-entry form exists for P only; J and P^T keep their timed choice
            assert l + 1 == len(levels) or lv[1] == 64
        else:
            assert lv[0] == lanes and (l + 1 == len(levels) or lv[1] == lv[2] == lanes)
        x = rng.normal(size=o.n[l])
        y = torch.zeros(o.n[l], dtype=torch.float64, device="cuda")
        inst.apply_op(m.MSP_OP_SPMV, l, dev(x), y)
        torch.cuda.synchronize()
        assert close(y.cpu().numpy(), o.spmv(x, l), 1e-14)
        if l + 1 < len(levels):
            xc = rng.normal(size=o.n[l + 1])
            yf = torch.zeros(o.n[l], dtype=torch.float64, device="cuda")
            inst.apply_op(m.MSP_OP_INTERP, l, dev(xc), yf)
            yc = torch.zeros(o.n[l + 1], dtype=torch.float64, device="cuda")
            inst.apply_op(m.MSP_OP_RESTRICT, l, dev(x), yc)
            torch.cuda.synchronize()
            assert close(yf.cpu().numpy(), o.interp(xc, l), 1e-14)
            assert close(yc.cpu().numpy(), o.restrict(x, l), 1e-14)
    xs = torch.zeros(o.n[0], dtype=torch.float64, device="cuda")
    st = inst.solve(xs, rtol=1e-10)
    xo, _ = o.fgmres(rtol=1e-10, restart=w["restart"])
    assert st["status"] == 0 and rel(xs.cpu().numpy(), xo) <= 1e-7


def test_results_reproducible_bitwise(P, torch):
    levels, w = workload("cube16_3lvl")
    h = make_hierarchy(levels, w, P)
    inst = h.assemble(syn.mu_draw(5), stream=torch.cuda.current_stream())
    inst.factor()
    n = levels[0].n_nodes
    xs = []
    for _ in range(2):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        inst.solve(x, rtol=1e-10)
        xs.append(x.cpu().numpy())
    np.testing.assert_array_equal(xs[0], xs[1])
