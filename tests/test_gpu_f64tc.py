"""FP64 factors with the panel and trailing products on the BF16 tensor cores
by exact digit slices (MSP_F64_TC).  On the levels factored in one persistent
launch, every product is computed from eight 7-bit digits per operand entry,
so the factors must match the FP64 oracle's at the FP64 tolerances (L within
1e-10 of max|L|, D within 1e-12, L D L^T = A_p within 1e-13) and the FP64
pipe's own factors to 1e-12 of the block's largest entry (D to 1e-13).  The coefficient spans
several orders of magnitude so that rows and columns of very different scale
meet in one product.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, make_oracle, rel

pytestmark = pytest.mark.gpu


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


# both smoothed levels have 100 blocks (at least half the SMs): the persistent path
LEVELS = dict(ns=(20, 10, 5), parts=((5, 5, 4), (5, 5, 4)))


@pytest.fixture(scope="module", params=[(1.0, 7), (3.0, 11)], ids=["scale1", "scale3"])
def setup(request, P, orc, torch):
    scale, mu_req = request.param
    levels = syn.hierarchy(LEVELS["ns"], LEVELS["parts"])
    w = dict(delta=2, nu=2, coef="cosexp", scale=scale, load="one", restart=30)
    mu = syn.mu_draw(mu_req)
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, w, P, precision="f64tc")
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.profile_enable(P.msp.KERNEL_CLASSES)
    inst.factor()
    prof = inst.profile()
    h64 = make_hierarchy(levels, w, P, precision="f64")
    i64 = h64.assemble(mu, stream=torch.cuda.current_stream())
    i64.factor()
    return dict(levels=levels, w=w, mu=mu, o=o, h=h, inst=inst, prof=prof, h64=h64, i64=i64)


def test_sliced_factors_match_the_oracle(setup, P):
    o, h, inst, i64 = setup["o"], setup["h"], setup["inst"], setup["i64"]
    assert setup["prof"]["ldlt_blocks"]["launches"] == 2  # both smoothed levels, one launch each
    for l in range(2):
        ns = o.get("n_subs", l)
        assert ns >= 76 and h.info(l)["fac_ctas"] > 0
        for p in sorted({0, ns // 3, ns // 2, ns - 1}):
            dofs = o.get("sub_dofs", l, p)
            n = dofs.size
            LU = o.get("sub_lu", l, p).reshape(n, n)
            Lo, do = np.tril(LU, -1) + np.eye(n), np.diag(LU)
            first = P.msp.tile_first_of(h, l, p)
            Lg, dg = P.msp.unpack_factor(inst.array(l, "factor", p), n, first)
            assert np.max(np.abs(Lg - Lo)) <= 1e-10 * max(1.0, np.max(np.abs(Lo)))
            assert rel(dg, do) <= 1e-12
            A = o.csr(l).toarray()[np.ix_(dofs, dofs)]
            assert np.linalg.norm(Lg @ np.diag(dg) @ Lg.T - A) <= 1e-13 * np.linalg.norm(A)
            L64, d64 = P.msp.unpack_factor(i64.array(l, "factor", p), n, first)
            assert np.max(np.abs(Lg - L64)) <= 1e-12 * max(1.0, np.max(np.abs(L64)))
            assert rel(dg, d64) <= 1e-13


def test_sliced_factors_every_block_against_fp64(setup, P):
    """Every block of both levels: the whole factor storage against the FP64
    pipe's, entry by entry, relative to the largest entry of its block."""
    h, inst, i64, o = setup["h"], setup["inst"], setup["i64"], setup["o"]
    for l in range(2):
        for p in range(o.get("n_subs", l)):
            a, b = inst.array(l, "factor", p), i64.array(l, "factor", p)
            assert a.shape == b.shape
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), (l, p)


def test_sliced_ras_and_solution(setup, P, torch):
    o, h, inst = setup["o"], setup["h"], setup["inst"]
    n0 = o.n[0]
    r = np.random.default_rng(3).normal(size=n0)
    z = torch.zeros(n0, dtype=torch.float64, device="cuda")
    inst.apply_op(P.msp.MSP_OP_RAS, 0, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), o.ras_apply(r, 0)) <= 1e-12
    xo, so = o.fgmres(rtol=1e-10)
    x = torch.zeros(n0, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-7
    assert abs(st["iterations"] - so["iters"]) <= 1


def test_sliced_factorisation_graph_replay_and_batch_refusal(setup, P, torch):
    """Re-factoring (the second call replays a CUDA graph) gives the same
    factors bit for bit; msp_factor_batch refuses these hierarchies."""
    h, inst = setup["h"], setup["inst"]
    a = inst.array(0, "factor", 5).copy()
    inst.factor()
    inst.factor()
    np.testing.assert_array_equal(inst.array(0, "factor", 5), a)
    with pytest.raises(P.MspError):
        P.msp.factor_batch([inst], stream=torch.cuda.current_stream())
