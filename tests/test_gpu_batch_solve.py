"""Batched solves (msp_batch_*): the re-assembly, factorisation and FGMRES
solves of several instances -- of one hierarchy and of hierarchies of
different sizes and depths, in FP64, FP32 and BF16 factors -- with their
launches shared.  Each member's arithmetic is that of its own msp_reassemble,
msp_factor and msp_solve, so factors, solutions, iteration counts and
residuals must be bitwise the same as one by one; and one member is checked
against the FP64 oracle.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import close, make_hierarchy, make_oracle, workload

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


def members(P, torch, spec):
    """spec: list of (workload, precision, mu request, restart or None)."""
    hs, insts = [], []
    for name, prec, req, restart in spec:
        levels, w = workload(name)
        kw = {} if restart is None else dict(restart=restart)
        h = make_hierarchy(levels, w, P, precision=prec, **kw)
        inst = h.assemble(syn.mu_draw(req), stream=torch.cuda.Stream())
        inst.factor()
        hs.append(h)
        insts.append(inst)
    return hs, insts


def one_by_one(torch, hs, insts, rtol, bs=None):
    xs, sts = [], []
    for k, (h, inst) in enumerate(zip(hs, insts)):
        x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
        b = None if bs is None else bs[k]
        sts.append(inst.solve(x, b=b, rtol=rtol))
        xs.append(x.cpu().numpy())
    return xs, sts


SPECS = {
    # one hierarchy, four parameters
    "same": [("cube16_3lvl", "f64", r, None) for r in (1, 2, 3, 4)],
    # uneven sizes and depths, mixed factor precisions, a short restart
    "uneven": [("cube16_3lvl", "f64", 5, None), ("cube20_3lvl", "f32", 6, None), ("cube8_2lvl", "f64", 7, None),
               ("cube20_3lvl", "bf16", 8, None), ("cube16_3lvl", "f32", 9, 3), ("elast12_3lvl", "f64", 10, None)],
}


@pytest.mark.parametrize("which", sorted(SPECS))
def test_batch_is_bitwise_one_by_one(P, torch, which):
    hs, insts = members(P, torch, SPECS[which])
    rtol = 1e-10
    xs_ref, st_ref = one_by_one(torch, hs, insts, rtol)
    batch = P.msp.Batch(insts, stream=torch.cuda.Stream())
    xs = [torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda") for h in hs]
    st = batch.solve(xs, rtol=rtol)
    for k in range(len(hs)):
        assert st[k]["status"] == 0
        assert st[k]["iterations"] == st_ref[k]["iterations"], k
        assert st[k]["rel_residual"] == st_ref[k]["rel_residual"], k
        np.testing.assert_array_equal(xs[k].cpu().numpy(), xs_ref[k])
    # again (the batch is reusable): batched re-assembly and factorisation with
    # new parameters, twice (the second factorisation replays a CUDA graph);
    # the factors are bitwise those of msp_factor, the solutions those of msp_solve
    for rnd in range(2):
        batch.assemble([syn.mu_draw(100 + 10 * rnd + k) for k in range(len(insts))])
        batch.factor()
        fac_b = [[inst.array(0, "factor", 0, dtype=np.uint8), inst.array(h.nlevels - 1, "factor", -1, dtype=np.uint8)]
                 for h, inst in zip(hs, insts)]
        st = batch.solve(xs, rtol=rtol)
        for inst in insts:
            inst.factor()
        for k, (h, inst) in enumerate(zip(hs, insts)):
            np.testing.assert_array_equal(inst.array(0, "factor", 0, dtype=np.uint8), fac_b[k][0])
            np.testing.assert_array_equal(inst.array(h.nlevels - 1, "factor", -1, dtype=np.uint8), fac_b[k][1])
        xs_ref, st_ref = one_by_one(torch, hs, insts, rtol)
        for k in range(len(hs)):
            assert st[k]["iterations"] == st_ref[k]["iterations"]
            np.testing.assert_array_equal(xs[k].cpu().numpy(), xs_ref[k])
    batch.close()


def test_batch_user_rhs_and_the_oracle(P, orc, torch):
    hs, insts = members(P, torch, [("cube16_3lvl", "f64", 11, None), ("cube20_3lvl", "f64", 12, None)])
    rng = np.random.default_rng(4)
    bs = []
    for k, name in enumerate(("cube16_3lvl", "cube20_3lvl")):
        levels, w = workload(name)
        b = rng.normal(size=levels[0].n_nodes)
        b[levels[0].dirichlet == 1] = 0.0
        bs.append(torch.tensor(b, device="cuda") if k == 0 else None)  # member 1: its load vector
    xs_ref, st_ref = one_by_one(torch, hs, insts, 1e-10, bs=bs)
    batch = P.msp.Batch(insts)
    xs = [torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda") for h in hs]
    st = batch.solve(xs, bs=bs, rtol=1e-10)
    for k in range(2):
        assert st[k]["iterations"] == st_ref[k]["iterations"]
        np.testing.assert_array_equal(xs[k].cpu().numpy(), xs_ref[k])
    levels, w = workload("cube20_3lvl")
    o = make_oracle(levels, w, orc)
    o.assemble(syn.mu_draw(12))
    o.factor()
    xo, so = o.fgmres(rtol=1e-10, restart=w["restart"])
    assert close(xs[1].cpu().numpy(), xo, 1e-7)
    assert abs(st[1]["iterations"] - so["iters"]) <= 1


def test_batch_refusals(P, torch):
    levels, w = workload("cube16_3lvl")
    h = make_hierarchy(levels, w, P)
    inst = h.assemble(syn.mu_draw(1), stream=torch.cuda.current_stream())
    with pytest.raises(P.MspError):
        P.msp.Batch([inst, inst])  # listed twice
    hi = make_hierarchy(levels, w, P, ilu=(0, 0))
    ii = hi.assemble(syn.mu_draw(1), stream=torch.cuda.current_stream())
    with pytest.raises(P.MspError):
        P.msp.Batch([inst, ii])  # ILU levels
    hn = make_hierarchy(levels, w, P, nu_pre=1, nu_post=1)
    inn = hn.assemble(syn.mu_draw(1), stream=torch.cuda.current_stream())
    with pytest.raises(P.MspError):
        P.msp.Batch([inst, inn])  # different smoothing
    b = P.msp.Batch([inst])
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(P.MspError):
        b.solve([x])  # not factored yet
