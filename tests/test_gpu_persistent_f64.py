"""Parity of the dominant FP64 kernel with the oracle, block by block.

With FP64 factors the smoothed levels that have at least half as many blocks
as the GPU has SMs are factored by one persistent launch over the blocks of
all of them (k_ldlt_blocks_batch).  This workload gives both smoothed levels
100 blocks (20^3 / 10^3 lattices cut into 5 x 5 x 4 boxes, overlap 2), so
both go through that launch, while the oracle still factors every block in
seconds.  Every block of both levels is compared with the oracle's Doolittle
LU (U = D L^T) entry by entry -- max |L - L_o| <= 1e-10 max(1, max |L_o|),
max |D - D_o| <= 1e-12 max |D_o|, and L D L^T reproduces the block to 1e-13 --
then the RAS application of both levels, the V-cycle and the FGMRES solution,
each both norm-wise and element-wise.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import close, make_hierarchy, make_oracle, rel, relmax

pytestmark = pytest.mark.gpu

LEVELS = dict(ns=(20, 10, 5), parts=((5, 5, 4), (5, 5, 4)))
W = dict(delta=2, nu=2, coef="cosexp", scale=1.0, load="one", restart=30)


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
def setup(P, orc, torch):
    levels = syn.hierarchy(LEVELS["ns"], LEVELS["parts"])
    mu = syn.mu_draw(23)
    o = make_oracle(levels, W, orc)
    o.assemble(mu)
    o.factor()
    h = make_hierarchy(levels, W, P, precision="f64")
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.profile_enable(P.msp.KERNEL_CLASSES)
    inst.factor()
    prof = inst.profile()
    inst.profile_enable([])
    return dict(levels=levels, o=o, h=h, inst=inst, prof=prof)


def test_both_levels_take_the_persistent_launch(setup):
    h, prof = setup["h"], setup["prof"]
    assert h.info(0)["fac_ctas"] > 0 and h.info(1)["fac_ctas"] > 0
    assert h.info(0)["n_sub"] == 100 and h.info(1)["n_sub"] == 100
    # one persistent launch for the blocks of both levels
    assert prof["ldlt_blocks"]["launches"] == 1


@pytest.mark.parametrize("level", [0, 1])
def test_every_block_matches_the_oracle(setup, P, level):
    o, h, inst = setup["o"], setup["h"], setup["inst"]
    ns = o.get("n_subs", level)
    A_all = o.csr(level).tocsr()
    worst_l = worst_d = worst_a = 0.0
    for p in range(ns):
        dofs = o.get("sub_dofs", level, p)
        n = dofs.size
        LU = o.get("sub_lu", level, p).reshape(n, n)
        Lo, do = np.tril(LU, -1) + np.eye(n), np.diag(LU)
        Lg, dg = P.msp.unpack_factor(inst.array(level, "factor", p), n, P.msp.tile_first_of(h, level, p))
        el = np.max(np.abs(Lg - Lo)) / max(1.0, np.max(np.abs(Lo)))
        ed = relmax(dg, do)
        A = A_all[dofs][:, dofs].toarray()
        ea = np.linalg.norm(Lg @ np.diag(dg) @ Lg.T - A) / np.linalg.norm(A)
        worst_l, worst_d, worst_a = max(worst_l, el), max(worst_d, ed), max(worst_a, ea)
        assert el <= 1e-10 and ed <= 1e-12 and ea <= 1e-13, (level, p, el, ed, ea)
    print(f"level {level}: {ns} blocks, worst L {worst_l:.2e}, D {worst_d:.2e}, LDL^T {worst_a:.2e}")


def test_ras_vcycle_and_solution(setup, P, torch):
    o, inst = setup["o"], setup["inst"]
    rng = np.random.default_rng(5)
    for level in (0, 1):
        r = rng.normal(size=o.n[level])
        z = torch.zeros(o.n[level], dtype=torch.float64, device="cuda")
        inst.apply_op(P.msp.MSP_OP_RAS, level, torch.tensor(r, device="cuda"), z)
        torch.cuda.synchronize()
        assert close(z.cpu().numpy(), o.ras_apply(r, level), 1e-12)
    r = rng.normal(size=o.n[0])
    z = torch.zeros(o.n[0], dtype=torch.float64, device="cuda")
    inst.apply(torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert close(z.cpu().numpy(), o.vcycle(r), 1e-12)
    xo, so = o.fgmres(rtol=1e-10)
    x = torch.zeros(o.n[0], dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and so["status"] == 0
    assert abs(st["iterations"] - so["iters"]) <= 1
    assert close(x.cpu().numpy(), xo, 1e-7), (rel(x.cpu().numpy(), xo), relmax(x.cpu().numpy(), xo))
