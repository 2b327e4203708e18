"""Work placement of the per-SM work lists.

The persistent FP64 factorisation and the staged RAS solves split their
blocks into lists per SM, and a CTA takes the list of the SM it runs on.
Lists that no CTA of their own SM takes must still be taken exactly once:
for the factorisation, a list whose SM the launch does not reach; for the RAS
solve, a list left when an SM holds fewer CTAs than its share while another
holds more.  msp_debug_spread_work makes half of the lists such lists (twice
as many as SMs), so both fallbacks run on every launch.  The blocks'
arithmetic does not depend on the CTA that takes them, so the factors, the
solution and the iteration count must be bitwise those of the normal
placement, and the solution must still meet its tolerance against the
system.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, workload

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


def test_spread_work_lists_are_bitwise_the_same(P, torch):
    # 343 blocks on each smoothed level: the FP64 factorisation runs one
    # persistent launch over both levels, and level 0's RAS solve has a list
    # per CTA of every SM
    levels, w = workload("cube48_3lvl")
    h = make_hierarchy(levels, w, P)
    assert h.info(0)["ras_ctas"] > 0
    inst = h.assemble(syn.mu_draw(7), stream=torch.cuda.current_stream())
    n = h.n_dofs(0)
    samples = [(0, 0), (0, 171), (0, 342), (1, 5), (1, 300)]

    def run():
        inst.factor()
        inst.factor()  # the second from the factorisation graph
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = inst.solve(x)
        torch.cuda.synchronize()
        return x.cpu().numpy(), st, [inst.array(l, "factor", sub=p) for l, p in samples]

    x0, st0, f0 = run()
    inst.spread_work(True)
    x1, st1, f1 = run()
    inst.spread_work(False)
    x2, st2, _ = run()
    assert st0["status"] == st1["status"] == 0
    assert st0["iterations"] == st1["iterations"] == st2["iterations"]
    assert st1["rel_residual"] <= 1e-8
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(x0, x2)
    for a, b in zip(f0, f1):
        np.testing.assert_array_equal(a, b)


def test_narrow_cluster_form_of_the_coarsest_solve(P, torch, orc):
    # the coarsest solve takes clusters of 16 CTAs where the GPU places them,
    # else 8; both forms against a sparse LU of the oracle's coarsest matrix,
    # on a coarsest block of 21 tile rows whose band reaches three tiles back
    import scipy.sparse.linalg as spla
    from _common import make_oracle, relmax
    levels, w = workload("cube48_3lvl")
    h = make_hierarchy(levels, w, P)
    mu = syn.mu_draw(11)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    L = len(levels) - 1
    oc = make_oracle([levels[L]], w, orc)
    oc.assemble(mu)
    Ac = oc.csr(0)
    lu = spla.splu(Ac.tocsc())
    rng = np.random.default_rng(13)
    for narrow in (False, True, False):
        inst.spread_work(False, narrow_cluster=narrow)
        for _ in range(4):
            r = rng.normal(size=Ac.shape[0])
            z = torch.zeros(Ac.shape[0], dtype=torch.float64, device="cuda")
            inst.apply_op(P.msp.MSP_OP_COARSE, L, torch.tensor(r, device="cuda"), z)
            torch.cuda.synchronize()
            assert relmax(z.cpu().numpy(), lu.solve(r)) <= 1e-11
    inst.spread_work(False)
