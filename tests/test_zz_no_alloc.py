"""The allocation-free dot product (msp_multidot_noalloc) against the solver.

msp_multidot_noalloc serves callers that may not allocate device memory when
they need a result (for example code under a memory manager that owns all
device memory, or a real-time loop that cannot risk an allocation stalling or
failing).  It keeps its partial sums in a fixed device array instead and runs
the solver's own reduction kernels.  This test checks, through the C ABI,
that calls in a row reproduce bit for bit the relative residual that
msp_solve (the existing entry point using the same reduction) reports, that
repeated calls on the same inputs agree bit for bit, and that the results
agree with a plain reference within the tolerance of the other GPU tests.
It lives in its own file so that it is collected last.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, workload

pytestmark = pytest.mark.gpu


def test_noalloc_dot_matches_solver_residual():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08981_gb300 import build as b
    b.build()
    import paper_2412_08981_gb300 as P
    m = P.msp
    levels, w = workload("cube16_3lvl")
    h = make_hierarchy(levels, w, P)
    stream = torch.cuda.current_stream()
    inst = h.assemble(syn.mu_draw(11), stream=stream)
    inst.factor()
    n = levels[0].n_nodes
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0
    bvec = torch.tensor(h.array(0, "load"), device="cuda")
    r = bvec.clone()
    inst.apply_op(m.MSP_OP_RESIDUAL, 0, x, r)  # r = b - A x
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    # two calls in a row, sharing the fixed scratch array
    m.multidot_noalloc(r, r, out[0:1], stream=stream)
    m.multidot_noalloc(bvec, bvec, out[1:2], stream=stream)
    torch.cuda.synchronize()
    rr, bb = out.cpu().numpy()
    relres = np.sqrt(rr) / np.sqrt(bb)
    # the solver's own reduction of the same vectors: the same bits
    assert relres == st["rel_residual"], (relres, st["rel_residual"])
    # the same inputs again: bitwise the same results
    again = torch.empty(2, dtype=torch.float64, device="cuda")
    m.multidot_noalloc(r, r, again[0:1], stream=stream)
    m.multidot_noalloc(bvec, bvec, again[1:2], stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(again.cpu().numpy(), out.cpu().numpy())
    rh, bh = r.cpu().numpy(), bvec.cpu().numpy()
    assert abs(rr - rh @ rh) <= 1e-12 * (rh @ rh)
    assert abs(bb - bh @ bh) <= 1e-12 * (bh @ bh)
    # several vectors at once, against a plain reference
    V = torch.randn(5, n, dtype=torch.float64, device="cuda")
    o5 = torch.empty(5, dtype=torch.float64, device="cuda")
    m.multidot_noalloc(V, r, o5, stream=stream)
    torch.cuda.synchronize()
    ref = V.cpu().numpy() @ rh
    assert np.max(np.abs(o5.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    # sizes beyond the fixed array are refused with a clear error
    big = torch.empty(m.MSP_NOALLOC_MAX_VECTORS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.MspError) as e:
        m.multidot_noalloc(r, r, big, nv=m.MSP_NOALLOC_MAX_VECTORS + 1, ld=n)
    assert e.value.code == m.MSP_ERR_INVALID
