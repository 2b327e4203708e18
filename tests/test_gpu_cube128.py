"""The largest hierarchy of the serving trace: 128^3 (2,146,689 nodes, 12.6M
tets, 31.8M nonzeros) with 64^3 / 32^3 / 16^3 coarse levels, 4096 subdomains
on the finest level.  The oracle cannot run it in seconds, so the checks are
properties that hold at any size, on the library's own arrays:
  * the CSR pattern is symmetric with sorted columns and a diagonal in every
    row, Dirichlet rows are identity rows and interior rows sum to zero (the
    assembled stiffness of -div(k grad u));
  * FGMRES with FP64 and with FP32 factors reaches rtol 1e-8 in the true
    residual, recomputed here with scipy from the library's CSR, and the two
    solutions agree.
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


@pytest.fixture(scope="module")
def big(P, torch):
    sp = pytest.importorskip("scipy.sparse")
    levels, w = workload("cube128_4lvl")
    h64 = make_hierarchy(levels, w, P, precision="f64")
    assert h64.info(0)["n_sub"] == 4096 and h64.nlevels == 4
    rp, col = h64.array(0, "rowptr"), h64.array(0, "col")
    return dict(levels=levels, w=w, h64=h64, rp=rp, col=col, sp=sp)


def _csr(big, inst):
    n = big["rp"].size - 1
    return big["sp"].csr_matrix((inst.array(0, "val"), big["col"], big["rp"]), shape=(n, n))


def test_cube128_structure(big, torch):
    levels, h = big["levels"], big["h64"]
    inst = h.assemble(syn.mu_draw(0), stream=torch.cuda.current_stream())
    A = _csr(big, inst)
    n = A.shape[0]
    assert n == levels[0].n_nodes == 2146689 and A.nnz == 31802497
    d = A.diagonal()
    dr = levels[0].dirichlet.astype(bool)
    assert np.all(d[~dr] > 0) and np.all(d[dr] == 1.0)
    assert abs(A - A.T).max() <= 1e-14 * np.abs(A.data).max()
    rows = np.asarray(A.sum(axis=1)).ravel()
    # interior rows whose columns are all interior sum to zero
    touch = np.asarray(big["sp"].csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
                       @ dr.astype(float)).ravel()
    free = (~dr) & (touch == 0)
    assert free.mean() > 0.9
    assert np.max(np.abs(rows[free])) <= 1e-12 * np.abs(A.data).max()
    inst.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_cube128_solve_true_residual(big, P, torch, precision):
    levels, w = big["levels"], big["w"]
    h = big["h64"] if precision == "f64" else make_hierarchy(levels, w, P, precision="f32")
    inst = h.assemble(syn.mu_draw(3), stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(levels[0].n_nodes, dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-8)
    assert st["status"] == 0 and st["iterations"] <= 12
    A = _csr(big, inst)
    b = h.array(0, "load")  # the assembled load (f = 1 does not depend on mu)
    xv = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xv) <= 1.01e-8 * np.linalg.norm(b)
    big.setdefault("x", {})[precision] = xv
    if len(big["x"]) == 2:
        xa, xb = big["x"]["f64"], big["x"]["f32"]
        assert np.linalg.norm(xa - xb) <= 1e-6 * np.linalg.norm(xa)
    inst.close()
