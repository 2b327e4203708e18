"""The precision study at its full size: the 96^3 L-shaped domain (unit cube
minus [0.5,1]^3, 802,081 nodes) with 48^3/24^3/12^3 non-nested coarse levels,
2048 subdomains of 294-1320 DoFs, k(x;mu) spanning 1e-2 .. 1e2.  Subdomain
factors in FP64 (also with the products on the tensor cores by exact digit
slices), FP32 and BF16 (FP32 accumulation) under the FP64 outer
FGMRES to rtol 1e-10, each against the FP64 oracle's solution: a seeded
sample of 1024 entries with its norm and iteration count, written by
tests/golden/make_lshape96.py from the oracle alone.
"""
import os

import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lshape96_4lvl_oracle.txt")


def read_golden(path=GOLDEN):
    meta, idx, val = {}, [], []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            a, b = line.split()
            if a.isdigit():
                idx.append(int(a))
                val.append(float(b))
            else:
                meta[a] = float(b)
    return meta, np.array(idx), np.array(val)


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
def study():
    levels, w = workload("lshape96_4lvl")
    meta, idx, val = read_golden()
    assert int(meta["n"]) == levels[0].n_nodes and idx.size == int(meta["samples"])
    return levels, w, meta, idx, val


@pytest.mark.parametrize("precision", ["f64", "f64tc", "f32", "bf16"])
def test_precision_study_against_the_oracle(P, torch, study, precision):
    levels, w, meta, idx, val = study
    h = make_hierarchy(levels, w, P, precision=precision)
    assert h.info(0)["n_sub"] == 2048
    inst = h.assemble(syn.mu_draw(0), stream=torch.cuda.current_stream())
    inst.factor()
    x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=w["rtol"])
    xg = x.cpu().numpy()
    assert st["status"] == 0 and st["rel_residual"] <= w["rtol"]
    err = np.linalg.norm(xg[idx] - val) / np.linalg.norm(val)
    assert err <= 1e-7, err
    assert abs(np.linalg.norm(xg) - meta["norm2_x"]) <= 1e-7 * meta["norm2_x"]
    it_o = int(meta["iterations"])
    if precision in ("f64", "f64tc"):  # FP64-class factors: the oracle's iteration count
        assert abs(st["iterations"] - it_o) <= 1
    else:  # the reduced-precision smoother may cost a few iterations, never accuracy
        assert st["iterations"] <= it_o + 3
