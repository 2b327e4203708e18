"""Batched factorisation (msp_factor_batch): the persistent-level blocks of
several instances, on hierarchies of different sizes, in one launch per
factor type.  Factors and solutions must be bitwise those of msp_factor on
each instance alone, in FP64 and FP32; BF16 batches and repeated instances
are refused.
"""
import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy

pytestmark = pytest.mark.gpu

# levels with more blocks than half the SMs take the persistent factorisation
UNEVEN = {
    "cube20b_3lvl": dict(ns=(20, 10, 5), parts=((5, 5, 4), (2, 2, 2)), delta=1, nu=2, coef="cosexp",
                         scale=1.0, load="one", rtol=1e-10, restart=30),
    "cube24b_3lvl": dict(ns=(24, 12, 6), parts=((6, 5, 5), (3, 3, 3)), delta=1, nu=2, coef="cosexp",
                         scale=1.0, load="one", rtol=1e-10, restart=30),
}


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


def _hier(P, name, precision):
    w = UNEVEN[name]
    levels = syn.hierarchy(w["ns"], w["parts"], hierarchy_id=3)
    return levels, make_hierarchy(levels, w, P, precision=precision)


def _snapshot(h, inst, dtype):
    out = []
    for l in range(h.nlevels):
        ns = h.info(l)["n_sub"]
        for p in sorted({0, max(ns // 2, 0), max(ns - 1, 0)}) if ns else [-1]:
            out.append(inst.array(l, "factor", p, dtype=np.float64 if l == h.nlevels - 1 else dtype))
    return out


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_is_bitwise_the_same_as_one_by_one(P, torch, precision):
    dtype = np.float64 if precision == "f64" else np.float32
    hs = [_hier(P, n, precision) for n in UNEVEN]
    for _, h in hs:
        assert h.info(0)["fac_ctas"] > 0  # level 0 is a persistent level: the batch path is exercised
    jobs = [(hs[k % 2], syn.mu_draw(700 + k)) for k in range(4)]
    stream = torch.cuda.current_stream()
    ref_f, ref_x = [], []
    for (levels, h), mu in jobs:
        inst = h.assemble(mu, stream=stream)
        inst.factor()
        ref_f.append(_snapshot(h, inst, dtype))
        x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
        assert inst.solve(x, rtol=1e-10)["status"] == 0
        ref_x.append(x.cpu().numpy())
        inst.close()
    for rep in range(2):  # twice: the work lists are rebuilt per call
        insts = [h.assemble(mu, stream=stream) for (_, h), mu in jobs]
        P.msp.factor_batch(insts, stream=stream)
        for k, ((levels, h), mu) in enumerate(jobs):
            for a, b in zip(_snapshot(h, insts[k], dtype), ref_f[k]):
                np.testing.assert_array_equal(a, b)
            x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
            assert insts[k].solve(x, rtol=1e-10)["status"] == 0
            np.testing.assert_array_equal(x.cpu().numpy(), ref_x[k])
        for i in insts:
            i.close()


def test_batch_refuses_bf16_and_repeats(P, torch):
    _, h = _hier(P, "cube20b_3lvl", "f64")
    _, hb = _hier(P, "cube20b_3lvl", "bf16")
    stream = torch.cuda.current_stream()
    a = h.assemble(syn.mu_draw(1), stream=stream)
    b = hb.assemble(syn.mu_draw(1), stream=stream)
    with pytest.raises(P.MspError):
        P.msp.factor_batch([a, b], stream=stream)
    with pytest.raises(P.MspError):
        P.msp.factor_batch([a, a], stream=stream)
    P.msp.factor_batch([a], stream=stream)  # a batch of one is msp_factor
    x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
    assert a.solve(x, rtol=1e-10)["status"] == 0


def test_instances_sharing_a_stream_across_threads(P, torch):
    """Two instances bound to ONE stream, driven from two host threads at once
    through reassemble / factor / solve, three parameters each: the second
    factorisation of each is captured into a CUDA graph while the other
    thread enqueues on the shared stream.  Solutions are bitwise those of
    the same instances run one after the other."""
    import threading
    _, h = _hier(P, "cube20b_3lvl", "f64")
    s = torch.cuda.Stream()
    mus = [[syn.mu_draw(900 + 10 * t + i) for i in range(3)] for t in range(2)]
    xs = [[torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda") for _ in range(3)] for _ in range(2)]
    torch.cuda.synchronize()  # the buffers exist before the other stream writes them
    ref = []
    for t in range(2):
        inst = h.assemble(mus[t][0], stream=s)
        out = []
        for i, mu in enumerate(mus[t]):
            inst.reassemble(mu)
            inst.factor()
            assert inst.solve(xs[t][i], rtol=1e-10)["status"] == 0
            out.append(xs[t][i].cpu().numpy())
        ref.append(out)
        inst.close()
    ys = [[torch.full_like(x, float("nan")) for x in row] for row in xs]
    insts = [h.assemble(mus[t][0], stream=s) for t in range(2)]
    torch.cuda.synchronize()
    got, errs = [[None] * 3 for _ in range(2)], []

    def worker(t):
        try:
            for i, mu in enumerate(mus[t]):
                insts[t].reassemble(mu)
                insts[t].factor()
                st = insts[t].solve(ys[t][i], rtol=1e-10)  # synchronises the shared stream
                got[t][i] = (st["status"], ys[t][i].cpu().numpy())
        except Exception as e:  # reported on the main thread
            errs.append(repr(e))
    th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errs, errs
    for t in range(2):
        for i in range(3):
            assert got[t][i][0] == 0
            np.testing.assert_array_equal(got[t][i][1], ref[t][i])
    for i in insts:
        i.close()
