"""Serving layer (msp_server_*): continuous batching over resident hierarchies.

Each result must be the same computed alone and in a mix of concurrent
requests (the slots use fixed-order reductions and do not share state), must
agree with the oracle, and admission must respect the device-memory budget.
"""
import time

import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, make_oracle, rel, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08981_gb300 import build as b
    b.build()
    import paper_2412_08981_gb300 as P
    hs = {}
    for name in ("cube16_3lvl", "cube8_2lvl"):
        levels, w = workload(name)
        hs[name] = (levels, w, make_hierarchy(levels, w, P, precision="f32" if name == "cube16_3lvl" else "f64"))
    return torch, P, hs


def alone(P, h, levels, mu, rtol):
    inst = h.assemble(mu)
    x = np.zeros(levels[0].n_nodes)
    st = inst.solve_host(mu, x, rtol=rtol)
    inst.close()
    assert st["status"] == 0
    return x


def test_results_same_alone_and_in_the_mix(env, orc):
    torch, P, hs = env
    names = list(hs)
    jobs = [(names[i % 2], syn.mu_draw(300 + i)) for i in range(10)]
    ref = [alone(P, hs[n][2], hs[n][0], mu, 1e-10) for n, mu in jobs]
    srv = P.Server(slots_per_hierarchy=3)
    ids = {n: srv.add(hs[n][2]) for n in names}
    rids = [srv.submit(ids[n], mu, rtol=1e-10) for n, mu in jobs]
    for (n, mu), rid, xr in zip(jobs, rids, ref):
        x = np.zeros(hs[n][0][0].n_nodes)
        rc, st = srv.poll(rid, x, timeout_ms=-1)
        assert rc == 0 and st["status"] == 0 and st["rel_residual"] <= 1e-10
        assert st["ms_total"] >= st["ms_queue"] >= 0
        np.testing.assert_array_equal(x, xr)  # bitwise: independent of the mix
    srv.close()
    # and one of them against the oracle
    n, mu = jobs[1]
    levels, w, _ = hs[n]
    o = make_oracle(levels, w, orc)
    o.assemble(mu)
    o.factor()
    xo, _ = o.fgmres(rtol=1e-10, restart=w["restart"])
    assert rel(ref[1], xo) <= 1e-7


def test_admission_by_memory_budget(env):
    torch, P, hs = env
    levels, w, h = hs["cube8_2lvl"]
    one = h.instance_bytes()
    srv = P.Server(slots_per_hierarchy=4, budget_bytes=int(one * 1.5))  # room for one slot
    hid = srv.add(h)
    rids = [srv.submit(hid, syn.mu_draw(400 + i)) for i in range(4)]
    stats = []
    for rid in rids:
        rc, st = srv.poll(rid, None, timeout_ms=-1)
        assert rc == 0
        stats.append(st)
    # served one after another by the single admitted slot: later ones queued
    assert max(s["ms_queue"] for s in stats[1:]) > 0.0
    srv.close()
    tiny = P.Server(slots_per_hierarchy=2, budget_bytes=max(1, one // 4))
    with pytest.raises(P.MspError) as e:
        tiny.add(h)
    assert e.value.code == P.msp.MSP_ERR_OOM
    tiny.close()


def test_poll_pending_and_errors(env):
    torch, P, hs = env
    levels, w, h = hs["cube16_3lvl"]
    srv = P.Server(slots_per_hierarchy=1)
    hid = srv.add(h)
    rid = srv.submit(hid, syn.mu_draw(500), rtol=1e-12)
    rc, st = srv.poll(rid, None, timeout_ms=0)
    assert rc in (P.msp.MSP_PENDING, 0)
    if rc == P.msp.MSP_PENDING:
        rc, st = srv.poll(rid, None, timeout_ms=-1)
    assert rc == 0
    with pytest.raises(P.MspError):
        srv.poll(rid, None, timeout_ms=0)  # already collected
    with pytest.raises(P.MspError):
        srv.submit(7, syn.mu_draw(1))
    srv.close()
