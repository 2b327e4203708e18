"""Failure paths that run on the GPU without faulting it, and pivots over
the whole double range.

* A bounded wait that runs out: msp_debug_expire_waits makes the next staged
  RAS application issue no tile copies, so its waits on the shared-memory
  ring expire after a short limit (no copy is ever in flight).  msp_solve must
  report MSP_ERR_TIMEOUT, and the same instance and a fresh one must then
  solve normally, bit for bit as before.
* Pivots outside the single-precision range: the factorisation's pivot
  reciprocals (correctly rounded, __drcp_rn) must hold there as anywhere,
  which an earlier single-precision-seeded form needed a guard for.  The
  meshes scaled by 2^133 and 2^-133 give pivots
  near 1e40 and 1e-40; since the scaling is by a power of two, the oracle's
  solution of the unscaled problem times 2^(2 * 133 * sign) is the exact
  solution of the scaled one (stiffness scales like the length, the load like
  its cube), and the GPU solution must match it at the FP64 tolerance.
"""
import copy

import numpy as np
import pytest

import synthetic as syn
from _common import close, make_hierarchy, make_oracle, rel, relmax, workload

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


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_expired_wait_is_reported_and_recovered(P, torch, precision):
    levels, w = workload("cube16_3lvl")
    h = make_hierarchy(levels, w, P, precision=precision)
    mu = syn.mu_draw(31)
    inst = h.assemble(mu, stream=torch.cuda.current_stream())
    inst.factor()
    n = h.n_dofs(0)
    x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    st0 = inst.solve(x0, rtol=1e-10)
    assert st0["status"] == 0
    ref = x0.cpu().numpy()
    inst.expire_waits(1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.MspError) as e:
        inst.solve(x, rtol=1e-10)
    assert e.value.code == P.msp.MSP_ERR_TIMEOUT
    # the same instance again: nothing was left behind
    st = inst.solve(x, rtol=1e-10)
    assert st["status"] == 0 and st["iterations"] == st0["iterations"]
    np.testing.assert_array_equal(x.cpu().numpy(), ref)
    # and a fresh instance of the same hierarchy
    i2 = h.assemble(mu, stream=torch.cuda.current_stream())
    i2.factor()
    x2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert i2.solve(x2, rtol=1e-10)["status"] == 0
    np.testing.assert_array_equal(x2.cpu().numpy(), ref)
    # a cancelled injection injects nothing
    inst.expire_waits(2)
    inst.expire_waits(0)
    assert inst.solve(x, rtol=1e-10)["status"] == 0
    with pytest.raises(P.MspError):
        inst.expire_waits(-1)


# both smoothed levels factored by the persistent launch (100 blocks each),
# and a coarsest block of two tiles (tile-step kernels)
LEVELS = dict(ns=(20, 10, 6), parts=((5, 5, 4), (5, 5, 4)))
W = dict(delta=2, nu=2, coef="const", scale=1.0, load="one", restart=30)


@pytest.fixture(scope="module")
def unscaled(orc):
    levels = syn.hierarchy(LEVELS["ns"], LEVELS["parts"])
    o = make_oracle(levels, W, orc)
    o.assemble(np.zeros(8))
    o.factor()
    xo, so = o.fgmres(rtol=1e-10)
    d0 = np.diag(o.get("sub_lu", 0, 0).reshape(o.get("sub_dofs", 0, 0).size, -1))
    return dict(levels=levels, xo=xo, so=so, d0=d0)


@pytest.mark.parametrize("e2", [133, -133])
def test_pivots_outside_the_float_range(P, torch, unscaled, e2):
    levels = copy.deepcopy(unscaled["levels"])
    s = 2.0 ** e2
    for lv in levels:
        lv.xyz = lv.xyz * s
    h = make_hierarchy(levels, W, P, precision="f64")
    assert h.info(0)["fac_ctas"] > 0 and h.info(1)["fac_ctas"] > 0
    inst = h.assemble(np.zeros(8), stream=torch.cuda.current_stream())
    inst.factor()
    # the pivots really are beyond the single-precision range
    n = int(h.array(0, "sub_ptr")[1])
    _, dg = P.msp.unpack_factor(inst.array(0, "factor", 0), n, P.msp.tile_first_of(h, 0, 0))
    d0 = unscaled["d0"] * s
    assert (np.min(np.abs(dg)) > 1e37) if e2 > 0 else (np.max(np.abs(dg)) < 1e-37)
    assert relmax(dg, d0) <= 1e-12
    x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
    st = inst.solve(x, rtol=1e-10)
    xs = unscaled["xo"] * (s * s)
    assert st["status"] == 0 and abs(st["iterations"] - unscaled["so"]["iters"]) <= 1
    xg = x.cpu().numpy()
    assert np.all(np.isfinite(xg))
    assert close(xg, xs, 1e-7), (rel(xg, xs), relmax(xg, xs))
