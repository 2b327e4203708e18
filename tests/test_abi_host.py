"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/msp.h declares, and its host-side set-up (CSR pattern, subdomains,
interpolation P and P^T) matches the oracle bit-exactly on the index
structures (values of P to 1e-13)."""
import os
import re
import subprocess

import numpy as np
import pytest

import synthetic as syn
from _common import make_hierarchy, make_oracle, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2412_08981_gb300 import build as b
    b.build()
    import paper_2412_08981_gb300 as pkg
    pkg.load()
    return pkg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "msp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(msp_\w+)\s*\(", src))
    # drop typedef'd function-pointer types
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol(P):
    lib = P.load()
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", P.msp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
    assert set(P.msp.EXPORTS) <= set(names)
    assert lib.msp_version().startswith(b"msp")


@pytest.mark.parametrize("name", ["cube8_2lvl", "cube16_3lvl", "cube20_3lvl"])
def test_host_structures_match_oracle(P, orc, name):
    levels, w = workload(name)
    h = make_hierarchy(levels, w, P, host_only=True)
    o = make_oracle(levels, w, orc)
    L = len(levels)
    for l in range(L):
        np.testing.assert_array_equal(h.array(l, "rowptr"), o.get("rowptr", l))
        np.testing.assert_array_equal(h.array(l, "col"), o.get("col", l))
    for l in range(L - 1):
        subs = o.subdomains(l)
        sp, sd, so = h.array(l, "sub_ptr"), h.array(l, "sub_dofs"), h.array(l, "sub_own")
        assert sp.size - 1 == len(subs)
        for p, (d, ow) in enumerate(subs):
            np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)
            np.testing.assert_array_equal(so[sp[p]:sp[p + 1]], ow)
        for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
            np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
        np.testing.assert_allclose(h.array(l, "P_val"), o.get("P_val", l), atol=1e-13)
        np.testing.assert_allclose(h.array(l, "PT_val"), o.get("PT_val", l), atol=1e-13)
    # coarsest block = all interior DoFs
    sd = h.array(L - 1, "sub_dofs")
    np.testing.assert_array_equal(sd, np.where(levels[-1].dirichlet == 0)[0])
    info = h.info(0)
    assert info["nnz"] == o.get("col", 0).size
    assert info["n_sub"] == o.get("n_subs", 0)


@pytest.mark.parametrize("name", ["cube8_2lvl", "cube16_3lvl", "cube20m_3lvl"])
@pytest.mark.parametrize("scaling", [True, False])
def test_host_mls_transfers_match_oracle(P, orc, name, scaling):
    """MLS weights (Section 3.2): same neighbourhoods bit-exactly, values to
    rounding; cube20m pairs subdomains across levels, the others do not."""
    levels, w = workload(name)
    h = make_hierarchy(levels, w, P, host_only=True, transfer="mls", restrict_scaling=scaling)
    o = make_oracle(levels, w, orc, transfer="mls", restrict_scaling=scaling)
    for l in range(len(levels) - 1):
        for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
            np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
        for a in ("P_val", "PT_val"):
            ref = o.get(a, l)
            np.testing.assert_allclose(h.array(l, a), ref, rtol=1e-12, atol=1e-13 * abs(ref).max())
        info = h.info(l)
        assert info["P_nnz"] == o.get("P_col", l).size and info["R_nnz"] == o.get("PT_col", l).size


def test_host_smoothed_coarsest_matches_oracle(P, orc):
    """MSP_COARSE_RAS: the coarsest level gets overlapping subdomains like the
    others (and needs an owner array)."""
    levels = syn.hierarchy((12, 6, 4), ((3, 3, 3), (3, 3, 3), (2, 2, 2)))
    h = P.Hierarchy(levels, delta=1, host_only=True, coarse="ras", transfer="mls",
                    restrict_scaling=False)
    o = orc.Oracle(levels, delta=1, coarse="ras", transfer="mls", restrict_scaling=False)
    for l in range(3):
        subs = o.subdomains(l)
        sp_, sd = h.array(l, "sub_ptr"), h.array(l, "sub_dofs")
        assert sp_.size - 1 == len(subs) and h.info(l)["n_sub"] == len(subs)
        for p, (d, _) in enumerate(subs):
            np.testing.assert_array_equal(sd[sp_[p]:sp_[p + 1]], d)
    for l in range(2):
        for a in ("P_col", "PT_col"):
            np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
    bare = [levels[0], levels[1], syn.cube_level(4, 99)]
    with pytest.raises(P.MspError):
        P.Hierarchy(bare, host_only=True, coarse="ras")
    with pytest.raises(P.MspError):
        P.Hierarchy(levels, host_only=True, coarse="ras", nu_pre=0)


@pytest.mark.parametrize("name,ilu", [("cube16_3lvl", (2, 0)), ("cube20_3lvl", (1, 1))])
def test_host_ilu_patterns_match_oracle(P, orc, name, ilu):
    """The ILU(p) level-of-fill pattern of every block (strict lower part; the
    blocks are symmetric) is the oracle's, bit for bit."""
    levels, w = workload(name)
    h = make_hierarchy(levels, w, P, host_only=True, ilu=ilu)
    o = make_oracle(levels, w, orc, ilu=ilu)
    o.assemble(syn.mu_draw(0))
    o.factor()
    for l in range(len(levels) - 1):
        ptr, col, sptr = h.array(l, "ilu_ptr"), h.array(l, "ilu_col"), h.array(l, "sub_ptr")
        for p in range(o.get("n_subs", l)):
            fp, fc = o.get("sub_ilu_ptr", l, p), o.get("sub_ilu_col", l, p)
            for i in range(fp.size - 1):
                oc = fc[fp[i]:fp[i + 1]]
                R = sptr[p] + i
                np.testing.assert_array_equal(col[ptr[R]:ptr[R + 1]], oc[oc < i])


def test_host_elasticity_structures_match_oracle(P, orc):
    """Three displacement fields per vertex: the DoF-level CSR pattern, the
    subdomain DoF lists and the field-split transfers P (x) I_3 are the
    oracle's bit for bit (values to rounding)."""
    levels, w = workload("elast12_3lvl")
    h = make_hierarchy(levels, w, P, host_only=True)
    o = make_oracle(levels, w, orc)
    L = len(levels)
    for l in range(L):
        assert h.info(l)["n_dofs"] == 3 * levels[l].n_nodes == o.n[l]
        assert h.info(l)["n_nodes"] == levels[l].n_nodes
        np.testing.assert_array_equal(h.array(l, "rowptr"), o.get("rowptr", l))
        np.testing.assert_array_equal(h.array(l, "col"), o.get("col", l))
    for l in range(L - 1):
        subs = o.subdomains(l)
        sp_, sd, so = h.array(l, "sub_ptr"), h.array(l, "sub_dofs"), h.array(l, "sub_own")
        assert sp_.size - 1 == len(subs)
        for p, (d, ow) in enumerate(subs):
            np.testing.assert_array_equal(sd[sp_[p]:sp_[p + 1]], d)
            np.testing.assert_array_equal(so[sp_[p]:sp_[p + 1]], ow)
        for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
            np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
        np.testing.assert_allclose(h.array(l, "P_val"), o.get("P_val", l), atol=1e-13)
        np.testing.assert_allclose(h.array(l, "PT_val"), o.get("PT_val", l), atol=1e-13)
    sd = h.array(L - 1, "sub_dofs")
    np.testing.assert_array_equal(sd, np.where(np.repeat(levels[-1].dirichlet, 3) == 0)[0])
    # the elasticity path takes the field-split barycentric transfers only
    with pytest.raises(P.MspError):
        make_hierarchy(levels, w, P, host_only=True, transfer="mls")
    with pytest.raises(P.MspError):
        make_hierarchy(levels, w, P, host_only=True, poisson=0.5)


def test_odd_partition_and_empty_boxes(P, orc):
    """Partition ids that skip values and boxes with only Dirichlet nodes."""
    fine = syn.cube_level(9, 3, parts=(5, 3, 2))
    fine.owner = (fine.owner * 7 + 3).astype(np.int32)  # sparse, non-contiguous ids
    coarse = syn.cube_level(4, 4)
    w = dict(delta=1, nu=1, coef="const", scale=1.0, load="one", restart=10)
    h = make_hierarchy([fine, coarse], w, P, host_only=True)
    o = make_oracle([fine, coarse], w, orc)
    subs = o.subdomains(0)
    sp, sd = h.array(0, "sub_ptr"), h.array(0, "sub_dofs")
    assert sp.size - 1 == len(subs)
    for p, (d, _) in enumerate(subs):
        np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)


def test_invalid_inputs_are_rejected(P):
    lv = syn.cube_level(3, 1, parts=(1, 1, 1))
    co = syn.cube_level(2, 2)
    bad = syn.cube_level(3, 1, parts=(1, 1, 1))
    bad.tets = bad.tets.copy()
    bad.tets[5, 3] = bad.tets[5, 2]  # degenerate tet
    with pytest.raises(P.MspError) as e:
        P.Hierarchy([bad, co], host_only=True)
    assert e.value.code == P.msp.MSP_ERR_INVALID
    bad2 = syn.cube_level(3, 1, parts=(1, 1, 1))
    bad2.tets = bad2.tets.copy()
    bad2.tets[0, 0] = 10 ** 6  # out of range
    with pytest.raises(P.MspError):
        P.Hierarchy([bad2, co], host_only=True)
    nown = syn.cube_level(3, 1)  # no owner on a smoothed level
    with pytest.raises(P.MspError):
        P.Hierarchy([nown, co], host_only=True)
    with pytest.raises(P.MspError):
        P.Hierarchy([lv, co], restart=0, host_only=True)
    with pytest.raises(P.MspError):
        P.Hierarchy([lv, co], delta=-1, host_only=True)
    h = P.Hierarchy([lv, co], host_only=True)
    with pytest.raises(P.MspError):  # no device state on a host-only handle
        h.assemble(np.zeros(8), stream=0)
    # unknown transfer kind, straight through the C ABI
    import ctypes as C
    arr = (P.msp.msp_level_desc * 2)()
    keep = []
    for i, m in enumerate((lv, co)):
        xyz = np.ascontiguousarray(m.xyz)
        tets = np.ascontiguousarray(m.tets, np.int32)
        dr = np.ascontiguousarray(m.dirichlet, np.uint8)
        ow = None if m.owner is None else np.ascontiguousarray(m.owner, np.int32)
        keep += [xyz, tets, dr, ow]
        arr[i] = P.msp.msp_level_desc(xyz.shape[0], xyz.ctypes.data, tets.shape[0], tets.ctypes.data,
                                      dr.ctypes.data, None if ow is None else ow.ctypes.data)
    o = P.msp.default_options(host_only=1, transfer=7)
    out = C.c_void_p()
    assert P.load().msp_load_hierarchy(arr, 2, C.byref(o), C.byref(out)) == P.msp.MSP_ERR_INVALID


@pytest.mark.parametrize("name", ["cube16_3lvl", "cube20_3lvl"])
def test_tile_envelope_holds_the_full_dense_lu(P, orc, name):
    """The library stores only the tile envelope of each block.  The oracle's
    full dense LU (no skipping) must be exactly zero outside it, in L and U."""
    levels, w = workload(name)
    h = make_hierarchy(levels, w, P, host_only=True)
    o = make_oracle(levels, w, orc)
    o.assemble(syn.mu_draw(0))
    o.factor()
    T = P.msp.MSP_TILE
    for l in range(len(levels)):
        coarse = l == len(levels) - 1
        ns = 1 if coarse else o.get("n_subs", l)
        for p in range(ns):
            sub = -1 if coarse else p
            first = P.msp.tile_first_of(h, l, sub)
            n = o.get("sub_dofs", l, sub).size
            LU = o.get("sub_lu", l, sub).reshape(n, n)
            assert np.all(np.diff(first) >= 0) and np.all(first <= np.arange(first.size))
            for I in range(first.size):
                c0 = int(first[I]) * T
                rows = slice(I * T, min(n, (I + 1) * T))
                assert not LU[rows, :c0].any()   # L outside the envelope
                assert not LU[:c0, rows].any()   # U = D L^T, mirrored
    # the envelope is much smaller than the full lower triangle of tiles
    info = h.info(0)
    nt = h.array(0, "sub_nt").astype(np.int64)
    assert info["factor_elems"] < 0.8 * np.sum(nt * (nt + 1) // 2) * T * T


def test_noalloc_binding_checks_its_tensors(P):
    """The binding of msp_multidot_noalloc refuses tensors whose extents the
    C side could not check (it sees raw pointers) before any device call."""
    torch = pytest.importorskip("torch")
    m = P.msp
    cpu = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        m.multidot_noalloc(cpu, cpu, cpu)


def test_random_small_setups_match_oracle(P, orc):
    """Seeded random small set-ups: P1 (2-3 levels of 4^3..12^3 cells, every
    box split of 1-3 a side, overlap 1-3, jitter 0-0.2, barycentric or MLS
    transfers), then P2, P2-P1 and three fields per vertex.  The library's
    host structures equal the oracle's: pattern, subdomains, owners and
    transfer structure bit for bit, transfer weights to rounding.  Partitions
    here include boxes that hold few or no vertices."""
    import random
    rng = random.Random(20261204)
    for _ in range(12):
        nl = rng.choice([2, 3])
        ns = [rng.choice([4, 5, 6, 7, 8, 9, 10, 11, 12])]
        for _ in range(nl - 1):
            ns.append(max(2, ns[-1] // 2 + rng.choice([-1, 0, 0, 1])))
        parts = tuple(tuple(rng.choice([1, 2, 3]) for _ in range(3)) for _ in range(nl - 1))
        transfer = rng.choice(["bary", "bary", "mls"])
        levels = syn.hierarchy(tuple(ns), parts, hierarchy_id=rng.randrange(5), jitter=rng.choice([0.0, 0.1, 0.2]))
        w = dict(delta=rng.choice([1, 2, 3]), nu=2, restart=30, coef="cosexp", scale=1.0, load="one")
        kw = {} if transfer == "bary" else dict(transfer="mls")
        h = make_hierarchy(levels, w, P, host_only=True, **kw)
        o = make_oracle(levels, w, orc, **kw)
        L = len(levels)
        for l in range(L):
            np.testing.assert_array_equal(h.array(l, "rowptr"), o.get("rowptr", l))
            np.testing.assert_array_equal(h.array(l, "col"), o.get("col", l))
        for l in range(L - 1):
            subs = o.subdomains(l)
            sp, sd, so = h.array(l, "sub_ptr"), h.array(l, "sub_dofs"), h.array(l, "sub_own")
            assert sp.size - 1 == len(subs)
            for p, (d, ow) in enumerate(subs):
                np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)
                np.testing.assert_array_equal(so[sp[p]:sp[p + 1]], ow)
            for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
                np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
            for a in ("P_val", "PT_val"):
                ref = o.get(a, l)
                np.testing.assert_allclose(h.array(l, a), ref, rtol=1e-12, atol=1e-13 * max(1.0, abs(ref).max()))
        np.testing.assert_array_equal(h.array(L - 1, "sub_dofs"), np.where(levels[-1].dirichlet == 0)[0])
        h.close()
    # and the other DoF distributions: P2, P2-P1, three fields per vertex
    for _ in range(9):
        nl = rng.choice([2, 3])
        ns = [rng.choice([4, 5, 6, 7, 8])]
        for _ in range(nl - 1):
            ns.append(max(2, ns[-1] // 2 + rng.choice([0, 0, 1])))
        parts = tuple(tuple(rng.choice([1, 2]) for _ in range(3)) for _ in range(nl - 1))
        pde = rng.choice(["poisson_p2", "p2p1", "elasticity"])
        levels = syn.hierarchy(tuple(ns), parts, hierarchy_id=rng.randrange(5), jitter=rng.choice([0.0, 0.1, 0.2]))
        w = dict(delta=rng.choice([1, 2]), nu=2, restart=30, coef="cosexp", scale=1.0, load="one", pde=pde,
                 poisson=0.3, coupling=1.0)
        h = make_hierarchy(levels, w, P, host_only=True)
        o = make_oracle(levels, w, orc)
        L = len(levels)
        for l in range(L):
            assert h.n_dofs(l) == o.n[l]
            np.testing.assert_array_equal(h.array(l, "rowptr"), o.get("rowptr", l))
            np.testing.assert_array_equal(h.array(l, "col"), o.get("col", l))
        for l in range(L - 1):
            subs = o.subdomains(l)
            sp, sd, so = h.array(l, "sub_ptr"), h.array(l, "sub_dofs"), h.array(l, "sub_own")
            assert sp.size - 1 == len(subs)
            for p, (d, ow) in enumerate(subs):
                np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)
                np.testing.assert_array_equal(so[sp[p]:sp[p + 1]], ow)
            for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
                np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
            np.testing.assert_allclose(h.array(l, "P_val"), o.get("P_val", l), atol=1e-13)
            np.testing.assert_allclose(h.array(l, "PT_val"), o.get("PT_val", l), atol=1e-13)
        h.close()


def test_binding_checks_vector_arguments(P):
    """Vectors handed to apply, apply_op, solve, solve_host, poll and a batch's
    solve reach the C side as raw pointers, so the binding checks them first:
    float64, contiguous, long enough for the level, and in the memory the call
    reads (device or host)."""
    m = P.msp
    m._vec(None, 10, "x", "cuda")  # NULL: the C side decides
    m._vec(np.zeros(10), 10, "x", "host")
    m._vec(np.zeros(12), 10, "x", "host")
    with pytest.raises(ValueError, match="entries"):
        m._vec(np.zeros(9), 10, "x", "host")
    with pytest.raises(ValueError, match="float64"):
        m._vec(np.zeros(10, np.float32), 10, "x", "host")
    with pytest.raises(ValueError, match="contiguous"):
        m._vec(np.zeros(20)[::2], 10, "x", "host")
    with pytest.raises(ValueError, match="CUDA"):
        m._vec(np.zeros(10), 10, "x", "cuda")
    with pytest.raises(ValueError, match="numpy"):
        m._vec([0.0] * 10, 10, "x", "host")
    ro = np.zeros(10)
    ro.flags.writeable = False
    m._vec(ro, 10, "b_host", "host")  # read only: fine for an input
    with pytest.raises(ValueError, match="writable"):
        m._vec(ro, 10, "x_host", "host", out=True)
    torch = pytest.importorskip("torch")
    t = torch.zeros(10, dtype=torch.float64)
    m._vec(t, 10, "x", "host")
    with pytest.raises(ValueError, match="CUDA"):
        m._vec(t, 10, "x", "cuda")
    with pytest.raises(ValueError, match="float64"):
        m._vec(t.float(), 10, "x", "host")
    with pytest.raises(ValueError, match="contiguous"):
        m._vec(torch.zeros(20, dtype=torch.float64)[::2], 10, "x", "host")
    with pytest.raises(ValueError, match="entries"):
        m._vec(torch.zeros(9, dtype=torch.float64), 10, "x", "host")


@pytest.mark.parametrize("name", ["p2cube6_3lvl", "p2cube12_3lvl", "p2p1cube6_3lvl", "p2p1cube12_3lvl"])
def test_host_p2_structures_match_oracle(P, orc, name):
    """Quadratic elements (DoFs on vertices and edges): the DoF-level pattern,
    subdomains and the P2 transfers of the library's host set-up against the
    oracle's, bit for bit (values of P to 1e-13)."""
    levels, w = workload(name)
    h = make_hierarchy(levels, w, P, host_only=True)
    o = make_oracle(levels, w, orc)
    L = len(levels)
    for l in range(L):
        assert h.n_dofs(l) == o.n[l]
        np.testing.assert_array_equal(h.array(l, "rowptr"), o.get("rowptr", l))
        np.testing.assert_array_equal(h.array(l, "col"), o.get("col", l))
    for l in range(L - 1):
        subs = o.subdomains(l)
        sp, sd, so = h.array(l, "sub_ptr"), h.array(l, "sub_dofs"), h.array(l, "sub_own")
        assert sp.size - 1 == len(subs)
        for p, (d, ow) in enumerate(subs):
            np.testing.assert_array_equal(sd[sp[p]:sp[p + 1]], d)
            np.testing.assert_array_equal(so[sp[p]:sp[p + 1]], ow)
        for a in ("P_rowptr", "P_col", "PT_rowptr", "PT_col"):
            np.testing.assert_array_equal(h.array(l, a), o.get(a, l))
        np.testing.assert_allclose(h.array(l, "P_val"), o.get("P_val", l), atol=1e-13)
        np.testing.assert_allclose(h.array(l, "PT_val"), o.get("PT_val", l), atol=1e-13)
    dirc = o.get("dofdir", L - 1)
    np.testing.assert_array_equal(h.array(L - 1, "sub_dofs"), np.where(dirc == 0)[0])


def test_binding_frees_dependents_before_their_hierarchy(P, monkeypatch):
    """The binding frees an instance before its hierarchy (and a batch before
    its instances) in either finalisation order of a reference cycle, and an
    explicit close() of a hierarchy closes its live instances first.  The
    library calls are replaced by a log: only the order is checked."""
    msp = P.msp
    log = []

    class Lib:
        def msp_free_hierarchy(self, h):
            log.append(("hierarchy", h))

        def msp_free_instance(self, i):
            log.append(("instance", i))

        def msp_batch_free(self, b):
            log.append(("batch", b))
    monkeypatch.setattr(msp, "load", lambda: Lib())

    def make():
        h = object.__new__(msp.Hierarchy)
        h._init_shared()
        h.h = "H"
        insts = []
        for k in range(2):
            i = object.__new__(msp.Instance)
            i.hier = h
            i._init_shared()
            i.inst = f"I{k}"
            h._acquire(i)
            insts.append(i)
        b = object.__new__(msp.Batch)
        b._insts = list(insts)
        b.b = "B"
        for i in insts:
            i._acquire(b)
        return h, insts, b

    def check(order):
        pos = {name: k for k, (_, name) in enumerate(log)}
        assert sorted(pos) == ["B", "H", "I0", "I1"]
        assert pos["B"] < pos["I0"] and pos["B"] < pos["I1"]
        assert pos["I0"] < pos["H"] and pos["I1"] < pos["H"], order

    # garbage-collector orders: finalisers in any order, no weak references left
    import itertools
    for perm in itertools.permutations(range(4)):
        log.clear()
        h, insts, b = make()
        objs = [h, insts[0], insts[1], b]
        for o in objs[:3]:
            o._deps.clear()
        for k in perm:
            objs[k].__del__()
        check(perm)
    # explicit close of the hierarchy with everything alive
    log.clear()
    h, insts, b = make()
    h.close()
    check("explicit")
    assert h.h is None and all(i.inst is None for i in insts) and b.b is None
