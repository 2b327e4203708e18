"""Pins for the oracle's ILU(p) subdomain solver (Section 4.4: ILU(2) on the
finest level, ILU(0) on the coarser ones, in place of the exact subdomain LU).

The level-of-fill pattern is checked against the fill-path characterisation
(entry (i, j) has level = length of the shortest path i -> j in the graph of
A through vertices numbered below min(i, j), minus one), computed here by a
breadth-first search; the numbers against a dense brute-force elimination
restricted to that pattern and against the defining property (L U)_ij = a_ij
on the pattern; special cases against exact LU.  CPU only.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _spd_block(orc, n=5, seed=3):
    lv = syn.cube_level(n, seed)
    o = orc.Oracle([lv], coef="cosexp", wave=syn.wave_vectors())
    o.assemble(syn.mu_draw(1))
    A = o.csr(0)
    inner = np.nonzero(lv.dirichlet == 0)[0]
    return sp.csr_matrix(A[inner][:, inner])


def _fill_path_levels(A, p):
    """lev(i, j) <= p for the pattern of ILU(p), by BFS over vertices < min(i, j)."""
    n = A.shape[0]
    G = sp.csr_matrix(A)
    pattern = set()
    for i in range(n):
        for j in range(n):
            lo = min(i, j)
            # shortest path i -> j whose interior vertices are all < lo
            dist = {i: 0}
            frontier = [i]
            found = i == j or G[i, j] != 0
            d = 0
            while not found and frontier and d < p + 1:
                d += 1
                nxt = []
                for u in frontier:
                    for v in G.indices[G.indptr[u]:G.indptr[u + 1]]:
                        if v == j:
                            found = True
                            break
                        if v < lo and v not in dist:
                            dist[v] = d
                            nxt.append(v)
                    if found:
                        break
                frontier = nxt
            if found:
                pattern.add((i, j))
    return pattern


def _dense_ilu(A, pattern):
    """Brute-force IKJ Gaussian elimination, dropping every entry outside `pattern`."""
    n = A.shape[0]
    W = A.toarray().astype(np.float64)
    mask = np.zeros((n, n), bool)
    for (i, j) in pattern:
        mask[i, j] = True
    for i in range(n):
        for k in range(i):
            if not mask[i, k]:
                continue
            W[i, k] /= W[k, k]
            for j in range(k + 1, n):
                if mask[i, j] and mask[k, j]:
                    W[i, j] -= W[i, k] * W[k, j]
    W[~mask] = 0.0
    return np.tril(W, -1) + np.eye(n), np.triu(W)


def test_no_fill_matrix_gives_exact_lu(orc):
    n = 40
    A = sp.diags([-1.0, 2.3, -1.0], [-1, 0, 1], shape=(n, n)).tocsr()
    L, U = orc.ilu_factor(A, 0)
    np.testing.assert_allclose((L @ U).toarray(), A.toarray(), atol=1e-14)


def test_full_fill_equals_exact_lu(orc):
    A = _spd_block(orc, n=4)
    n = A.shape[0]
    L, U = orc.ilu_factor(A, n)
    np.testing.assert_allclose((L @ U).toarray(), A.toarray(), atol=1e-13 * abs(A).max())
    b = np.random.default_rng(0).normal(size=n)
    x = sp.linalg.spsolve_triangular(U, sp.linalg.spsolve_triangular(L, b, lower=True), lower=False)
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-10)


@pytest.mark.parametrize("p", [0, 1, 2])
def test_pattern_matches_fill_paths_and_numbers_brute_force(orc, p):
    A = _spd_block(orc, n=4, seed=7)
    L, U = orc.ilu_factor(A, p)
    F = (sp.tril(L, -1) + U).tocsr()
    got = set(zip(*F.nonzero())) | {(i, i) for i in range(A.shape[0])}
    # keep explicit zeros of the factor in the comparison: use its structure
    got = set()
    for i in range(F.shape[0]):
        for j in F.indices[F.indptr[i]:F.indptr[i + 1]]:
            got.add((i, int(j)))
    want = _fill_path_levels(A, p)
    assert got == want
    if p == 0:
        assert got == set((i, int(j)) for i in range(A.shape[0])
                          for j in A.indices[A.indptr[i]:A.indptr[i + 1]])
    Ld, Ud = _dense_ilu(A, want)
    np.testing.assert_allclose(L.toarray(), Ld, atol=1e-13)
    np.testing.assert_allclose(U.toarray(), Ud, atol=1e-13 * abs(A).max())
    # the defining property: L U reproduces A on the pattern
    R = (L @ U - A).toarray()
    for (i, j) in want:
        assert abs(R[i, j]) <= 1e-13 * abs(A).max()


def test_more_fill_is_a_better_approximation(orc):
    A = _spd_block(orc, n=5, seed=11)
    Ad = A.toarray()
    errs = []
    for p in (0, 1, 2, 4):
        L, U = orc.ilu_factor(A, p)
        errs.append(np.linalg.norm(Ad - (L @ U).toarray()) / np.linalg.norm(Ad))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[0] < 0.5


def test_ras_with_full_fill_single_subdomain_is_exact(orc):
    lv = syn.cube_level(5, 21, parts=(1, 1, 1))
    co = syn.cube_level(2, 22)
    o = orc.Oracle([lv, co], delta=1, coef="cosexp", wave=syn.wave_vectors(), ilu=(10 ** 6, 0))
    o.assemble(syn.mu_draw(2))
    o.factor()
    A = o.csr(0).toarray()
    r = np.random.default_rng(3).normal(size=lv.n_nodes)
    np.testing.assert_allclose(o.ras_apply(r, 0), np.linalg.solve(A, r), rtol=1e-9, atol=1e-12)


def test_fgmres_with_ilu_smoothers_converges(orc):
    levels, w = syn.workload("cube16_3lvl")
    kw = dict(delta=w["delta"], coef="cosexp", wave=syn.wave_vectors(), load="one")
    its = {}
    for tag, ilu in (("lu", None), ("ilu20", (2, 0))):
        o = orc.Oracle(levels, ilu=ilu, **kw)
        o.assemble(syn.mu_draw(0))
        o.factor()
        x, st = o.fgmres(rtol=1e-10)
        A = o.csr(0)
        b = o.get("b")
        assert st["status"] == 0
        assert np.linalg.norm(A @ x - b) <= 1.01e-10 * np.linalg.norm(b)
        its[tag] = st["iters"]
    assert its["lu"] <= its["ilu20"] < 60
