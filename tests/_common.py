"""Shared helpers of the test suite: the same seeded workload is handed to the
oracle and to the library, each through its own entry points."""
import numpy as np

import synthetic as syn

# small parity workloads (oracle finishes in seconds, several tiles + a ragged tail)
PARITY = ["cube8_2lvl", "cube16_3lvl", "cube20_3lvl"]

syn.WORKLOADS.setdefault("cube20_3lvl", dict(ns=(20, 10, 5), parts=((3, 3, 3), (2, 2, 2)),
                                              delta=2, nu=2, coef="cosexp", scale=1.0,
                                              load="one", rtol=1e-10, restart=30))

# the same sizes with one box grid on both RAS levels, so that the MLS transfer
# pairs subdomain q of one level with subdomain q of the other
syn.WORKLOADS.setdefault("cube20m_3lvl", dict(ns=(20, 10, 5), parts=((3, 3, 3), (3, 3, 3)),
                                               delta=2, nu=2, coef="cosexp", scale=1.0,
                                               load="one", rtol=1e-10, restart=30))


def workload(name, hierarchy_id=0):
    return syn.workload(name, hierarchy_id)


def _pde(w):
    if "pde" not in w:
        return {}
    return dict(pde=w["pde"], poisson=w.get("poisson", 0.3), coupling=w.get("coupling", 1.0))


def make_oracle(levels, w, orc, **kw):
    args = dict(delta=w["delta"], nu_pre=w["nu"], nu_post=w["nu"], coef=w["coef"],
                wave=syn.wave_vectors(), scale=w["scale"], load=w["load"], **_pde(w))
    args.update(kw)
    return orc.Oracle(levels, **args)


def make_hierarchy(levels, w, P, **kw):
    args = dict(delta=w["delta"], nu_pre=w["nu"], nu_post=w["nu"], restart=w["restart"],
                coef=w["coef"], wave=syn.wave_vectors(), scale=w["scale"], load=w["load"], **_pde(w))
    args.update(kw)
    return P.Hierarchy(levels, **args)


def n_dofs(levels, w, level=0):
    """Vector length of a level of a workload (P1 DoF distributions only; with
    P2 elements take the oracle's count)."""
    assert w.get("pde") != "poisson_p2"
    return (3 if w.get("pde") == "elasticity" else 1) * levels[level].n_nodes


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def relmax(a, b):
    """Element-wise relative difference: max |a - b| over max |b|."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0)) if a.size else 0.0


def close(a, b, tol):
    """Both the norm-wise and the element-wise relative difference within tol."""
    return rel(a, b) <= tol and relmax(a, b) <= tol
