"""Jittered Kuhn-split tetrahedral meshes of the unit cube and the L-shape.

Recipe (every choice here is an input convention, not part of the method):

* Lattice: an n^3 hex grid of the unit cube, nodes (i, j, k), 0 <= i,j,k <= n,
  numbered x-fastest: id = i + (n+1) * (j + (n+1) * k).  For the L-shape
  (cube minus the open octant (0.5,1]^3) the hexes whose centre lies in the
  removed octant are dropped and the surviving nodes are renumbered in the
  same lattice order.
* Each hex (cells numbered x-fastest) is cut into the 6 Kuhn tetrahedra that
  share the hex diagonal (0,0,0)-(1,1,1): for every permutation (p0,p1,p2) of
  the axes, in lexicographic order, the tet is
  c, c+e_p0, c+e_p0+e_p1, c+(1,1,1).
* Dirichlet nodes are the nodes on the domain boundary (cube faces; for the
  L-shape also the three re-entrant faces).  They are never jittered.
* Every other node is moved by an independent U[-0.2h, 0.2h] draw per
  coordinate from numpy's default_rng(seed).
* Box partition of the vertices by lattice index on an N = n+1 point lattice:
  box (floor(i*px/N), floor(j*py/N), floor(k*pz/N)), box id
  bx + px*(by + py*bz).

Seeds: mesh level l of hierarchy h uses 1000 + 17*l + 1009*h; the wave
vectors use 7; request r draws mu from 2024 + r.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_PERMS = list(itertools.permutations((0, 1, 2)))


@dataclass
class Level:
    """One mesh level: coordinates, tets, Dirichlet flags, vertex owners."""
    n: int                      # hex cells per axis of the generating lattice
    xyz: np.ndarray             # float64 [N, 3]
    tets: np.ndarray            # int32   [m, 4]
    dirichlet: np.ndarray       # uint8   [N]
    owner: Optional[np.ndarray] = None   # int32 [N] box id, or None (coarsest)
    lattice: Optional[np.ndarray] = None  # int32 [N, 3]
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _lattice_nodes(n: int, lshape: bool):
    ii, jj, kk = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1),
                             indexing="ij")
    # x-fastest order: flatten with k slowest
    lat = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                    kk.transpose(2, 1, 0).ravel()], axis=1).astype(np.int64)
    return lat


def cube_level(n: int, seed: int, jitter: float = 0.2, lshape: bool = False,
               parts: Optional[Sequence[int]] = None) -> Level:
    """Jittered Kuhn mesh on an n^3 lattice (see the module docstring)."""
    if lshape and n % 2:
        raise ValueError("the L-shape needs an even n")
    N = n + 1
    lat = _lattice_nodes(n, lshape)
    full_id = lambda i, j, k: i + N * (j + N * k)  # noqa: E731

    # hex cells, x-fastest
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(),
                      ck.transpose(2, 1, 0).ravel()], axis=1).astype(np.int64)
    if lshape:
        h2 = n // 2
        keep = ~((cells[:, 0] >= h2) & (cells[:, 1] >= h2) & (cells[:, 2] >= h2))
        cells = cells[keep]
    tets = []
    for cell in (cells,):
        c = cell
        for p in _PERMS:
            e0 = np.zeros(3, np.int64); e0[p[0]] = 1
            e1 = e0.copy(); e1[p[1]] = 1
            v = [c, c + e0, c + e1, c + 1]
            tets.append(np.stack([full_id(x[:, 0], x[:, 1], x[:, 2]) for x in v], axis=1))
    # interleave: tet index = 6*cell + perm
    tets = np.stack(tets, axis=1).reshape(-1, 4)

    used = np.zeros(N ** 3, bool)
    used[tets.ravel()] = True
    renum = -np.ones(N ** 3, np.int64)
    renum[used] = np.arange(int(used.sum()))
    tets = renum[tets].astype(np.int32)
    lat = lat[used]

    on_face = np.any((lat == 0) | (lat == n), axis=1)
    if lshape:
        h2 = n // 2
        in_oct = np.all(lat >= h2, axis=1)   # closed removed octant: re-entrant faces
        on_face |= in_oct
    dirichlet = on_face.astype(np.uint8)

    h = 1.0 / n
    xyz = lat.astype(np.float64) * h
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    interior = dirichlet == 0
    xyz[interior] += jit[interior]

    owner = None
    if parts is not None:
        px, py, pz = (int(v) for v in parts)
        bx = (lat[:, 0] * px) // N
        by = (lat[:, 1] * py) // N
        bz = (lat[:, 2] * pz) // N
        owner = (bx + px * (by + py * bz)).astype(np.int32)
    return Level(n=n, xyz=np.ascontiguousarray(xyz), tets=np.ascontiguousarray(tets),
                 dirichlet=dirichlet, owner=owner, lattice=lat.astype(np.int32),
                 meta=dict(seed=seed, jitter=jitter, lshape=lshape, parts=parts))


def level_seed(level: int, hierarchy_id: int = 0) -> int:
    return 1000 + 17 * level + 1009 * hierarchy_id


def hierarchy(ns: Sequence[int], parts: Sequence[Optional[Sequence[int]]],
              hierarchy_id: int = 0, lshape: bool = False, jitter: float = 0.2):
    """Independently jittered, non-nested levels, finest first."""
    return [cube_level(n, level_seed(l, hierarchy_id), jitter=jitter, lshape=lshape,
                       parts=parts[l] if l < len(parts) else None)
            for l, n in enumerate(ns)]


def wave_vectors(seed: int = 7) -> np.ndarray:
    """Integer wave vectors a_j in {1,2,3}^3, j = 1..8 (int32 [8, 3])."""
    return np.random.default_rng(seed).integers(1, 4, size=(8, 3)).astype(np.int32)


def mu_draw(request: int) -> np.ndarray:
    """mu ~ U[-1, 1]^8 for request number `request`."""
    return np.random.default_rng(2024 + request).uniform(-1.0, 1.0, size=8)


# Workloads: name -> hierarchy recipe and solver options.
#   coef: "const" (k = 1) or "cosexp" (k = exp(s * sum_j mu_j 0.5 cos(pi a_j.x)))
#   load: "sines" (f = 3 pi^2 sin sin sin) or "one" (f = 1; elasticity: f = (0, 0, -1))
#   pde: "poisson" (default), "elasticity" (with its Poisson ratio "poisson"),
#        "poisson_p2" (quadratic elements: DoFs on the vertices and the edges) or
#        "p2p1" (a quadratic field u and a linear field p coupled with the
#        coefficient "coupling")
WORKLOADS = {
    # two-level plain FP64, 8^3 -> 4^3, 2x2x2 boxes, overlap 1
    "cube8_2lvl": dict(ns=(8, 4), parts=((2, 2, 2),), delta=1, nu=2, coef="const",
                       scale=1.0, load="sines", rtol=1e-8, restart=30),
    # small multi-tile parity case
    "cube16_3lvl": dict(ns=(16, 8, 4), parts=((4, 4, 4), (2, 2, 2)), delta=2, nu=2,
                        coef="cosexp", scale=1.0, load="one", rtol=1e-10, restart=30),
    "cube24_3lvl": dict(ns=(24, 12, 6), parts=((3, 3, 3), (2, 2, 2)), delta=2, nu=2,
                        coef="cosexp", scale=1.0, load="one", rtol=1e-10, restart=30),
    # profiling case of the same kernels: 64 subdomains of up to ~1700 DoFs
    "cube32_3lvl": dict(ns=(32, 16, 8), parts=((4, 4, 4), (4, 4, 4)), delta=2, nu=2,
                        coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30),
    # mid-size profiling case (persistent factorisation path): 343 blocks of
    # ~1300 DoFs, like the 64^3 case
    "cube48_3lvl": dict(ns=(48, 24, 12), parts=((7, 7, 7), (7, 7, 7)), delta=2, nu=2,
                        coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30),
    # three-level plain FP64, 64^3 -> 32^3 -> 16^3, 512 boxes per RAS level, overlap 2
    "cube64_3lvl": dict(ns=(64, 32, 16), parts=((8, 8, 8), (8, 8, 8)), delta=2, nu=2,
                        coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30),
    # batched uneven solves: the 32^3 hierarchy of the batch, with enough
    # subdomains (5x5x5) for its finest level to take the persistent
    # factorisation (the 48^3 one is cube48_3lvl)
    "cube32b_3lvl": dict(ns=(32, 16, 8), parts=((5, 5, 5), (3, 3, 3)), delta=2, nu=2,
                         coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30),
    # the largest serving hierarchy: 128^3 (2,146,689 nodes, 12.6M tets) with
    # 64^3 / 32^3 / 16^3 coarse levels (four levels: a 32^3 coarsest level would
    # need a 10 GB dense factor), 16^3 boxes of ~500 owned DoFs on the finest
    # level and 8^3 on the coarser smoothed ones
    "cube128_4lvl": dict(ns=(128, 64, 32, 16), parts=((16, 16, 16), (8, 8, 8), (8, 8, 8)), delta=2, nu=2,
                         coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30),
    # precision study: L-shaped domain (unit cube minus [0.5,1]^3), 96^3 with
    # 48^3/24^3/12^3 coarse levels, 2048 subdomains of 294-1320 DoFs on the
    # finest level, k spanning 1e-2 .. 1e2 (s = 1.15: |sum_j 0.5 mu_j cos| <= 4),
    # FGMRES to rtol 1e-10
    "lshape96_4lvl": dict(ns=(96, 48, 24, 12), parts=((16, 16, 9), (8, 8, 8), (4, 4, 4)), lshape=True,
                          delta=2, nu=2, coef="cosexp", scale=1.15, load="one", rtol=1e-10, restart=30),
    # linear elasticity (three displacement fields per vertex, Poisson ratio
    # 0.3, unit body force along -z): parity case with blocks of ~1500 DoFs
    "elast12_3lvl": dict(ns=(12, 6, 3), parts=((2, 2, 2), (2, 2, 2)), delta=1, nu=2,
                         coef="cosexp", scale=1.0, load="one", rtol=1e-10, restart=30,
                         pde="elasticity", poisson=0.3),
    # quadratic (P2) elements: one DoF per vertex and per edge (N = (1,1,0,0));
    # a small pin / parity case and the measured one (32^3: 35,937 vertices,
    # 274,625 DoFs with the edges, 512 + 64 subdomains of ~1,500 / ~1,300 DoFs)
    "p2cube6_3lvl": dict(ns=(6, 3, 2), parts=((2, 2, 2), (1, 1, 1)), delta=1, nu=2,
                         coef="cosexp", scale=1.0, load="one", rtol=1e-10, restart=30, pde="poisson_p2"),
    "p2cube12_3lvl": dict(ns=(12, 6, 3), parts=((3, 3, 3), (2, 2, 2)), delta=1, nu=2,
                          coef="cosexp", scale=1.0, load="one", rtol=1e-10, restart=30, pde="poisson_p2"),
    "p2cube32_3lvl": dict(ns=(32, 16, 8), parts=((8, 8, 8), (4, 4, 4)), delta=1, nu=2,
                          coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30, pde="poisson_p2"),
    # two fields of different element order (u quadratic, p linear) coupled by
    # sigma k (u - p): field-split transfers, P2 interpolation for u, P1 for p
    "p2p1cube6_3lvl": dict(ns=(6, 3, 2), parts=((2, 2, 2), (1, 1, 1)), delta=1, nu=2, coef="cosexp",
                           scale=1.0, load="one", rtol=1e-10, restart=30, pde="p2p1", coupling=1.0),
    "p2p1cube12_3lvl": dict(ns=(12, 6, 3), parts=((3, 3, 3), (2, 2, 2)), delta=1, nu=2, coef="cosexp",
                            scale=1.0, load="one", rtol=1e-10, restart=30, pde="p2p1", coupling=1.0),
    "p2p1cube32_3lvl": dict(ns=(32, 16, 8), parts=((8, 8, 8), (4, 4, 4)), delta=1, nu=2, coef="cosexp",
                            scale=1.0, load="one", rtol=1e-8, restart=30, pde="p2p1", coupling=1.0),
    # and the measured case: 107,811 DoFs on 32^3, 64 + 8 blocks of ~3000 DoFs
    "elast32_3lvl": dict(ns=(32, 16, 8), parts=((4, 4, 4), (2, 2, 2)), delta=1, nu=2,
                         coef="cosexp", scale=1.0, load="one", rtol=1e-8, restart=30,
                         pde="elasticity", poisson=0.3),
}


def workload(name: str, hierarchy_id: int = 0):
    """Return (levels, options dict) for a named workload."""
    w = dict(WORKLOADS[name])
    levels = hierarchy(w["ns"], w["parts"], hierarchy_id=hierarchy_id,
                       lshape=w.get("lshape", False))
    return levels, w
