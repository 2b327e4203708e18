"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only *generates inputs*: jittered structured tetrahedral meshes
(the stand-in for the paper's unstructured meshes, Section 4), their Dirichlet
flags, a box partition of the vertices (the stand-in for the graph partitioner
that distributes the mesh over np processors, Section 2.2), the wave vectors of
the coefficient family and the parameter draws mu.  It holds none of the
method's arithmetic: no stiffness, no interpolation weights, no solver.
"""
from .mesh import (Level, cube_level, hierarchy, wave_vectors, mu_draw,
                   WORKLOADS, workload)

__all__ = ["Level", "cube_level", "hierarchy", "wave_vectors", "mu_draw",
           "WORKLOADS", "workload"]
