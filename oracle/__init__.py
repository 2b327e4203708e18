"""FP64 CPU oracle for the non-nested multilevel smoothed Schwarz method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`.  It never runs on the library's
product path.  The arithmetic lives in `msp_oracle.cpp` (plain C++17, FP64,
-ffp-contract=off); this module compiles it with g++ and wraps it with ctypes.

Parity status per function (what pins it, tests/test_oracle_pins.py):
  tet stiffness      reference-tet closed form, affine patch test, energy identity
  CSR pattern        independent numpy construction from the tets
  assembly           symmetry, zero row sums, 7-point stencil on an unjittered
                     grid, O(h^2) L2 convergence to a manufactured solution,
                     energy of affine fields vs a Gauss-quadrature integral of k
  load vector        O(h^2) convergence (with the assembly)
  subdomains         partition of unity; overlap = graph distance <= delta (BFS)
  LU / solve         ||LU - A|| / ||A|| and scipy.linalg.solve
  RAS                one subdomain (or full overlap) gives A^{-1} exactly;
                     dense numpy formula sum R0^T (R A R^T)^{-1} R
  interpolation P    affine reproduction, unit row sums, identity on equal meshes
  MLS transfer       every row against a brute-force weighted least-squares fit
                     (numpy BFS neighbourhood, SVD rank, monomial basis, pinv);
                     affine reproduction; Dirichlet handling; nodal-volume
                     scaling (tests/test_oracle_mls_pins.py)
  V-cycle            dense numpy composition of the same operators on tiny meshes,
                     also with the coarsest level RAS-smoothed and for the
                     one-level RAS preconditioner (tests/test_oracle_alg2_pins.py)
  FGMRES             Krylov least-squares optimality (M = I), direct solve
  elasticity         (three displacement fields per vertex) element stiffness
                     against an independent Voigt B^T D B construction, rigid
                     modes, rank and the energy of linear fields; patch test
                     and rigid modes of the assembled operator; Dirichlet rows
                     and body-force load; O(h^2) convergence to a manufactured
                     solution; field-split transfers reproduce affine vector
                     fields; RAS, V-cycle and FGMRES against dense compositions
                     (tests/test_oracle_elasticity_pins.py)
Iteration counts of the preconditioned solver: parity unpinned (the paper
reports counts only for other PDEs and meshes).
"""
from .oracle import (Oracle, build, lib, tet_stiffness, tet_elasticity, tet_p2, tet_p2p1, lame, lu_factor, lu_solve,
                     build_interp, build_mls, mesh_h, ilu_factor)

__all__ = ["Oracle", "build", "lib", "tet_stiffness", "tet_elasticity", "tet_p2", "tet_p2p1", "lame", "lu_factor", "lu_solve",
           "build_interp", "build_mls", "mesh_h", "ilu_factor"]
