"""CPU oracle for the H-IDBF-LU hot path.

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()`
and by the `cpu_baseline` / `--impl reference` legs of `bench.py`, never by the
product package.  It shares no code with the CUDA path; the only common
module is `workloads` (seeded input definitions, no method arithmetic).

Contents (fp64 numpy, plain and slow):
  hankel    - own H0^(2) (series, Miller + Neumann, Hankel asymptotics)
  geometry  - equal-arc-length chord discretisation of open curves
  efie      - dense impedance matrix, rescaling, plane-wave RHS, exact rows
  dense     - LU with partial pivoting, triangular solves, L~ / U~
  idbf      - naive IDBF (full-block IDs), H-IDBF (Alg. 1), apply (Alg. 2),
              sweeps (Algs. 3-4) and their adjoints
  krylov    - GMRES(restart) on the split-preconditioned system
  farfield  - bistatic / monostatic far field
"""
from . import dense, efie, farfield, geometry, hankel, idbf, krylov  # noqa: F401
