"""FP64 CPU oracle for the multi-rhs / multi-shift twisted-mass multigrid solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or
runs this package: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` do. It shares no code with the CUDA path; the two
meet only in the seeded input generators of ``synth``.

Everything is plain numpy in complex128, written from the paper's description
of the method (arXiv:2201.03872, Sec. 2 "DDalphaAMG", Sec. 3 "Multiple Right
Hand Sides", Sec. 4 "Block Solvers", Fig. 6 caption for the twisted-mass
operator) and from the standard definitions it relies on. Where the paper is
silent, the module docstrings state the reading taken.

Modules:
  gamma   -- Dirac matrices in the chiral basis, sigma_{mu nu}
  dirac   -- clover term and the operator D(mu) = D_W + c_sw C + i mu gamma5
  krylov  -- (F)GMRES and block GMRES
  sap     -- red-black Schwarz alternating procedure with minimal-residual block solves
  amg     -- aggregation, test vectors, P / R, coarse operator, AMG cycle and solver
"""
