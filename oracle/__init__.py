"""FP64 CPU oracle for the Chebyshev Gaussian-basis DFT hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, calls or links this package; only the tests, the
smoke check and the benchmark's CPU-baseline leg do.  It shares no code with
the CUDA path: the only common input is the seeded geometry from `workloads`.

Every function cites the passage of arXiv 2108.13478 it follows (section,
equation or algorithm).  Where the paper is silent the reading taken is stated
in the docstring.

Modules
  basis       normalised Cartesian Gaussians, windows (Eq. A.4), separable
              tables (Supp. A.1), closed-form S and T (Obara-Saika)
  grid_ops    quadrature V = h^3 sum phi v phi (Eq. 2.5 / A.6) and
              collocation n = 2 sum P phi phi (Eq. 2.7 / A.5)
  dm          generalised eigensolve, Fermi-Dirac DM (Eq. 2.9), Chebyshev
              expansion and recurrence (Supp. B), mu bisection (Eq. 2.8)
  poisson     free-space Hartree potential by zero-padded FFT, Slater exchange
  pseudo      non-local Kleinman-Bylander V^NL from synthetic projectors
              (Eqs. 2.3-2.4, Supp. A.2.2)
  sparse      density-matrix columns by the sparse-operator route: the
              vector recurrence with S^-1 by PCG (Section 2, Supp. B)
  scf         local pseudopotential, initial density, energy, SCF cycle (A.3)
  warmstart   atom-centred descriptor, MLP, start-potential assembly and
              their gradients (the learned warm start; not in the paper)

Parity status: every function is pinned by the `-m "not gpu"` tests in
tests/test_oracle_*.py against closed forms, brute force or library routines;
none is "parity unpinned".
"""
