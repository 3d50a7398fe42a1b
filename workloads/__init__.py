"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the method: it builds atom coordinates,
the basis specification (exponents and angular momenta per shell), the grid
geometry and the run parameters.  Normalisation constants, windows, integrals
and everything downstream are computed independently by the oracle and by the
CUDA library.
"""
from .si_clusters import (  # noqa: F401
    SI_A0, DIAMOND_BASIS, SHELL_SPEC, System,
    diamond_supercell, diamond_sphere, make_system, config_system, batch_systems, config_batch,
)
