"""The Chebyshev order the mixed path runs at, justified with the oracle.

N_C is the smallest order whose coefficient tail sum_{l >= N_C} |a_l| is
below a tolerance (Supp. B's expansion; the paper's own rule is
N_C ~ 2 beta dE).  The FP64 path uses 1e-10 so that P matches to 1e-9; the
mixed path's products already cost ~4e-6 Ha/atom, and at 1e-5 (the bench's
default for the mixed path) or 1e-6 the truncation adds orders of magnitude
less than that while the order drops by half or by 40%.  On
the 64-atom cluster's first Fock matrix: the truncated density matrix of
each tolerance (same padded bounds as the library: 2% of the width + 1e-3
Ha each side) against the exact Fermi-Dirac one.
"""
import numpy as np
import pytest

import workloads as w
from oracle import dm, scf


@pytest.fixture(scope="module")
def cluster():
    s = w.config_system("cluster64")
    st = scf.setup(s, scf.Model(neutral=True))
    v, _, _ = scf.potential(st, scf.ion_density(s))
    F = scf.fock(st, v)
    beta = 1.0 / s.kT
    eps, C = dm.geneig(F, st.S)
    width = eps[-1] - eps[0]
    lo, hi = eps[0] - 0.02 * width - 1e-3, eps[-1] + 0.02 * width + 1e-3
    ex = dm.dm_exact(F, st.S, s.n_electrons, beta)
    return s, st, F, beta, eps, C, lo, hi, ex


_CACHE = {}


def _truncated(cluster, tol):
    if tol in _CACHE:
        return _CACHE[tol]
    s, st, F, beta, eps, C, lo, hi, ex = cluster
    eb, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    n_c = dm.cheb_order(eb, beta, lo, hi, tol)
    x = (eps - eb) / de
    mom = dm.moments_from_eigs(x, n_c)
    mu = dm.bisect(lambda m: dm.electron_count(m, beta, lo, hi, mom), s.n_electrons, lo - 40 / beta, hi + 40 / beta)
    p = dm.cheb_eval(x, dm.cheb_coeffs(mu, beta, lo, hi, n_c))
    dP = (C * p) @ C.T - ex["P"]
    e_kin = abs(2 * np.sum(dP * st.T)) / s.n_atoms
    e_band = abs(2 * np.sum(dP * F)) / s.n_atoms
    _CACHE[tol] = (n_c, e_kin, e_band)
    return _CACHE[tol]


def test_mixed_path_order_costs_far_less_than_its_arithmetic(cluster):
    s, st, F, beta, eps, C, lo, hi, ex = cluster
    n10 = dm.cheb_order(0.5 * (hi + lo), beta, lo, hi, 1e-10)     # the FP64 path's order
    n6, k6, b6 = _truncated(cluster, 1e-6)
    assert n6 < 0.65 * n10                       # ~40% fewer recurrence steps
    assert k6 < 1e-8 and b6 < 1e-8               # vs ~4e-6 Ha/atom from the split-FP16 products


def test_truncation_error_falls_with_the_tolerance(cluster):
    e5 = max(_truncated(cluster, 1e-5)[1:])
    e6 = max(_truncated(cluster, 1e-6)[1:])
    assert e5 > e6 and e5 < 1e-6


def test_bench_default_tolerance_stays_two_orders_below_the_arithmetic(cluster):
    # 1e-5: 17% fewer steps than 1e-6, truncation ~1e-8 Ha/atom
    n6 = _truncated(cluster, 1e-6)[0]
    n5, k5, b5 = _truncated(cluster, 1e-5)
    assert n5 < 0.85 * n6
    assert k5 < 5e-8 and b5 < 5e-8
