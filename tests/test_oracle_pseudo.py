"""Pins of the oracle's non-local Kleinman-Bylander matrix V^NL (Eqs. 2.3,
2.4, Supp. A.2.2) and of the PW92 LDA correlation (Section 4), against the
paper's two-stage grid algorithm, closed-form Gaussian overlaps, invariants
of the separable operator and the exact limits the PW92 form was built on."""
import math

import numpy as np
import pytest

import workloads as w
from oracle import basis, poisson, pseudo


def two_atoms(h):
    xyz = np.array([[0.0, 0.0, 0.0], [2.1, -1.3, 0.9]])
    return w.make_system(xyz, h=h, pad=6.0)


def test_two_stage_grid_algorithm_equals_projection_form():
    """Supp. A.2.2 as written (psi_Cb = v_nl^C phi_b h^3 on W^C, then
    V^C_ab = phi_a . psi_Cb h^3, summed over atoms) equals B^T diag(e) B for
    the separable KB operator, on a grid coarse enough for the dense
    v_nl^C(r_g, r_g') of each atom; a transposed projection, a missing h^3
    or a wrong energy per channel breaks it."""
    s = two_atoms(0.55)
    kb = pseudo.KB(zeta=1.3, e_s=1.7, e_p=-0.6)
    V1 = pseudo.vnl(s, kb)
    V2 = pseudo.vnl_two_stage(s, kb)
    assert np.max(np.abs(V1 - V2)) < 1e-12 * np.max(np.abs(V1))
    assert np.max(np.abs(V1)) > 1e-3


def test_projections_converge_to_closed_form_overlaps():
    """As h -> 0 the grid projections B_pb = h^3 sum chi_p phi_b tend to the
    continuum overlaps <chi_p | phi_b> of the Cartesian Gaussians (closed
    form, Obara-Saika); the trapezoid sums of Gaussians converge faster than
    any power of h, so the error falls by orders between h = 0.3 and 0.15."""
    kb = pseudo.KB()
    ref = None
    errs = []
    for h in (0.3, 0.15):
        s = two_atoms(h)
        if ref is None:
            ref = pseudo.projections_closed_form(s, kb)
        B, _ = pseudo.projections(s, kb, windowed=False)
        errs.append(np.max(np.abs(B - ref)) / np.max(np.abs(ref)))
    assert errs[1] < 1e-8 and errs[1] < 1e-2 * errs[0], errs


def test_windowed_projections_within_the_window_bound():
    """Windows (Eq. A.4, eta) drop only the tails: the windowed projections
    differ from the unwindowed ones by far less than the charge fraction
    outside (sqrt(eta) for the product of two functions)."""
    s = two_atoms(0.4)
    kb = pseudo.KB()
    Bw, _ = pseudo.projections(s, kb, eta=1e-10)
    Bf, _ = pseudo.projections(s, kb, windowed=False)
    assert np.max(np.abs(Bw - Bf)) < 1e-5 * np.max(np.abs(Bf))


def test_vnl_symmetric_semidefinite_low_rank():
    """V^NL = sum_C sum_p e_p |B_p><B_p| is symmetric, positive
    semidefinite for positive energies (negative semidefinite for negative
    ones), and its rank is at most the number of projectors."""
    s = w.config_system("tiny5")
    for kb, sign in ((pseudo.KB(e_s=1.5, e_p=0.5), 1.0), (pseudo.KB(e_s=-0.8, e_p=-0.3), -1.0)):
        V = pseudo.vnl(s, kb)
        assert np.max(np.abs(V - V.T)) <= 1e-14 * np.max(np.abs(V))
        ev = np.linalg.eigvalsh(V) * sign
        assert ev.min() > -1e-12 * ev.max()
        nproj = 4 * s.n_atoms
        assert np.sum(ev > 1e-10 * ev.max()) <= nproj
    # s projectors only: rank at most one per atom
    V = pseudo.vnl(s, pseudo.KB(with_p=False))
    ev = np.linalg.eigvalsh(V)
    assert np.sum(ev > 1e-10 * ev.max()) <= s.n_atoms


def test_vnl_translation_by_a_grid_vector():
    """Moving the atoms and the grid origin by a grid vector leaves V^NL
    unchanged (the grid sums see the same points relative to every centre)."""
    s = w.config_system("tiny5")
    V = pseudo.vnl(s, pseudo.KB())
    shift = s.grid_h * np.array([3, -2, 5])
    s2 = w.make_system(s.xyz + shift, h=s.grid_h, grid_n=s.grid_n, grid_origin=s.grid_origin + shift)
    V2 = pseudo.vnl(s2, pseudo.KB())
    assert np.max(np.abs(V - V2)) < 1e-13 * np.max(np.abs(V))


def test_projector_normalisation():
    """Each projector has unit continuum norm: <chi_p|chi_p> = 1 (closed
    form), like the basis functions."""
    s = two_atoms(0.4)
    pj = pseudo.projectors(s, pseudo.KB(zeta=0.7))
    S, _ = basis.overlap_kinetic(pj)
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-13


def test_pw92_high_density_limit_and_construction():
    """PW92's A is the exact high-density coefficient of ln r_s,
    (1 - ln 2) / pi^2 (Gell-Mann and Brueckner); b1 and b2 are fixed by the
    next term of that expansion, b1 = exp(-c1 / 2A) / 2A with c1 = 0.046644
    and b2 = 2 A b1^2.  A mistyped constant breaks one of these."""
    A = poisson.PW92_A
    b1, b2, _, _ = poisson.PW92_B
    assert abs(A - (1.0 - math.log(2.0)) / math.pi ** 2) < 2e-5 * A
    assert abs(b1 - math.exp(-0.046644 / (2 * A)) / (2 * A)) < 5e-5 * b1
    assert abs(b2 - 2 * A * b1 * b1) < 5e-5 * b2
    # the form itself: eps_c - A ln r_s tends to a constant as r_s -> 0
    rs = np.array([1e-6, 1e-7])
    n = 3.0 / (4.0 * math.pi * rs ** 3)
    _, e = poisson.pw92_correlation(n)
    d = e - A * np.log(rs)
    assert abs(d[0] - d[1]) < 1e-3 * abs(d[1])


def test_pw92_potential_is_the_derivative():
    """v_c = d(n eps_c)/dn (central differences), negative and monotone in
    n; zero below the density floor."""
    n = np.geomspace(1e-6, 10.0, 40)
    v, e = poisson.pw92_correlation(n)
    dn = 1e-5 * n
    _, ep = poisson.pw92_correlation(n + dn)
    _, em = poisson.pw92_correlation(n - dn)
    fd = ((n + dn) * ep - (n - dn) * em) / (2 * dn)
    assert np.max(np.abs(fd - v) / np.abs(v)) < 1e-8
    assert np.all(e < 0) and np.all(np.diff(e) < 0)
    v0, e0 = poisson.pw92_correlation(np.array([0.0, 1e-31]))
    assert np.all(v0 == 0) and np.all(e0 == 0)
