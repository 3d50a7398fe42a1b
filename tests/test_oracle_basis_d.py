"""Pins of the oracle's contracted spherical Gaussians up to d (Supp. A.1,
Eqs. A.1-A.3, Table A.1): normalisation, the solid harmonics' orthogonality
and rotational invariance, closed-form kinetic values, the closed forms
against fine-grid sums, and the grid transforms of contracted functions
against each other."""
import math

import numpy as np

import workloads as w
from oracle import basis, grid_ops, scf


def one_atom(shells, spherical, h=0.1, pad=7.0):
    return w.make_system(np.zeros((1, 3)), h=h, pad=pad, shells=shells, spherical=spherical)


def test_contracted_functions_are_normalised():
    for name in ("dtiny5", "ctiny5"):
        S, T = basis.overlap_kinetic_system(w.config_system(name))
        assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-13
        assert np.max(np.abs(S - S.T)) < 1e-14 and np.max(np.abs(T - T.T)) < 1e-13
        assert np.linalg.eigvalsh(S).min() > 0 and np.linalg.eigvalsh(T).min() > 0


def test_spherical_d_orthonormal_and_kinetic():
    """One d primitive on one centre: the five functions of Table A.1 are
    orthonormal (the weights give every real solid harmonic the same norm),
    and <-1/2 lap> of a normalised Gaussian of angular momentum l is
    zeta (l + 3/2) = 7 zeta / 2."""
    z = 0.7
    s = one_atom(((2, (z,), (1.0,)),), spherical=True)
    S, T = basis.overlap_kinetic_system(s)
    assert S.shape == (5, 5)
    assert np.max(np.abs(S - np.eye(5))) < 1e-14
    assert np.max(np.abs(T - 3.5 * z * np.eye(5))) < 1e-13


def test_cartesian_d_overlaps():
    """Cartesian d on one centre: x^2 and y^2 overlap by <x^2 y^2>/<x^4> =
    1/3 once normalised, and xy is orthogonal to both.  Kinetic energy
    T = 1/2 sum_d <(d_d phi)^2> / <phi^2> with Gaussian moments of variance
    1/(4 zeta): xy is a pure l = 2 function, 7 zeta / 2; x^2 mixes in the
    s-type r^2/3, 13 zeta / 6."""
    z = 1.3
    s = one_atom(((2, (z,), (1.0,)),), spherical=False)
    S, T = basis.overlap_kinetic_system(s)
    # order xx, yy, zz, xy, xz, yz
    assert abs(S[0, 1] - 1.0 / 3.0) < 1e-14 and abs(S[1, 2] - 1.0 / 3.0) < 1e-14
    assert np.max(np.abs(S[:3, 3:])) < 1e-15
    assert abs(T[0, 0] - 13.0 / 6.0 * z) < 1e-13 and abs(T[3, 3] - 3.5 * z) < 1e-13


def test_solid_harmonics_square_sum_is_rotation_invariant():
    """sum_m Phi_2m(r)^2 depends on |r| only (the degree-2 real solid
    harmonics of Table A.1 span a rotation-invariant space with equal
    weights): equal at random directions of one radius, and equal to r^4."""
    rng = np.random.default_rng(3)
    u = rng.normal(size=(20, 3))
    pts = 1.3 * u / np.linalg.norm(u, axis=1)[:, None]
    tot = np.zeros(len(pts))
    for comp in basis.SOLID[2]:
        val = np.zeros(len(pts))
        for (i, j, k), wgt in comp:
            val += wgt * pts[:, 0] ** i * pts[:, 1] ** j * pts[:, 2] ** k
        tot += val ** 2
    assert np.max(np.abs(tot - tot[0])) < 1e-12 * tot[0]
    # and equal to r^4 (along z only m = 0 is nonzero, (z^2)^2 = r^4)
    assert abs(tot[0] - 1.3 ** 4) < 1e-12


def test_closed_form_matches_fine_grid_sums_contracted():
    """Eq. 2.1 on a fine grid (plain sums of phi_a phi_b over all points, no
    windows) converges to the closed-form overlap of contracted functions
    with s, p and spherical d shells on two centres."""
    shells = ((0, (3.0, 1.0), (0.3, 0.8)), (1, (1.2, 0.5), (0.5, 0.6)), (2, (0.9,), (1.0,)))
    xyz = np.array([[0.0, 0.0, 0.0], [0.9, 0.4, -1.1]])
    s = w.make_system(xyz, h=0.1, pad=6.0, shells=shells, spherical=True)
    S, _ = basis.overlap_kinetic_system(s)
    Sg = grid_ops.potential_matrix(s, np.ones(tuple(int(t) for t in s.grid_n[::-1])), windowed=False, planes=8)
    assert np.max(np.abs(Sg - S)) < 1e-9


def test_quadrature_and_collocation_agree_for_contracted_functions():
    """For contracted functions the dense quadrature (slab by slab) and the
    separable one agree, and h^3 sum_g n = 2 Tr[P S_grid] with the same
    windows (Eqs. 2.1, 2.7), for a symmetric P."""
    s = w.config_system("dtiny5")
    shp = tuple(int(t) for t in s.grid_n[::-1])
    Sg = grid_ops.potential_matrix(s, np.ones(shp))
    Ss = grid_ops.potential_matrix_separable(s, [tuple(np.ones(int(k)) for k in s.grid_n)])
    assert np.max(np.abs(Sg - Ss)) < 1e-12
    rng = np.random.default_rng(1)
    A = rng.normal(size=Sg.shape) * 0.05
    P = A + A.T
    n = grid_ops.density_on_grid(s, P)
    assert abs(s.grid_h ** 3 * n.sum() - 2.0 * np.sum(P * Sg)) < 1e-10 * max(1.0, abs(n.sum()))


def test_energy_gradient_with_contracted_d_basis():
    """The directional derivative of E(P) is 2 Tr[D F] also for the
    contracted basis with d shells (Eq. 2.6 from the energy terms)."""
    xyz = np.array([[0.0, 0.0, 0.0], [2.3, 0.7, -0.4]])
    s = w.make_system(xyz, h=0.4, shells=w.si_clusters.SHELL_SPEC_D, spherical=True)
    st = scf.setup(s, scf.Model(neutral=True))
    r = scf.step(st, scf.ion_density(s))
    P = r["P"]
    rng = np.random.default_rng(5)
    A = rng.normal(size=P.shape) * 0.02
    D = A + A.T

    def E(eps):
        Pe = P + eps * D
        return scf.energy(st, Pe, grid_ops.density_on_grid(s, Pe, st.model.eta))["total"]
    fd = (E(1e-4) - E(-1e-4)) / 2e-4
    v, _, _ = scf.potential(st, grid_ops.density_on_grid(s, P, st.model.eta))
    an = 2.0 * float(np.sum(D * scf.fock(st, v)))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)
