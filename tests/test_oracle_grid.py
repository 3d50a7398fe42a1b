"""Pins for oracle.grid_ops (Eqs. 2.1, 2.5, 2.7, A.5, A.6), oracle.poisson
and the energy's translation invariance."""
import math

import numpy as np
import pytest
from scipy import special

import workloads as w
from oracle import basis, dm, grid_ops, poisson, scf


@pytest.fixture(scope="module")
def tiny():
    s = w.config_system("tiny8")
    fn = basis.functions(s)
    S, T = basis.overlap_kinetic(fn)
    return s, fn, S, T


def test_unit_potential_is_grid_overlap(tiny):
    s, fn, S, _ = tiny
    ones = np.ones(tuple(int(t) for t in s.grid_n[::-1]))
    Sg = grid_ops.potential_matrix(s, ones)
    assert np.max(np.abs(Sg - Sg.T)) < 1e-14
    # the grid overlap approaches the closed form (h sqrt(zeta_max) = 0.87 here,
    # so only the smooth functions agree closely)
    smooth = np.nonzero(fn["zeta"] <= 0.3)[0]
    assert np.max(np.abs(Sg[np.ix_(smooth, smooth)] - S[np.ix_(smooth, smooth)])) < 2e-3


def test_linearity_and_symmetry(tiny):
    s, fn, _, _ = tiny
    rng = np.random.default_rng(0)
    shp = tuple(int(t) for t in s.grid_n[::-1])
    v1, v2 = rng.normal(size=shp), rng.normal(size=shp)
    A = grid_ops.potential_matrix(s, v1)
    B = grid_ops.potential_matrix(s, v2)
    C = grid_ops.potential_matrix(s, 2.5 * v1 - 0.5 * v2)
    assert np.max(np.abs(C - (2.5 * A - 0.5 * B))) < 1e-12
    assert np.max(np.abs(A - A.T)) < 1e-13


def test_quadrature_matches_direct_pair_sums(tiny):
    """Table-based V against a direct evaluation of Eq. A.6 restricted to
    the window intersection box, pair by pair."""
    s, fn, _, _ = tiny
    rng = np.random.default_rng(1)
    v = rng.normal(size=tuple(int(t) for t in s.grid_n[::-1]))
    V = grid_ops.potential_matrix(s, v)
    K = len(fn["zeta"])
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, K, (25, 2))] + [(0, 0), (3, 77), (44, 45)]
    got = grid_ops.potential_entries(s, v, pairs)
    ref = np.array([V[a, b] for a, b in pairs])
    assert np.max(np.abs(got - ref)) < 1e-12


def test_window_error_bound(tiny):
    s, fn, _, _ = tiny
    v = np.cos(np.arange(s.n_grid) * 0.37).reshape(tuple(int(t) for t in s.grid_n[::-1]))
    for eta in (1e-4, 1e-8):
        Vw = grid_ops.potential_matrix(s, v, eta=eta)
        Vf = grid_ops.potential_matrix(s, v, windowed=False)
        assert np.max(np.abs(Vw - Vf)) <= 3.0 * np.max(np.abs(v)) * math.sqrt(3 * eta)
    assert np.max(np.abs(grid_ops.potential_matrix(s, v, eta=1e-4) - Vf)) > 1e-9


def test_density_count_and_pair_density(tiny):
    s, fn, _, _ = tiny
    K = len(fn["zeta"])
    rng = np.random.default_rng(2)
    A = rng.normal(size=(K, K)) * 0.1
    P = A + A.T
    n = grid_ops.density_on_grid(s, P)
    ones = np.ones_like(n)
    Sg = grid_ops.potential_matrix(s, ones)
    assert abs(s.grid_h ** 3 * n.sum() - 2 * np.sum(P * Sg)) < 1e-10 * max(1.0, abs(n.sum()))
    # P = e_a e_b^T + e_b e_a^T gives n = 4 phi_a phi_b (windowed) pointwise
    a, b = 5, 17
    E = np.zeros((K, K))
    E[a, b] = E[b, a] = 1.0
    nab = grid_ops.density_on_grid(s, E)
    lo, hi = basis.window_ranges(s, fn, 1e-10)
    xs = [s.grid_origin[d] + s.grid_h * np.arange(s.grid_n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    ph = basis.phi_at({k: v[[a, b]] for k, v in fn.items()}, pts)
    iz, iy, ix = np.meshgrid(*[np.arange(s.grid_n[d]) for d in (2, 1, 0)], indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1)
    inside = lambda f: np.all((idx >= lo[f]) & (idx <= hi[f]), axis=1)
    ref = 4 * ph[:, 0] * ph[:, 1] * inside(a) * inside(b)
    assert np.max(np.abs(nab.ravel() - ref)) < 1e-13
    # sampled evaluation agrees with the full grid
    pick = rng.integers(0, n.size, 40)
    assert np.max(np.abs(grid_ops.density_at(s, P, pick) - n.ravel()[pick])) < 1e-12
    # the absolute-term sum bounds |n|, and equals n for a nonnegative P on s functions
    A = grid_ops.density_at(s, P, pick, absolute=True)
    assert np.all(A >= np.abs(n.ravel()[pick]) - 1e-13)
    sfun = np.nonzero(fn["l"] == 0)[0]
    Ps = np.zeros((K, K))
    Ps[np.ix_(sfun, sfun)] = np.abs(P[np.ix_(sfun, sfun)])
    assert np.max(np.abs(grid_ops.density_at(s, Ps, pick, absolute=True) - grid_ops.density_at(s, Ps, pick))) < 1e-13


def test_cube_constant_closed_form():
    assert abs(poisson.cube_inv_r_constant() - (3 * math.log(2 + math.sqrt(3)) - math.pi / 2)) < 1e-12


def test_fft_size():
    assert poisson.fft_size(154) == 160 and poisson.fft_size(97) == 98 and poisson.fft_size(1) == 1


def test_fft_convolution_equals_direct_sum():
    s = w.make_system(np.array([[0.0, 0.0, 0.0]]), h=0.5, pad=2.2)
    rho = np.random.default_rng(3).normal(size=tuple(int(t) for t in s.grid_n[::-1]))
    a = poisson.hartree(s, rho)
    b = poisson.hartree_direct(s, rho)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_gaussian_charge_potential():
    """rho = q (alpha/pi)^(3/2) exp(-alpha r^2) has v = q erf(sqrt(alpha) r)/r;
    the discrete convolution converges to it as h -> 0."""
    q, alpha = 2.0, 0.8
    errs = []
    for h in (0.4, 0.2):
        s = w.make_system(np.array([[0.0, 0.0, 0.0]]), h=h, pad=7.0)
        xs, ys, zs = scf.grid_points(s)
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        r = np.sqrt(X * X + Y * Y + Z * Z)
        rho = q * (alpha / math.pi) ** 1.5 * np.exp(-alpha * r * r)
        v = poisson.hartree(s, rho)
        with np.errstate(invalid="ignore", divide="ignore"):
            ref = np.where(r > 1e-12, q * special.erf(math.sqrt(alpha) * r) / np.where(r > 0, r, 1), q * 2 * math.sqrt(alpha / math.pi))
        errs.append(np.max(np.abs(v - ref)) / np.max(ref))
    assert errs[0] < 1e-2 and errs[1] < 0.3 * errs[0], errs


def test_slater_exchange_closed_form():
    n = np.array([math.pi / 3, 1.0, 8.0, 0.0, -1e-3])
    vx, ex = poisson.slater_exchange(n)
    assert abs(vx[0] + 1.0) < 1e-15
    assert abs(vx[2] - 2 * vx[1]) < 1e-14
    assert np.allclose(vx[:3], 4.0 / 3.0 * ex[:3], rtol=1e-15)
    assert vx[3] == 0 and vx[4] == 0 and ex[4] == 0


def test_energy_translation_invariance():
    """Moving every atom and the grid by one grid vector leaves one SCF
    step's energy unchanged (to roundoff)."""
    s = w.config_system("tiny8")
    r1 = scf.step(scf.setup(s), scf.ion_density(s))
    sh = np.array([s.grid_h, -2 * s.grid_h, s.grid_h])
    s2 = w.make_system(s.xyz + sh, h=s.grid_h, grid_n=s.grid_n, grid_origin=s.grid_origin + sh)
    r2 = scf.step(scf.setup(s2), scf.ion_density(s2))
    assert abs(r1["E"]["total"] - r2["E"]["total"]) < 1e-9 * abs(r1["E"]["total"])


def test_band_energy_double_counting_identity():
    """2 Tr[P V[v]] = h^3 sum v n[P] for any v (quadrature and collocation use
    the same windowed functions)."""
    s = w.config_system("tiny8")
    st = scf.setup(s)
    n0 = scf.ion_density(s)
    r = scf.step(st, n0)
    V = r["F"] - st.T
    assert abs(2 * np.sum(r["P"] * V) - s.grid_h ** 3 * np.sum(r["v"] * r["n_out"])) < 1e-9


def test_poisson_far_field_and_linearity():
    """Far from a compact charge Q the potential tends to Q/|r - r_c| (r_c its
    centroid), with the quadrupole remainder falling like 1/r^3; the solve is
    linear in the charge."""
    s = w.make_system(np.array([[0.0, 0.0, 0.0]]), h=0.4, pad=6.0)
    nx, ny, nz = (int(t) for t in s.grid_n)
    rng = np.random.default_rng(7)
    rho = np.zeros((nz, ny, nx))
    c = [n // 2 for n in (nz, ny, nx)]
    rho[c[0] - 2:c[0] + 3, c[1] - 2:c[1] + 3, c[2] - 2:c[2] + 3] = rng.uniform(0.0, 1.0, (5, 5, 5))
    h3 = s.grid_h ** 3
    Q = h3 * rho.sum()
    xs, ys, zs = scf.grid_points(s)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    rc = np.array([np.sum(rho * X), np.sum(rho * Y), np.sum(rho * Z)]) * h3 / Q
    d = np.sqrt((X - rc[0]) ** 2 + (Y - rc[1]) ** 2 + (Z - rc[2]) ** 2)
    v = poisson.hartree(s, rho)
    rel = np.abs(v * d / Q - 1.0)
    far, mid = d > 9.0, (d > 4.0) & (d < 5.0)
    assert rel[far].max() < 2e-3
    assert rel[far].max() < rel[mid].max()
    rho2 = rng.normal(size=rho.shape)
    v2 = poisson.hartree(s, rho2)
    v3 = poisson.hartree(s, 1.5 * rho - 2.0 * rho2)
    assert np.max(np.abs(v3 - (1.5 * v - 2.0 * v2))) < 1e-12 * np.max(np.abs(v3))


def test_energy_invariant_under_quarter_turn():
    """A 90-degree turn of the atoms about z, on a grid centred on the axis
    with equal x and y sizes, maps the grid, the windows and the s/p shells
    onto themselves: one SCF step's energy is unchanged and the density turns
    with the atoms."""
    h, n = 0.4, 43
    xyz = np.array([[0.0, 0.0, 0.0], [2.3, 0.7, -0.4], [-1.1, 1.9, 0.8]])
    c = 0.5 * (n - 1) * h
    nz = int(math.ceil((1.2 + 12.0) / h)) + 1
    org = np.array([-c, -c, -0.4 - 6.0])
    s1 = w.make_system(xyz, h=h, grid_n=np.array([n, n, nz]), grid_origin=org)
    rot = np.stack([-xyz[:, 1], xyz[:, 0], xyz[:, 2]], 1)
    s2 = w.make_system(rot, h=h, grid_n=np.array([n, n, nz]), grid_origin=org)
    r1 = scf.step(scf.setup(s1), scf.ion_density(s1))
    r2 = scf.step(scf.setup(s2), scf.ion_density(s2))
    assert abs(r1["E"]["total"] - r2["E"]["total"]) < 1e-9 * abs(r1["E"]["total"])
    # point (x, y) of the first grid is point (-y, x) of the second
    n1, n2 = r1["n_out"], r2["n_out"]
    assert np.max(np.abs(n2 - n1[:, ::-1, :].transpose(0, 2, 1))) < 1e-10 * np.max(n1)


@pytest.mark.parametrize("neutral,full", [(False, False), (True, False), (True, True)])
def test_energy_gradient_is_the_fock_matrix(neutral, full):
    """The Kohn-Sham potential is the functional derivative of the energy
    (Eq. 2.6 from the energy terms): for n = n[P] the directional derivative
    of E(P) along a symmetric D is 2 Tr[D F[n(P)]], F = T + V^NL + V[v_KS].
    A wrong Hartree factor, an exchange or correlation potential that is not
    d(n eps_xc)/dn, a wrong sign on the ionic charge, or a non-local energy
    that is not 2 Tr[P V^NL] all break it.  full: with the KB projectors
    (s and p) and PW92 correlation."""
    from oracle import pseudo
    xyz = np.array([[0.0, 0.0, 0.0], [2.3, 0.7, -0.4], [-1.1, 1.9, 0.8]])
    s = w.make_system(xyz, h=0.4)
    st = scf.setup(s, scf.Model(neutral=neutral, nl=pseudo.KB() if full else None, pw92=full))
    r = scf.step(st, scf.ion_density(s))
    P = r["P"]
    K = P.shape[0]
    rng = np.random.default_rng(5)
    A = rng.normal(size=(K, K)) * 0.02
    for D in (P, A + A.T):
        def E(eps):
            Pe = P + eps * D
            return scf.energy(st, Pe, grid_ops.density_on_grid(s, Pe, st.model.eta))["total"]
        eps = 1e-4
        fd = (E(eps) - E(-eps)) / (2 * eps)
        v, _, _ = scf.potential(st, grid_ops.density_on_grid(s, P, st.model.eta))
        an = 2.0 * float(np.sum(D * scf.fock(st, v)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_separable_quadrature_equals_grid_sum(tiny):
    """The factorised quadrature of a sum of separable potentials equals the
    plain grid sum of Eq. 2.5 over the same windows (and without them)."""
    s, fn, _, _ = tiny
    nx, ny, nz = (int(t) for t in s.grid_n)
    rng = np.random.default_rng(9)
    factors = [tuple(rng.normal(size=n) for n in (nx, ny, nz)) for _ in range(2)]
    # a factor that vanishes on most lines, so that whole functions drop out
    band = [np.where(np.abs(np.arange(n) - n // 3) < 3, rng.normal(size=n), 0.0) for n in (nx, ny, nz)]
    factors.append(tuple(band))
    v = sum(np.einsum("z,y,x->zyx", fz, fy, fx) for fx, fy, fz in factors)
    for windowed in (True, False):
        ref = grid_ops.potential_matrix(s, v, windowed=windowed)
        got = grid_ops.potential_matrix_separable(s, factors, windowed=windowed)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # the sum of absolute terms bounds |V| and equals it where no term is
    # negative (s functions are positive; a positive one-term potential)
    A = grid_ops.potential_matrix_separable(s, factors, absolute=True)
    assert np.all(A >= np.abs(got) - 1e-13 * np.max(A))
    pos = [tuple(np.abs(f) for f in factors[0])]
    sfun = np.nonzero(fn["l"] == 0)[0]
    Vp = grid_ops.potential_matrix_separable(s, pos)[np.ix_(sfun, sfun)]
    Ap = grid_ops.potential_matrix_separable(s, pos, absolute=True)[np.ix_(sfun, sfun)]
    assert np.max(np.abs(Ap - Vp)) < 1e-13 * np.max(Ap)
    assert np.max(np.abs(grid_ops.potential_matrix_separable(s, pos, absolute=True) -
                         grid_ops.potential_matrix_separable(s, pos))) > 1e-6   # p functions change sign
