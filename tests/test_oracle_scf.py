"""Pins of the oracle's SCF mixers (Section 2: Pulay/DIIS acceleration;
Kerker preconditioning) against closed forms and a textbook property."""
import types

import numpy as np

from oracle import scf


def _box(nx, ny, nz, h):
    return types.SimpleNamespace(grid_n=np.array([nx, ny, nz]), grid_h=h)


def test_kerker_plane_wave_eigenfunction():
    """A plane wave of the periodic box is an eigenfunction of the Kerker
    filter with eigenvalue G^2 / (G^2 + q0^2); a constant is removed."""
    nx, ny, nz, h, q0 = 12, 10, 8, 0.5, 0.8
    k = _box(nx, ny, nz, h)
    z, y, x = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    mx, my, mz = 2, 1, 3
    g = 2 * np.pi * np.array([mx / (nx * h), my / (ny * h), mz / (nz * h)])
    f = np.cos(g[0] * x + g[1] * y + g[2] * z)
    g2 = float(g @ g)
    out = scf.kerker(k, q0)(f)
    assert np.max(np.abs(out - g2 / (g2 + q0 * q0) * f)) < 1e-12
    assert np.max(np.abs(scf.kerker(k, q0)(np.full_like(f, 3.0)))) < 1e-12


def test_pulay_one_vector_is_linear_mixing():
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=50), rng.normal(size=50)
    mix = scf.Pulay(alpha=0.3, hist=1)
    assert np.allclose(mix(a, b), scf.linear_mix(0.3)(a, b), rtol=0, atol=1e-14)


def test_pulay_solves_affine_fixed_point_in_dim_plus_one_steps():
    """On n_out = M n_in + c, DIIS with unlimited history is equivalent to
    GMRES on (I - M) n = c, so it reaches the fixed point after at most
    dim + 1 residuals (exact arithmetic); a wrong sign, constraint or
    combination in the DIIS step breaks this."""
    dim = 6
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
    M = Q @ np.diag(np.linspace(-0.8, 0.9, dim)) @ Q.T
    c = rng.normal(size=dim)
    n_star = np.linalg.solve(np.eye(dim) - M, c)
    mix = scf.Pulay(alpha=0.5, hist=20)
    n = np.zeros(dim)
    for _ in range(dim + 2):
        n = mix(n, M @ n + c)
    assert np.max(np.abs(n - n_star)) < 1e-8
    # plain linear mixing is still far away after the same number of steps
    n_lin = np.zeros(dim)
    for _ in range(dim + 2):
        n_lin = scf.linear_mix(0.5)(n_lin, M @ n_lin + c)
    assert np.max(np.abs(n_lin - n_star)) > 1e-3


def test_gaussian_fields_of_one_atom():
    """Ionic charge and local potential of a lone atom: the charge sums to 4 e
    (a Gaussian of width 1.5 bohr sampled at h = 0.4 sums to its integral to
    roundoff, by the Poisson summation formula), the potential is -4 Ha at the
    nucleus and falls as exp(-r^2 / 1.5^2)."""
    import workloads as w
    s = w.make_system(np.array([[0.0, 0.0, 0.0]]), h=0.4, pad=8.0)
    n = scf.ion_density(s)
    assert abs(s.grid_h ** 3 * n.sum() - 4.0) < 1e-10
    v = scf.vloc(s)
    nx, ny, nz = (int(t) for t in s.grid_n)
    c = (nz // 2, ny // 2, nx // 2)
    xs, ys, zs = scf.grid_points(s)
    assert abs(xs[c[2]]) < 1e-12 and abs(ys[c[1]]) < 1e-12 and abs(zs[c[0]]) < 1e-12
    assert abs(v[c] + 4.0) < 1e-14
    r = xs[c[2] + 5]                                    # 2 bohr along x
    assert abs(v[c[0], c[1], c[2] + 5] + 4.0 * np.exp(-r * r / 2.25)) < 1e-14
    assert abs(n[c] - 4.0 * (np.pi * 2.25) ** -1.5) < 1e-14
