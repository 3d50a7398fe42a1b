"""Pins for oracle.basis: closed forms, brute-force grid integrals, Eq. A.4."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as w
from oracle import basis


def two_atom_system(d=(1.3, -0.7, 2.1), h=0.1, pad=6.0):
    xyz = np.array([[0.0, 0.0, 0.0], list(d)])
    return w.make_system(xyz, h=h, pad=pad)


def test_self_overlap_and_kinetic_diagonal():
    s = two_atom_system()
    fn = basis.functions(s)
    S, T = basis.overlap_kinetic(fn)
    assert np.allclose(np.diag(S), 1.0, atol=1e-14)
    # <-1/2 lap> of a normalised Cartesian Gaussian: 3 zeta/2 (s), 5 zeta/2 (p)
    expect = np.where(fn["l"] == 0, 1.5 * fn["zeta"], 2.5 * fn["zeta"])
    assert np.allclose(np.diag(T), expect, rtol=1e-13)


def test_same_centre_s_overlap_closed_form():
    s = two_atom_system()
    fn = basis.functions(s)
    S, _ = basis.overlap_kinetic(fn)
    z = fn["zeta"]
    for a in range(4):
        for b in range(4):
            exp = (2.0 * math.sqrt(z[a] * z[b]) / (z[a] + z[b])) ** 1.5
            assert abs(S[a, b] - exp) < 1e-14
    # s and p on the same centre are orthogonal by parity
    assert np.all(np.abs(S[:4, 4:10]) < 1e-15)


def test_two_centre_s_overlap_gaussian_product():
    s = two_atom_system()
    fn = basis.functions(s)
    S, T = basis.overlap_kinetic(fn)
    R2 = float(np.sum(np.array([1.3, -0.7, 2.1]) ** 2))
    for a in range(4):
        for b in range(10, 14):
            za, zb = fn["zeta"][a], fn["zeta"][b]
            p, mu = za + zb, za * zb / (za + zb)
            exp = (4 * za * zb / math.pi ** 2) ** 0.75 * (math.pi / p) ** 1.5 * math.exp(-mu * R2)
            assert abs(S[a, b] - exp) < 1e-14 * max(1, exp)
            # s-s kinetic: mu (3 - 2 mu R^2) S
            assert abs(T[a, b] - mu * (3 - 2 * mu * R2) * exp) < 1e-13


def test_symmetric_positive_definite():
    s = w.config_system("tiny8")
    S, T = basis.overlap_kinetic(basis.functions(s))
    assert np.max(np.abs(S - S.T)) < 1e-15 and np.max(np.abs(T - T.T)) < 1e-13
    assert np.linalg.eigvalsh(S).min() > 0
    assert np.linalg.eigvalsh(T).min() > 0


def test_closed_form_matches_fine_grid_sums():
    """Eqs. 2.1 and 2.2 on a fine grid (direct evaluation and analytic
    gradients, no tables, no windows) converge to the closed forms."""
    s = two_atom_system(d=(0.9, 0.4, -1.1), h=0.1, pad=7.0)
    fn = basis.functions(s)
    S, T = basis.overlap_kinetic(fn)
    # keep the diffuse shells out: they need a bigger box than a test wants
    keep = np.nonzero(fn["zeta"] >= 0.3)[0]
    sub = {k: v[keep] for k, v in fn.items()}
    xs = [s.grid_origin[d] + s.grid_h * np.arange(s.grid_n[d]) for d in range(3)]
    h3 = s.grid_h ** 3
    Sg = np.zeros((len(keep), len(keep)))
    Tg = np.zeros_like(Sg)
    for iz in range(len(xs[2])):
        Y, X = np.meshgrid(xs[1], xs[0], indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, xs[2][iz])], 1)
        ph = basis.phi_at(sub, pts)
        d = pts[:, None, :] - sub["center"][None]
        e = sub["norm"][None] * np.exp(-sub["zeta"][None] * (d * d).sum(-1))
        poly = [d[..., ax] ** sub["pw"][None, :, ax] for ax in range(3)]
        grad = []
        for ax in range(3):
            # d/dx [x^i e^{-z x^2}] = (i x^{i-1} - 2 z x^{i+1}) e^{-z x^2}
            i = sub["pw"][None, :, ax]
            dpoly = np.where(i > 0, i * d[..., ax] ** np.maximum(i - 1, 0), 0.0) - 2 * sub["zeta"][None] * d[..., ax] * poly[ax]
            others = [poly[b] for b in range(3) if b != ax]
            grad.append(e * dpoly * others[0] * others[1])
        Sg += h3 * ph.T @ ph
        Tg += 0.5 * h3 * sum(g.T @ g for g in grad)
    assert np.max(np.abs(Sg - S[np.ix_(keep, keep)])) < 1e-9
    assert np.max(np.abs(Tg - T[np.ix_(keep, keep)])) < 1e-8


@pytest.mark.parametrize("l", [0, 1, 2])
@pytest.mark.parametrize("eta", [1e-3, 1e-6, 1e-10])
def test_window_length_solves_charge_equation(l, eta):
    """Eq. A.4: c(L sqrt(zeta), l) = 1 - eta with c the normalised partial
    charge, checked by direct numerical integration."""
    zeta = 0.37
    L = float(basis.window_halfwidth(zeta, l, eta))
    d = L * math.sqrt(zeta)
    num = integrate.quad(lambda x: x ** l * math.exp(-x * x), d, np.inf, epsabs=0, epsrel=1e-12)[0]
    den = integrate.quad(lambda x: x ** l * math.exp(-x * x), 0, np.inf, epsabs=0, epsrel=1e-12)[0]
    assert abs(num / den - eta) < 1e-6 * eta


def test_tables_reproduce_direct_evaluation():
    s = w.config_system("tiny8")
    fn = basis.functions(s)
    tabs = basis.axis_tables(s, fn, None)
    rng = np.random.default_rng(3)
    ix = rng.integers(0, s.grid_n[0], 50)
    iy = rng.integers(0, s.grid_n[1], 50)
    iz = rng.integers(0, s.grid_n[2], 50)
    pts = s.grid_origin + s.grid_h * np.stack([ix, iy, iz], 1)
    direct = basis.phi_at(fn, pts)
    sep = tabs[0][ix] * tabs[1][iy] * tabs[2][iz]
    assert np.max(np.abs(direct - sep)) < 1e-14
