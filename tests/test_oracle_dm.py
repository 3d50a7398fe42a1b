"""Pins for oracle.dm: eigensolve identities, Fermi-Dirac DM identities
(Eqs. 2.8, 2.9), and the Chebyshev expansion of Supp. B by brute force."""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import dm


def random_pair(K, seed, gap=None):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(K, K))
    S = A @ A.T / K + np.eye(K)              # SPD, modest condition
    B = rng.normal(size=(K, K))
    F = (B + B.T) / 2
    if gap is not None:
        # put a spectral gap of `gap` in the middle of S^-1 F
        eps, C = dm.geneig(F, S)
        eps = np.where(np.arange(K) < K // 2, eps - gap / 2, eps + gap / 2)
        Sc = S @ C
        F = Sc @ np.diag(eps) @ Sc.T
        F = (F + F.T) / 2
    return F, S


def test_geneig_identities():
    F, S = random_pair(24, 0)
    eps, C = dm.geneig(F, S)
    assert np.max(np.abs(F @ C - S @ C * eps[None, :])) < 1e-12
    assert np.max(np.abs(C.T @ S @ C - np.eye(24))) < 1e-12


def test_exact_dm_identities():
    F, S = random_pair(30, 1)
    r = dm.dm_exact(F, S, n_e=20.0, beta=7.0)
    P = r["P"]
    assert abs(2 * np.trace(P @ S) - 20.0) < 1e-10          # Eq. 2.8
    assert np.max(np.abs(F @ P @ S - S @ P @ F)) < 1e-10 * np.abs(F).max()   # f(S^-1F)S^-1 commutes
    assert abs(2 * np.trace(P @ F) - 2 * np.sum(r["occ"] * r["eps"])) < 1e-10
    assert np.max(np.abs(P - P.T)) < 1e-12


def test_zero_temperature_idempotent_in_s_metric():
    F, S = random_pair(30, 2, gap=2.0)
    r = dm.dm_exact(F, S, n_e=30.0, beta=200.0)
    P = r["P"]
    assert np.max(np.abs(P @ S @ P - P)) < 1e-10


def test_fermi_definition():
    e = np.linspace(-3, 3, 13)
    assert np.allclose(dm.fermi(e, 0.4, 2.5), 1.0 / (1.0 + np.exp(2.5 * (e - 0.4))), rtol=1e-14, atol=1e-16)


def test_coeffs_match_dct_ii():
    """a_l from the direct sum equal the DCT-II of the node values (the
    paper's 'FFT methods', Supp. B)."""
    mu, beta, lo, hi, n_c = 0.3, 40.0, -1.7, 2.2, 300
    m = 8 * n_c
    a = dm.cheb_coeffs(mu, beta, lo, hi, n_c)
    th = np.pi * (np.arange(m) + 0.5) / m
    fk = dm.fermi(0.5 * (hi + lo) + 0.5 * (hi - lo) * np.cos(th), mu, beta)
    y = scipy.fft.dct(fk, type=2) / m
    y[0] *= 0.5
    assert np.max(np.abs(a - y[:n_c])) < 1e-14


def test_expansion_converges_to_fermi_with_tail_bound():
    mu, beta, lo, hi = 0.1, 30.0, -2.0, 2.0
    n_c = dm.cheb_order(mu, beta, lo, hi, 1e-10)
    a = dm.cheb_coeffs(mu, beta, lo, hi, 4 * n_c)
    tail = np.sum(np.abs(a[n_c:]))
    x = np.linspace(-1, 1, 2001)
    p = dm.cheb_eval(x, a[:n_c])
    f = dm.fermi(0.5 * (hi + lo) + 0.5 * (hi - lo) * x, mu, beta)
    err = np.max(np.abs(p - f))
    assert tail < 1e-10
    assert err <= tail + 1e-13
    # the paper's rule of thumb N_C ~ 2 dE beta is the right order
    assert 1.0 < n_c / (2 * 0.5 * (hi - lo) * beta) < 10.0


def test_cheb_eval_matches_cosine_form():
    a = np.random.default_rng(4).normal(size=40)
    x = np.linspace(-1, 1, 77)
    ref = np.cos(np.outer(np.arccos(x), np.arange(40))) @ a
    assert np.max(np.abs(dm.cheb_eval(x, a) - ref)) < 1e-12


@pytest.mark.parametrize("form", ["paper", "symmetric"])
def test_matrix_recurrence_equals_eigenvalue_form(form):
    """Brute force on a small pair: the three-term matrix recurrence of
    Supp. B reaches C p(x) C^T."""
    F, S = random_pair(20, 5)
    eps, C = dm.geneig(F, S)
    lo, hi = eps[0] - 0.1, eps[-1] + 0.1
    a = dm.cheb_coeffs(0.2, 5.0, lo, hi, 60)
    x = (eps - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    ref = (C * dm.cheb_eval(x, a)[None, :]) @ C.T
    got = dm.dm_cheb_recurrence(F, S, a, lo, hi, form)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_diagonal_reduces_to_scalar():
    d = np.array([-1.0, -0.3, 0.05, 0.4, 1.3])
    F, S = np.diag(d), np.eye(5)
    lo, hi = -1.5, 1.5
    a = dm.cheb_coeffs(0.1, 20.0, lo, hi, 400)
    got = dm.dm_cheb_recurrence(F, S, a, lo, hi, "paper")
    assert np.max(np.abs(got - np.diag(dm.fermi(d, 0.1, 20.0)))) < 1e-12


def test_cheb_dm_mu_and_count():
    F, S = random_pair(26, 6)
    eps = dm.geneig(F, S)[0]
    lo, hi = eps[0] - 0.05, eps[-1] + 0.05
    r = dm.dm_cheb(F, S, 14.0, 6.0, lo, hi, 200)
    assert abs(2 * np.trace(r["P"] @ S) - 14.0) < 1e-10
    # N(mu) is increasing around the solution
    mus = r["mu"] + np.linspace(-0.5, 0.5, 11)
    counts = [dm.electron_count(m, 6.0, lo, hi, r["moments"]) for m in mus]
    assert np.all(np.diff(counts) > 0)
    # moments equal the traces of T_l(H_N) computed by the matrix recurrence
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    HN = (Li @ F @ Li.T - 0.5 * (hi + lo) * np.eye(26)) / (0.5 * (hi - lo))
    X0, X1 = np.eye(26), HN.copy()
    tr = [np.trace(X0), np.trace(X1)]
    for _ in range(2, 20):
        X0, X1 = X1, 2 * HN @ X1 - X0
        tr.append(np.trace(X1))
    assert np.max(np.abs(np.array(tr) - r["moments"][:20])) < 1e-10
    # exact and truncated DMs agree once the expansion has converged
    ex = dm.dm_exact(F, S, 14.0, 6.0)
    assert np.max(np.abs(ex["P"] - r["P"])) < 1e-9


def test_doubling_moments_equal_direct_traces():
    """T_m T_n = (T_{m+n} + T_{|m-n|}) / 2 gives m_{2l} = 2 <X_l, X_l> - m_0 and
    m_{2l+1} = 2 <X_{l+1}, X_l> - m_1 from the first half of the recurrence
    (Supp. B's moments, the doubling the moments pass relies on); they must
    equal the oracle's moments taken from the eigenvalues."""
    K, n_half = 21, 30
    F, S = random_pair(K, 11)
    eps = dm.geneig(F, S)[0]
    lo, hi = eps[0] - 0.2, eps[-1] + 0.3
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    HN = (Li @ F @ Li.T - 0.5 * (hi + lo) * np.eye(K)) / (0.5 * (hi - lo))
    X = [np.eye(K), HN.copy()]
    for _ in range(2, n_half + 1):
        X.append(2 * HN @ X[-1] - X[-2])
    m0, m1 = float(K), float(np.trace(HN))
    dbl = np.zeros(2 * n_half)
    for l in range(n_half):
        dbl[2 * l] = 2 * np.sum(X[l] * X[l]) - m0
        dbl[2 * l + 1] = 2 * np.sum(X[l + 1] * X[l]) - m1
    x = (eps - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    ref = dm.moments_from_eigs(x, 2 * n_half)
    assert np.max(np.abs(dbl - ref)) < 1e-10 * K
    # and against the cosine form on [-1, 1]: T_l(cos t) = cos(l t)
    assert np.max(np.abs(ref - np.cos(np.outer(np.arange(2 * n_half), np.arccos(x))).sum(1))) < 1e-10 * K


def test_empty_and_full_occupation():
    """Degenerate fillings: N_e -> 0 leaves P -> 0, N_e -> 2K fills every
    state so that P -> S^-1 (f(S^-1 F) -> I), for the exact and the Chebyshev
    density matrix alike."""
    K = 18
    F, S = random_pair(K, 21)
    eps = dm.geneig(F, S)[0]
    lo, hi = eps[0] - 0.1, eps[-1] + 0.1
    beta = 4.0
    n_c = dm.cheb_order(0.5 * (lo + hi), beta, lo, hi, 1e-12)
    Si = np.linalg.inv(S)
    for n_e, ref in ((1e-9, np.zeros((K, K))), (2 * K - 1e-9, Si)):
        ex = dm.dm_exact(F, S, n_e, beta)
        ch = dm.dm_cheb(F, S, n_e, beta, lo, hi, n_c)
        for r in (ex, ch):
            assert abs(2 * np.trace(r["P"] @ S) - n_e) < 1e-8
            assert np.max(np.abs(r["P"] - ref)) < 1e-8 * max(1.0, np.max(np.abs(Si)))
