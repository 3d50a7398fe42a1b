"""Density matrix P = f_FD(S^-1 F) S^-1 (oracle).

Test infrastructure only; see the package docstring.

Two routes:
  * exact: generalised eigensolve F C = S C eps, P = C f(eps) C^T (Eq. 2.9;
    LAPACK dsygvd through scipy),
  * Chebyshev-truncated: the same matrix function with f replaced by its
    N_C-term Chebyshev expansion on [E_min, E_max] (Supp. B), evaluated
    either on the eigenvalues or by the three-term matrix recurrence.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def fermi(e, mu, beta):
    """f_FD(e) = 1 / (1 + exp(beta (e - mu)))  (Section 2), in the
    overflow-free form (1 - tanh(beta (e - mu) / 2)) / 2."""
    return 0.5 * (1.0 - np.tanh(0.5 * beta * (np.asarray(e) - mu)))


def geneig(F, S):
    """Generalised symmetric eigenproblem F C = S C eps with C^T S C = I."""
    eps, C = sla.eigh(F, S)
    return eps, C


def bisect(count, target, lo, hi, iters=200):
    """Root of count(mu) = target on [lo, hi] by bisection (the paper fixes
    mu through Eq. 2.8 but gives no method; bisection is the reading taken).
    count must be non-decreasing.  Stops when the bracket stops shrinking."""
    flo = count(lo) - target
    fhi = count(hi) - target
    if flo > 0 or fhi < 0:
        raise ValueError("mu bracket does not contain the electron count")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count(mid) - target < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def dm_exact(F, S, n_e, beta):
    """P = C f(eps) C^T with mu fixed by 2 Tr[PS] = 2 sum_i f(eps_i) = N_e
    (Eqs. 2.8, 2.9).  Returns dict(P, mu, eps, C, occ)."""
    eps, C = geneig(F, S)
    span = 40.0 / beta
    mu = bisect(lambda m: 2.0 * fermi(eps, m, beta).sum(), n_e, eps[0] - span, eps[-1] + span)
    occ = fermi(eps, mu, beta)
    P = (C * occ[None, :]) @ C.T
    return dict(P=P, mu=mu, eps=eps, C=C, occ=occ)


def cheb_coeffs(mu, beta, e_min, e_max, n_c, m_nodes=None):
    """Chebyshev coefficients of f_FD on [E_min, E_max] (Supp. B, Eq. B.1):
    f(Ebar + dE x) ~ sum_{l<N_C} a_l T_l(x), Ebar, dE the centre and half
    width.  The paper computes a_l by FFT; here the same Gauss-Chebyshev
    quadrature is summed directly:
      a_l = (2 - delta_l0)/M sum_k f(Ebar + dE cos th_k) cos(l th_k),
      th_k = pi (k + 1/2) / M,  M = 8 N_C unless given.
    """
    m = int(m_nodes) if m_nodes else 8 * int(n_c)
    eb = 0.5 * (e_max + e_min)
    de = 0.5 * (e_max - e_min)
    th = math.pi * (np.arange(m) + 0.5) / m
    fk = fermi(eb + de * np.cos(th), mu, beta)
    l = np.arange(n_c)
    a = (np.cos(np.outer(l, th)) @ fk) * (2.0 / m)
    a[0] *= 0.5
    return a


def cheb_eval(x, a):
    """p(x) = sum_l a_l T_l(x) by the scalar three-term recurrence
    T_{l+1} = 2x T_l - T_{l-1} (Supp. B)."""
    x = np.asarray(x, dtype=np.float64)
    t0 = np.ones_like(x)
    p = a[0] * t0
    if len(a) == 1:
        return p
    t1 = x.copy()
    p = p + a[1] * t1
    for l in range(2, len(a)):
        t2 = 2.0 * x * t1 - t0
        p = p + a[l] * t2
        t0, t1 = t1, t2
    return p


def cheb_order(mu, beta, e_min, e_max, tol, n_max=200000):
    """Smallest N_C with sum_{j >= N_C} |a_j| < tol (the paper's rule of
    thumb N_C ~ 2 dE beta is reported separately; the tail rule is the
    reading taken for a fixed accuracy)."""
    n = max(16, int(2 * beta * 0.5 * (e_max - e_min)))
    while True:
        a = cheb_coeffs(mu, beta, e_min, e_max, 4 * n)
        tail = np.cumsum(np.abs(a)[::-1])[::-1]
        ok = np.nonzero(tail < tol)[0]
        if len(ok) and ok[0] < 2 * n:
            return int(ok[0])
        n *= 2
        if n > n_max:
            raise ValueError("Chebyshev order above n_max")


def moments_from_eigs(x, n_c):
    """m_l = Tr T_l(H_N) = sum_i T_l(x_i) for the normalised eigenvalues."""
    x = np.asarray(x, dtype=np.float64)
    m = np.zeros(n_c)
    t0 = np.ones_like(x)
    m[0] = t0.sum()
    if n_c > 1:
        t1 = x.copy()
        m[1] = t1.sum()
    for l in range(2, n_c):
        t2 = 2.0 * x * t1 - t0
        m[l] = t2.sum()
        t0, t1 = t1, t2
    return m


def electron_count(mu, beta, e_min, e_max, mom, m_nodes=None):
    """N(mu) = 2 sum_l a_l(mu) m_l = 2 Tr p(H_N)  (Eq. 2.8 with the expansion)."""
    a = cheb_coeffs(mu, beta, e_min, e_max, len(mom), m_nodes)
    return 2.0 * float(a @ mom)


def dm_cheb(F, S, n_e, beta, e_min, e_max, n_c, m_nodes=None):
    """Chebyshev-truncated DM: P = C p(x) C^T with x = (eps - Ebar)/dE and mu
    by bisection on 2 sum_l a_l(mu) m_l = N_e.  This is the result the matrix
    recurrence of Supp. B reaches, evaluated in the eigenbasis."""
    eps, C = geneig(F, S)
    eb = 0.5 * (e_max + e_min)
    de = 0.5 * (e_max - e_min)
    x = (eps - eb) / de
    mom = moments_from_eigs(x, n_c)
    span = 40.0 / beta
    mu = bisect(lambda m: electron_count(m, beta, e_min, e_max, mom, m_nodes), n_e,
                e_min - span, e_max + span)
    a = cheb_coeffs(mu, beta, e_min, e_max, n_c, m_nodes)
    p = cheb_eval(x, a)
    P = (C * p[None, :]) @ C.T
    return dict(P=P, mu=mu, eps=eps, C=C, occ=p, moments=mom, coeffs=a)


def dm_cheb_recurrence(F, S, a, e_min, e_max, form="symmetric"):
    """Matrix three-term recurrence of Supp. B for given coefficients a.

    form="paper":     U_0 = S^-1 (all unit columns at once), U_1 = H_N U_0,
                      H = S^-1 F; rho = sum_l a_l U_l is P directly.
    form="symmetric": F~ = L^-1 F L^-T with S = L L^T, X_0 = I,
                      X_1 = H~_N, rho = sum_l a_l X_l, P = L^-T rho L^-1
                      (f(S^-1 F) S^-1 = L^-T f(F~) L^-1 in exact arithmetic).
    """
    K = F.shape[0]
    eb = 0.5 * (e_max + e_min)
    de = 0.5 * (e_max - e_min)
    if form == "paper":
        H = np.linalg.solve(S, F)
        HN = (H - eb * np.eye(K)) / de
        U0 = np.linalg.inv(S)
    else:
        L = np.linalg.cholesky(S)
        Li = sla.solve_triangular(L, np.eye(K), lower=True)
        HN = (Li @ F @ Li.T - eb * np.eye(K)) / de
        U0 = np.eye(K)
    rho = a[0] * U0
    U1 = HN @ U0
    if len(a) > 1:
        rho = rho + a[1] * U1
    for l in range(2, len(a)):
        U2 = 2.0 * HN @ U1 - U0
        rho = rho + a[l] * U2
        U0, U1 = U1, U2
    if form == "paper":
        return rho
    return Li.T @ rho @ Li
