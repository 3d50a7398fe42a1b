"""Sparse-operator density-matrix columns (oracle): P u_alpha by the Chebyshev
recurrence on vectors, with S^-1 applied by preconditioned conjugate
gradients.

Test infrastructure only; see the package docstring.

Section 2 (the column-by-column traces, Eq. 2.10, and the passage after it)
applies the DM to one unit column at a time, rho_alpha = P u_alpha =
f_FD(S^-1 F) S^-1 u_alpha, with S^-1 v computed by PCG from repeated
products of the sparse overlap matrix (its footnote on PCG: incomplete
Cholesky preconditioning), and f_FD(S^-1 F) by the Chebyshev recurrence of
Supp. B: U_0 = S^-1 u_alpha, U_1 = H_N U_0, rho = a_0 U_0 + a_1 U_1, then
U_2 = 2 H_N U_1 - U_0 and rho += a_l U_2 for l = 2 .. N_C - 1, where
H_N v = (S^-1 (F v) - Ebar v) / dE.

Readings (the paper names the method and the HSL codes, not their settings):
  * sparsity: entries with |A_ij| <= thresh are dropped (thresh = 0 keeps
    every entry);
  * incomplete Cholesky IC(0): the Cholesky recurrence evaluated only on the
    lower pattern of the (thresholded) S, no fill-in; on a non-positive
    pivot the factorisation restarts on S + sigma diag(S) with sigma = 1e-3,
    doubled until it succeeds (the diagonal-shift rule of HSL MI28);
  * block-Jacobi: the exact inverse of each atom's diagonal block of S, a
    preconditioner applied independently per atom;
  * PCG stops per column when ||r||_2 <= tol ||b||_2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def sparsify(A, thresh=0.0):
    """CSR matrix of the entries of A with |A_ij| > thresh (all nonzeros
    when thresh = 0)."""
    A = np.asarray(A, dtype=np.float64)
    return sp.csr_matrix(np.where(np.abs(A) > thresh, A, 0.0))


def ic0(S, sigma0=1e-3, max_shifts=40):
    """IC(0) factor L (dense lower-triangular array) with L L^T ~ S + sigma
    diag(S), computed only on the lower nonzero pattern of S.  Returns
    (L, sigma) with sigma = 0 when no shift was needed.

    Left-looking column form: L_kk = sqrt(S_kk - sum_{j<k} L_kj^2),
    L_ik = (S_ik - sum_{j<k} L_ij L_kj) / L_kk for i > k with S_ik != 0."""
    A0 = S.toarray() if sp.issparse(S) else np.array(S, dtype=np.float64)
    K = A0.shape[0]
    pat = np.tril(A0 != 0.0)
    sigma = 0.0
    for _ in range(max_shifts):
        A = A0 + sigma * np.diag(np.diag(A0))
        L = np.zeros_like(A)
        ok = True
        for k in range(K):
            d = A[k, k] - L[k, :k] @ L[k, :k]
            if not d > 0.0:
                ok = False
                break
            L[k, k] = np.sqrt(d)
            col = (A[k + 1:, k] - L[k + 1:, :k] @ L[k, :k]) / L[k, k]
            L[k + 1:, k] = np.where(pat[k + 1:, k], col, 0.0)
        if ok:
            return L, sigma
        sigma = sigma0 if sigma == 0.0 else 2.0 * sigma
    raise RuntimeError("IC(0) failed after the diagonal shifts")


def ic0_apply(L):
    """z = (L L^T)^-1 r by a forward and a backward triangular solve."""
    import scipy.linalg as sla

    def apply(r):
        y = sla.solve_triangular(L, r, lower=True)
        return sla.solve_triangular(L.T, y, lower=False)
    return apply


def block_jacobi(S, atom_of):
    """z_I = (S_II)^-1 r_I for every atom I (basis functions grouped by
    the atom they sit on)."""
    A = S.toarray() if sp.issparse(S) else np.asarray(S, dtype=np.float64)
    atom_of = np.asarray(atom_of)
    blocks = [(idx, np.linalg.inv(A[np.ix_(idx, idx)])) for idx in
              (np.nonzero(atom_of == a)[0] for a in np.unique(atom_of))]

    def apply(r):
        z = np.empty_like(r)
        for idx, inv in blocks:
            z[idx] = inv @ r[idx]
        return z
    return apply


def pcg(A, b, apply_m, tol=1e-12, maxit=1000):
    """Preconditioned conjugate gradients for A x = b (A symmetric positive
    definite, one right-hand side), starting from x = 0.  Returns (x,
    iterations, ||r|| / ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = apply_m(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / nb
        if rel <= tol:
            return x, it, rel
        z = apply_m(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, rel


def columns(F, S, cols, a, e_min, e_max, thresh=0.0, tol=1e-12, precond="ic0", atom_of=None, maxit=1000):
    """rho_alpha = P u_alpha for alpha in cols by the vector recurrence with
    PCG solves (see the module docstring).  Returns (rho, stats): rho is
    K x len(cols), column c being P u_{cols[c]}; stats holds the PCG
    iteration counts and the largest relative residual."""
    Fs = sparsify(F, thresh)
    Ss = sparsify(S, thresh)
    K = Fs.shape[0]
    if precond == "ic0":
        L, _ = ic0(Ss)
        apply_m = ic0_apply(L)
    elif precond == "block_jacobi":
        apply_m = block_jacobi(Ss, atom_of)
    elif precond == "none":
        def apply_m(r):
            return r
    else:
        raise ValueError(precond)
    eb = 0.5 * (e_max + e_min)
    de = 0.5 * (e_max - e_min)
    its, worst = [], 0.0

    def s_inv(v):
        nonlocal worst
        x, it, rel = pcg(Ss, v, apply_m, tol, maxit)
        its.append(it)
        worst = max(worst, rel)
        return x

    def h_n(v):
        return (s_inv(Fs @ v) - eb * v) / de

    out = np.zeros((K, len(cols)))
    for c, alpha in enumerate(cols):
        u = np.zeros(K)
        u[alpha] = 1.0
        U0 = s_inv(u)
        rho = a[0] * U0
        if len(a) > 1:
            U1 = h_n(U0)
            rho = rho + a[1] * U1
            for l in range(2, len(a)):
                U2 = 2.0 * h_n(U1) - U0
                rho = rho + a[l] * U2
                U0, U1 = U1, U2
        out[:, c] = rho
    return out, dict(pcg_iterations=np.array(its), max_rel_residual=worst)
