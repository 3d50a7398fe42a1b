"""Pins for oracle.sparse (the column-by-column sparse-operator route of
Section 2 with PCG solves): IC(0) against its definition and the cases where
it is the exact Cholesky factor, PCG against direct solves, and the vector
recurrence against the dense matrix recurrence of Supp. B."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import basis, dm
from oracle import sparse as osp


def spd(K, seed, density=1.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(K, K)) * (rng.random((K, K)) < density)
    return A @ A.T / K + np.eye(K)


def test_ic0_with_full_pattern_is_cholesky():
    S = spd(30, 0)
    L, sigma = osp.ic0(S)
    assert sigma == 0.0
    assert np.max(np.abs(L - np.linalg.cholesky(S))) < 1e-13


def test_ic0_of_tridiagonal_is_exact():
    # a tridiagonal matrix has no fill-in: IC(0) is its Cholesky factor
    K = 40
    rng = np.random.default_rng(1)
    off = rng.uniform(-0.4, 0.4, K - 1)
    S = np.diag(np.full(K, 1.0)) + np.diag(off, 1) + np.diag(off, -1)
    L, sigma = osp.ic0(sp.csr_matrix(S))
    assert sigma == 0.0
    assert np.max(np.abs(L @ L.T - S)) < 1e-14
    assert np.count_nonzero(np.tril(L, -2)) == 0


def test_ic0_residual_vanishes_on_the_pattern():
    # the defining property of IC(0): L keeps the lower pattern of S and
    # (L L^T)_ij = S_ij wherever S_ij != 0 (fill-in is only dropped elsewhere)
    s = w.config_system("tiny8")
    S, _ = basis.overlap_kinetic_system(s)
    Ss = osp.sparsify(S, 1e-3)
    A = Ss.toarray()
    L, sigma = osp.ic0(Ss)
    assert sigma == 0.0
    assert np.all((np.tril(L) != 0) <= (np.tril(A) != 0))
    R = L @ L.T - A
    assert np.max(np.abs(R[A != 0])) < 1e-13
    assert np.max(np.abs(R)) > 1e-6          # dropped fill-in: not the exact factor


def test_ic0_shift_on_breakdown():
    # a symmetric positive definite matrix whose IC(0) breaks down on its
    # pattern is factorised after the diagonal shift
    S = np.array([[3.0, -2.0, 0.0, 2.0], [-2.0, 3.0, -2.0, 0.0], [0.0, -2.0, 3.0, -2.0], [2.0, 0.0, -2.0, 3.0]])
    assert np.all(np.linalg.eigvalsh(S) > 0)
    with np.errstate(invalid="ignore"):
        L, sigma = osp.ic0(sp.csr_matrix(S))
    assert sigma > 0.0
    A = S + sigma * np.diag(np.diag(S))
    R = L @ L.T - A
    assert np.max(np.abs(R[A != 0])) < 1e-12


def test_pcg_matches_direct_solve():
    s = w.config_system("tiny8")
    S, _ = basis.overlap_kinetic_system(s)
    fn = basis.functions(s)
    b = np.random.default_rng(2).normal(size=S.shape[0])
    x_ref = np.linalg.solve(S, b)
    Ss = sp.csr_matrix(S)
    L, _ = osp.ic0(osp.sparsify(S, 1e-6))
    for apply_m in (lambda r: r, osp.ic0_apply(L), osp.block_jacobi(S, fn["atom"])):
        x, it, rel = osp.pcg(Ss, b, apply_m, tol=1e-13, maxit=5000)
        assert rel <= 1e-13
        assert np.linalg.norm(x - x_ref) < 1e-8 * np.linalg.norm(x_ref)


def test_pcg_with_exact_preconditioners_takes_one_iteration():
    S = spd(25, 3)
    b = np.random.default_rng(4).normal(size=25)
    inv = np.linalg.inv(S)
    _, it, rel = osp.pcg(S, b, lambda r: inv @ r, tol=1e-12)
    assert it == 1 and rel < 1e-12
    # block-Jacobi on a block-diagonal matrix is its exact inverse
    blocks = [spd(5, 10 + i) for i in range(5)]
    B = np.zeros((25, 25))
    for i, blk in enumerate(blocks):
        B[5 * i:5 * i + 5, 5 * i:5 * i + 5] = blk
    _, it, rel = osp.pcg(B, b, osp.block_jacobi(B, np.repeat(np.arange(5), 5)), tol=1e-12)
    assert it == 1 and rel < 1e-12


def test_pcg_without_preconditioner_is_cg_in_k_steps():
    # exact arithmetic CG ends in at most K steps; with 8 distinct
    # eigenvalues in at most 8
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(40, 40)))
    lam = np.repeat(np.linspace(1.0, 3.0, 8), 5)
    A = (Q * lam) @ Q.T
    _, it, rel = osp.pcg(A, rng.normal(size=40), lambda r: r, tol=1e-10)
    assert it <= 8 and rel <= 1e-10


def _tiny_problem(n_c=48):
    s = w.config_system("tiny8")
    S, T = basis.overlap_kinetic_system(s)
    K = S.shape[0]
    rng = np.random.default_rng(6)
    D = rng.normal(size=(K, K)) * 0.02
    F = T - 0.5 * S + (D + D.T) / 2          # symmetric, spectrum not that of T alone
    eps, _ = dm.geneig(F, S)
    e_min, e_max = eps[0] - 0.05, eps[-1] + 0.05
    mu = 0.5 * (eps[8] + eps[9])
    a = dm.cheb_coeffs(mu, 20.0, e_min, e_max, n_c)
    return s, F, S, a, e_min, e_max


@pytest.mark.parametrize("precond", ["ic0", "block_jacobi", "none"])
def test_columns_equal_dense_recurrence(precond):
    s, F, S, a, e_min, e_max = _tiny_problem()
    P = dm.dm_cheb_recurrence(F, S, a, e_min, e_max, form="paper")
    cols = [0, 7, 33, 79]
    rho, st = osp.columns(F, S, cols, a, e_min, e_max, thresh=0.0, tol=1e-14, precond=precond,
                          atom_of=basis.functions(s)["atom"], maxit=5000)
    assert st["max_rel_residual"] <= 1e-14
    assert np.max(np.abs(rho - P[:, cols])) < 1e-9 * np.max(np.abs(P))


def test_columns_give_the_electron_count():
    # 2 sum_alpha (S rho_alpha)_alpha = 2 Tr[S P] = 2 sum_l a_l Tr T_l(H_N)
    s, F, S, a, e_min, e_max = _tiny_problem(n_c=32)
    K = S.shape[0]
    rho, _ = osp.columns(F, S, list(range(K)), a, e_min, e_max, tol=1e-14, precond="ic0", maxit=5000)
    n_cols = 2.0 * np.trace(S @ rho)
    eps, _ = dm.geneig(F, S)
    x = (eps - 0.5 * (e_max + e_min)) / (0.5 * (e_max - e_min))
    n_eig = 2.0 * float(a @ dm.moments_from_eigs(x, len(a)))
    assert abs(n_cols - n_eig) < 1e-9 * K


def test_threshold_changes_columns_within_bound():
    # dropping entries below 1e-9 moves the columns by a small multiple of it
    s, F, S, a, e_min, e_max = _tiny_problem(n_c=32)
    cols = [3, 40]
    r0, _ = osp.columns(F, S, cols, a, e_min, e_max, thresh=0.0, tol=1e-14, maxit=5000)
    r1, _ = osp.columns(F, S, cols, a, e_min, e_max, thresh=1e-9, tol=1e-14, maxit=5000)
    d = np.max(np.abs(r1 - r0))
    assert 0.0 < d < 1e-4
