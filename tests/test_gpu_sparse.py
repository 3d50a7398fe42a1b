"""The sparse-operator route (dft_density_matrix_columns): columns of P by the
Chebyshev recurrence on vectors with S^-1 by PCG on the sparse S (Section 2,
Eq. 2.10 and the passage after it; Supp. B), against the oracle's plain
column-by-column route and its dense matrix recurrence.

Inputs on both sides: F = T - 0.5 S + D with S, T computed independently by
each side and D a seeded random symmetric matrix; mu and the expansion
interval come from the oracle's eigenvalues."""
import numpy as np
import pytest

import workloads as w
from oracle import basis, dm
from oracle import sparse as osp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402


def problem(name, n_c, seed=6, precision=dft.DFT_PREC_FP64):
    s = w.config_system(name)
    S_o, T_o = basis.overlap_kinetic_system(s)
    K = S_o.shape[0]
    rng = np.random.default_rng(seed)
    D = rng.normal(size=(K, K)) * 0.02
    D = (D + D.T) / 2
    F_o = T_o - 0.5 * S_o + D
    eps, _ = dm.geneig(F_o, S_o)
    e_min, e_max = eps[0] - 0.05, eps[-1] + 0.05
    n_occ = int(round(s.n_electrons / 2))
    mu = 0.5 * (eps[n_occ - 1] + eps[n_occ])
    beta = 1.0 / s.kT
    a = dm.cheb_coeffs(mu, beta, e_min, e_max, n_c, m_nodes=4 * n_c)   # the library's node count
    ctx = dft.Context(s, precision=precision)
    S_g, T_g = ctx.overlap_kinetic()
    F_g = (T_g - 0.5 * S_g + torch.from_numpy(D).cuda()).contiguous()
    return dict(s=s, K=K, F_o=F_o, S_o=S_o, a=a, mu=mu, e_min=e_min, e_max=e_max, ctx=ctx, F_g=F_g, n_c=n_c)


def atom_of(s):
    return basis.functions(s)["atom"]


def test_columns_match_the_oracle():
    p = problem("tiny8", 96)
    cols = [0, 9, 41, 79]
    out, info = p["ctx"].density_matrix_columns(p["F_g"], cols, p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                pcg_tol=1e-12)
    got = out.cpu().numpy()
    ref, st = osp.columns(p["F_o"], p["S_o"], cols, p["a"], p["e_min"], p["e_max"], tol=1e-12,
                          precond="block_jacobi", atom_of=atom_of(p["s"]))
    dense = dm.dm_cheb_recurrence(p["F_o"], p["S_o"], p["a"], p["e_min"], p["e_max"], form="paper")[:, cols]
    scale = np.max(np.abs(dense))
    print(f"tiny8 columns: max|d| vs oracle columns {np.max(np.abs(got - ref)):.2e}, vs dense "
          f"{np.max(np.abs(got - dense)):.2e} (max|P| {scale:.2e}); PCG {info.pcg_iterations} iterations over "
          f"{info.pcg_solves} solves (oracle {st['pcg_iterations'].sum()} over {len(st['pcg_iterations'])})")
    assert info.not_converged == 0 and info.max_rel_residual <= 1e-12
    # thresh 0 keeps every nonzero: all entries above rounding level, at most all of the oracle's nonzeros
    # (entries that vanish by symmetry can be exact zeros on one side and 1e-14 on the other)
    assert np.count_nonzero(np.abs(p["S_o"]) > 1e-12) <= info.nnz_s <= np.count_nonzero(p["S_o"])
    assert info.pcg_solves == p["n_c"]
    assert np.max(np.abs(got - ref)) < 1e-9 * scale
    assert np.max(np.abs(got - dense)) < 1e-9 * scale
    p["ctx"].close()


@pytest.mark.parametrize("precond", [dft.DFT_PRECOND_BLOCK_JACOBI, dft.DFT_PRECOND_NONE])
def test_columns_with_threshold_match_the_oracle(precond):
    p = problem("tiny8", 64, seed=7)
    cols = [3, 50]
    thr = 1e-6
    out, info = p["ctx"].density_matrix_columns(p["F_g"], cols, p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                thresh=thr, precond=precond, pcg_tol=1e-12)
    name = "block_jacobi" if precond == dft.DFT_PRECOND_BLOCK_JACOBI else "none"
    ref, st = osp.columns(p["F_o"], p["S_o"], cols, p["a"], p["e_min"], p["e_max"], thresh=thr, tol=1e-12,
                          precond=name, atom_of=atom_of(p["s"]))
    nnz = osp.sparsify(p["S_o"], thr).nnz
    ref_its = int(st["pcg_iterations"].reshape(len(cols), p["n_c"]).max(axis=0).sum())
    print(f"thresh {thr}, {name}: nnz(S) {info.nnz_s} (oracle {nnz}), PCG {info.pcg_iterations} "
          f"(oracle {ref_its}), max|d| {np.max(np.abs(out.cpu().numpy() - ref)):.2e}")
    assert abs(info.nnz_s - nnz) <= 4          # entries at the threshold may round either way
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-9 * np.max(np.abs(ref))
    # the iteration counts follow the oracle's (the same method in FP64): per
    # solve the slowest column, within one iteration per solve for rounding
    assert abs(info.pcg_iterations - ref_its) <= p["n_c"]
    p["ctx"].close()


def test_block_jacobi_needs_fewer_iterations():
    p = problem("tiny8", 32)
    res = {}
    for pc in (dft.DFT_PRECOND_BLOCK_JACOBI, dft.DFT_PRECOND_NONE):
        out, info = p["ctx"].density_matrix_columns(p["F_g"], [5], p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                    precond=pc, pcg_tol=1e-12)
        res[pc] = (out.cpu().numpy(), info.pcg_iterations)
    a, b = res[dft.DFT_PRECOND_BLOCK_JACOBI], res[dft.DFT_PRECOND_NONE]
    print(f"PCG iterations: block-Jacobi {a[1]}, none {b[1]}")
    assert a[1] < b[1]
    assert np.max(np.abs(a[0] - b[0])) < 1e-9 * np.max(np.abs(a[0]))
    p["ctx"].close()


def test_columns_in_blocks_with_repeats():
    # 29 columns with a repeat: two blocks of at most K / 4 = 20 columns
    p = problem("tiny8", 48)
    cols = list(range(0, 80, 3)) + [0, 79]
    out, info = p["ctx"].density_matrix_columns(p["F_g"], cols, p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                pcg_tol=1e-12)
    got = out.cpu().numpy()
    assert info.block_cols == 20
    assert np.array_equal(got[:, 0], got[:, cols.index(0, 1)])
    dense = dm.dm_cheb_recurrence(p["F_o"], p["S_o"], p["a"], p["e_min"], p["e_max"], form="paper")[:, cols]
    assert np.max(np.abs(got - dense)) < 1e-9 * np.max(np.abs(dense))
    p["ctx"].close()


def test_all_columns_give_the_electron_count():
    # 2 sum_alpha (S rho_alpha)_alpha = 2 Tr[P S] = 2 sum_l a_l Tr T_l(H_N)
    p = problem("tiny8", 64)
    K = p["K"]
    out, _ = p["ctx"].density_matrix_columns(p["F_g"], list(range(K)), p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                             pcg_tol=1e-12)
    n_cols = 2.0 * np.trace(p["S_o"] @ out.cpu().numpy())
    eps, _ = dm.geneig(p["F_o"], p["S_o"])
    x = (eps - 0.5 * (p["e_max"] + p["e_min"])) / (0.5 * (p["e_max"] - p["e_min"]))
    n_eig = 2.0 * float(p["a"] @ dm.moments_from_eigs(x, p["n_c"]))
    print(f"electron count from the columns {n_cols:.12f}, from the eigenvalues {n_eig:.12f}")
    assert abs(n_cols - n_eig) < 1e-8 * K
    p["ctx"].close()


def test_columns_on_the_64_atom_cluster():
    p = problem("cluster64", 128)
    cols = [0, 333, 639]
    out, info = p["ctx"].density_matrix_columns(p["F_g"], cols, p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                pcg_tol=1e-12)
    dense = dm.dm_cheb_recurrence(p["F_o"], p["S_o"], p["a"], p["e_min"], p["e_max"], form="paper")[:, cols]
    d = np.max(np.abs(out.cpu().numpy() - dense))
    print(f"cluster64 columns: max|d| vs dense oracle {d:.2e} of {np.max(np.abs(dense)):.2e}; "
          f"PCG {info.pcg_iterations} iterations over {info.pcg_solves} solves, nnz(S) {info.nnz_s}, "
          f"{info.ms:.1f} ms")
    assert info.not_converged == 0
    assert d < 1e-9 * np.max(np.abs(dense))
    p["ctx"].close()


@pytest.mark.parametrize("name", ["dtiny5", "ctiny5"])
def test_columns_with_contracted_d_functions(name):
    # contracted spherical / Cartesian d bases: the route works on the
    # functions (S from the contracted terms); the oracle solves without a
    # preconditioner, which changes nothing beyond the solver tolerance
    p = problem(name, 48, precision=dft.DFT_PREC_FP16X3)
    K = p["K"]
    cols = [0, K // 2, K - 1]
    out, info = p["ctx"].density_matrix_columns(p["F_g"], cols, p["mu"], p["e_min"], p["e_max"], p["n_c"],
                                                pcg_tol=1e-12)
    ref, _ = osp.columns(p["F_o"], p["S_o"], cols, p["a"], p["e_min"], p["e_max"], tol=1e-12, precond="none",
                         maxit=5000)
    assert info.not_converged == 0
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-8 * np.max(np.abs(ref))
    p["ctx"].close()
