"""The paper's parallel scheme for the density matrix, on CPU ranks.

Supplement B applies the Chebyshev recurrence to the columns of S^-1
independently: U_0 = S^-1 u_a, U_{l+1} = 2 H_N U_l - U_{l-1} with H = S^-1 F,
P u_a = sum_l a_l U_l.  So the columns shard over ranks with the Hamiltonian
replicated; the only exchanges are one reduction of the N_C partial moments
m_l = Tr[T_l(H_N)] = Tr[U_l S] (each rank sums the diagonal of S U_l over its
own columns) before mu is fixed by the electron count (Eq. 2.8), and the
gather of the column panels at the end.  The symmetric form that the
single-GPU path runs (X_0 = I, F~ = L^-1 F L^-T) shards the same way but
needs one more exchange, a sum of K x K contributions, because
P = L^-T rho L^-1 mixes every column of rho.  Every run here has one GPU, so
both decompositions are exercised on gloo ranks in host memory; the result
must equal the unsharded Chebyshev density matrix of the oracle.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import dm  # noqa: E402


def _problem(K=48, seed=3):
    """A small symmetric-definite pair (F, S) with a spread spectrum."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(K, K))
    S = A @ A.T / K + np.eye(K)
    B = rng.normal(size=(K, K))
    F = 0.5 * (B + B.T)
    eps = dm.geneig(F, S)[0]
    lo, hi = eps[0] - 0.1, eps[-1] + 0.1
    return F, S, lo, hi


def _panel(K, rank, world):
    return (K * rank) // world, (K * (rank + 1)) // world


def _rank_main(rank, world, port, n_e, beta, n_c, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        F, S, lo, hi = _problem()
        K = F.shape[0]
        c0, c1 = _panel(K, rank, world)
        eb, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
        HN = (np.linalg.solve(S, F) - eb * np.eye(K)) / de        # replicated
        U0 = np.linalg.inv(S)[:, c0:c1]                            # this rank's columns of S^-1

        def passes(a=None):
            """Moments (a is None) or the weighted sum over this rank's columns."""
            u0, u1 = U0, HN @ U0
            mom = np.zeros(n_c)
            acc = None
            for l in range(n_c):
                ul = u0 if l == 0 else u1
                if l >= 2:
                    u2 = 2.0 * HN @ u1 - u0
                    u0, u1 = u1, u2
                    ul = u2
                if a is None:
                    mom[l] = float(np.sum(S[c0:c1, :] * ul.T))    # sum_j in panel (S U_l)_jj
                else:
                    acc = a[l] * ul if acc is None else acc + a[l] * ul
            return mom if a is None else acc

        part = torch.from_numpy(passes())
        dist.all_reduce(part, op=dist.ReduceOp.SUM)                # the one reduction
        mom = part.numpy()
        span = 40.0 / beta
        mu = dm.bisect(lambda m: dm.electron_count(m, beta, lo, hi, mom), n_e, lo - span, hi + span)
        a = dm.cheb_coeffs(mu, beta, lo, hi, n_c)
        panel = torch.from_numpy(np.ascontiguousarray(passes(a)))
        # gather the column panels (uneven widths allowed): each rank broadcasts its own
        gathered = []
        for r in range(world):
            a0, a1 = _panel(K, r, world)
            buf = panel.clone() if r == rank else torch.zeros(K, a1 - a0, dtype=torch.float64)
            dist.broadcast(buf, src=r)
            gathered.append(buf)
        P = torch.cat(gathered, dim=1).numpy()
        q.put((rank, mu, P))
    finally:
        dist.destroy_process_group()


def _rank_main_symmetric(rank, world, port, n_e, beta, n_c, q):
    """The symmetric form (F~ = L^-1 F L^-T, X_0 = I): panels of X_l and rho
    are independent as well, but P = L^-T rho L^-1 mixes every column of rho,
    so the last step is one sum-reduction of the K x K contributions
    L^-T rho[:, panel] L^-1[panel, :]."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        F, S, lo, hi = _problem()
        K = F.shape[0]
        c0, c1 = _panel(K, rank, world)
        eb, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
        Li = np.linalg.inv(np.linalg.cholesky(S))
        HN = (Li @ F @ Li.T - eb * np.eye(K)) / de                 # replicated
        X0 = np.eye(K)[:, c0:c1]                                    # this rank's columns of I

        def passes(a=None):
            u0, u1 = X0, HN @ X0
            mom = np.zeros(n_c)
            acc = None
            for l in range(n_c):
                ul = u0 if l == 0 else u1
                if l >= 2:
                    u2 = 2.0 * HN @ u1 - u0
                    u0, u1 = u1, u2
                    ul = u2
                if a is None:
                    mom[l] = float(np.trace(ul[c0:c1, :]))          # diagonal entries in this panel
                else:
                    acc = a[l] * ul if acc is None else acc + a[l] * ul
            return mom if a is None else acc

        part = torch.from_numpy(passes())
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        mom = part.numpy()
        span = 40.0 / beta
        mu = dm.bisect(lambda m: dm.electron_count(m, beta, lo, hi, mom), n_e, lo - span, hi + span)
        a = dm.cheb_coeffs(mu, beta, lo, hi, n_c)
        rho_panel = passes(a)
        contrib = torch.from_numpy(np.ascontiguousarray(Li.T @ rho_panel @ Li[c0:c1, :]))
        dist.all_reduce(contrib, op=dist.ReduceOp.SUM)               # the exchange of K^2 numbers
        q.put((rank, mu, contrib.numpy()))
    finally:
        dist.destroy_process_group()


def _run(target, world, monkeypatch):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(var, "1")                 # one BLAS thread per rank process
    F, S, lo, hi = _problem()
    n_e, beta = 20.0, 8.0
    n_c = dm.cheb_order(0.5 * (lo + hi), beta, lo, hi, 1e-12)
    ref = dm.dm_cheb(F, S, n_e, beta, lo, hi, n_c)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=target, args=(r, world, port, n_e, beta, n_c, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    return S, n_e, ref, res


@pytest.mark.parametrize("world", [2, 3])
def test_symmetric_form_shards_with_one_exchange(world, monkeypatch):
    S, n_e, ref, res = _run(_rank_main_symmetric, world, monkeypatch)
    for rank, mu, P in res:
        assert abs(mu - ref["mu"]) < 1e-10
        assert np.max(np.abs(P - ref["P"])) < 1e-10 * max(1.0, np.max(np.abs(ref["P"])))
        assert abs(2.0 * np.trace(P @ S) - n_e) < 1e-8


@pytest.mark.parametrize("world", [2, 3, 5])
def test_column_shards_reproduce_the_unsharded_density_matrix(world, monkeypatch):
    S, n_e, ref, res = _run(_rank_main, world, monkeypatch)
    for rank, mu, P in res:
        assert abs(mu - ref["mu"]) < 1e-10
        assert np.max(np.abs(P - ref["P"])) < 1e-10 * max(1.0, np.max(np.abs(ref["P"])))
        assert abs(2.0 * np.trace(P @ S) - n_e) < 1e-8
