"""Write the oracle's exact density-matrix traces for a fixed Fock matrix.

Calls only the FP64 oracle.  For a named workload the Fock matrix is the
one-electron Hamiltonian of the workload without its density-dependent
terms, F = T + V[v_loc]: the closed-form kinetic matrix (continuum limit of
Eq. 2.2) plus the windowed grid quadrature (Eq. 2.5 / A.6) of the bare local
pseudopotential v_loc = sum_A -4 exp(-|r - R_A|^2 / 1.5^2).  Every well is a
product of three one-dimensional factors, so V is summed per atom in the
separable form of the oracle (the factors are cut where they fall below
1e-18, about 9.7 bohr from the atom).  The exact density matrix is then
P = C f(eps) C^T from one generalised eigensolve F C = S C eps (Eq. 2.9),
with mu fixed by 2 sum_i f(eps_i) = N_e (Eq. 2.8).

Stored (JSON, a few hundred bytes): mu, the eigenvalue range, the traces
2 Tr[P T] (kinetic), 2 Tr[P F] (band), 2 Tr[P V], 2 Tr[P S], and fingerprints
of the inputs (Tr F, ||F||_F, Tr S, ||S||_F, Tr T) by which a consumer that
builds F on its own checks that it holds the same matrix.

    python tests/golden/make_dm_golden.py sphere40      # K = 19630: ~1 h, ~35 GB
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as w  # noqa: E402
from oracle import basis, dm, grid_ops, scf  # noqa: E402

CUT = 1e-18
ROWS = 512   # row block of the closed-form S and T (bounds the temporaries)


def well_factors(s):
    """(fx, fy, fz) of -4 exp(-|r - R|^2 / 1.5^2) per atom, each cut below CUT."""
    xs, ys, zs = scf.grid_points(s)

    def well(x, c):
        e = np.exp(-(x - c) ** 2 / 1.5 ** 2)
        return np.where(e > CUT, e, 0.0)
    return [(-4.0 * well(xs, R[0]), well(ys, R[1]), well(zs, R[2])) for R in s.xyz]


def overlap_kinetic_blocked(fn):
    K = len(fn["zeta"])
    S = np.empty((K, K))
    T = np.empty((K, K))
    for r0 in range(0, K, ROWS):
        rows = np.arange(r0, min(K, r0 + ROWS))
        S[rows], T[rows] = basis.overlap_kinetic(fn, rows=rows)
    return S, T


def main(names):
    for name in names:
        s = w.config_system(name)
        t0 = time.time()
        fn = basis.functions(s)
        S, T = overlap_kinetic_blocked(fn)
        print(name, "S, T", time.time() - t0, flush=True)
        V = grid_ops.potential_matrix_separable(s, well_factors(s))
        print(name, "V", time.time() - t0, flush=True)
        fp = {"trace_F": float(np.trace(T) + np.trace(V)), "trace_S": float(np.trace(S)),
              "trace_T": float(np.trace(T)), "frob_S": float(np.linalg.norm(S))}
        F = V
        F += T
        fp["frob_F"] = float(np.linalg.norm(F))
        ex = dm.dm_exact(F, S, s.n_electrons, 1.0 / s.kT)
        print(name, "eigensolve", time.time() - t0, flush=True)
        P = ex["P"]
        e_kin = 2.0 * float(np.vdot(P, T))
        e_band = 2.0 * float(np.vdot(P, F))
        n_e = 2.0 * float(np.vdot(P, S))
        eps, occ = ex["eps"], ex["occ"]
        homo = int(np.searchsorted(eps, ex["mu"]))
        out = {
            "workload": name, "n_atoms": s.n_atoms, "n_basis": s.n_basis, "n_electrons": s.n_electrons,
            "kT": s.kT, "eta": 1e-10, "fock": "T + V[v_loc], v_loc = sum_A -4 exp(-|r-R_A|^2/1.5^2), "
                                             "separable factors cut below 1e-18",
            "mu": float(ex["mu"]), "eps_min": float(eps[0]), "eps_max": float(eps[-1]),
            "eps_below_mu": float(eps[homo - 1]) if homo > 0 else None,
            "eps_above_mu": float(eps[homo]) if homo < len(eps) else None,
            "e_kin": e_kin, "e_band": e_band, "e_band_eigen": 2.0 * float(np.sum(occ * eps)),
            "e_loc": e_band - e_kin, "n_e_trace": n_e, "n_e_occ": 2.0 * float(np.sum(occ)),
            "max_abs_P": float(np.max(np.abs(P))), "fingerprint": fp, "seconds": time.time() - t0,
            "source": "oracle.dm.dm_exact (generalised eigensolve, Eq. 2.9) on oracle.basis closed-form S, T "
                      "and oracle.grid_ops.potential_matrix_separable",
        }
        with open(os.path.join(HERE, f"dm_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["sphere40"])
