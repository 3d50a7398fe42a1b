"""Write the oracle's converged SCF energies used by the GPU SCF tests.

Calls only the FP64 oracle (exact Fermi-Dirac density matrix by the
generalised eigensolve) on the seeded workloads, with the charge-neutral
model and Pulay mixing preconditioned by Kerker (alpha 0.3, history 8,
q0 0.8 bohr^-1), until |Delta E|/atom < 1e-8 and max|n_out - n_in| < 1e-5.

    python tests/golden/make_scf_golden.py tiny8 cluster64 tiny37 tiny8_nlpw92
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as w  # noqa: E402
from oracle import pseudo, scf  # noqa: E402

# "<workload>_nlpw92": the same model plus the synthetic Kleinman-Bylander
# projectors (s and p Gaussians, exponent 1, energies 1.5 and 0.5 Ha) and PW92
# correlation
NLPW92 = "_nlpw92"


def main(names):
    for name in names:
        full = name.endswith(NLPW92)
        s = w.config_system(name[:-len(NLPW92)] if full else name)
        model = scf.Model(neutral=True, nl=pseudo.KB(zeta=1.0, e_s=1.5, e_p=0.5) if full else None, pw92=full)
        st = scf.setup(s, model)
        mixer = scf.Pulay(alpha=0.3, hist=8, precond=scf.kerker(s, 0.8))
        t0 = time.time()
        r = scf.run(st, mixer=mixer, max_iter=80, tol_e=1e-8, tol_n=1e-5,
                    log=lambda h: print(name, h["iter"], h["E"] / s.n_atoms, h["dE_per_atom"], h["residual"],
                                        flush=True))
        out = {
            "workload": name, "n_atoms": s.n_atoms, "n_basis": s.n_basis,
            "model": "neutral" + (", KB s+p projectors zeta 1 e 1.5/0.5, PW92 correlation" if full else ""),
            "mixer": "pulay alpha=0.3 hist=8 kerker q0=0.8", "converged": bool(r["converged"]),
            "iterations": len(r["history"]), "E_total": r["E"]["total"], "E_per_atom": r["E"]["total"] / s.n_atoms,
            "E_terms": r["E"], "mu": float(r["mu"]), "seconds": time.time() - t0,
            "source": "oracle.scf.run with the exact density matrix (Eq. 2.9 via the generalised eigensolve)",
        }
        with open(os.path.join(HERE, f"scf_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny8", "cluster64"])
