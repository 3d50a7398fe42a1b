"""Converged SCF energies of the GPU paths against the FP64 oracle.

The oracle's converged energies are stored in tests/golden/scf_<name>.json by
tests/golden/make_scf_golden.py (oracle only).  Both GPU precisions run the
same model (charge-neutral), start (superposition of atoms) and mixer
(Pulay + Kerker) until the energy change between cycles is below what their
arithmetic resolves -- |dE|/atom < 1e-8 for FP64; 1e-7 for split FP16, whose
products carry about 22 bits, so cycle-to-cycle energies scatter by ~1e-7
Ha/atom -- and max|n_out - n_in| < 1e-5; the gate is the method's target,
1e-5 Ha/atom against the oracle.
"""
import json
import os

import pytest

import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    p = os.path.join(GOLD, f"scf_{name}.json")
    if not os.path.exists(p):
        pytest.skip(f"no oracle golden energy for {name}")
    g = json.load(open(p))
    assert g["converged"]
    return g


@pytest.mark.parametrize("name,prec,tail,reuse", [
    ("tiny8", "fp64", 1e-10, 0), ("tiny8", "fp16x3", 1e-10, 0), ("cluster64", "fp16x3", 1e-10, 0),
    ("cluster64", "fp64", 1e-10, 0), ("tiny8", "fp16x3", 1e-6, 0), ("cluster64", "fp16x3", 1e-6, 0),
    ("tiny8", "fp16x3", 1e-6, 1), ("tiny37", "fp16x3", 1e-6, 1), ("cluster64", "fp16x3", 1e-6, 1)])
def test_converged_energy(name, prec, tail, reuse):
    """tail 1e-6 is the mixed path's Chebyshev order in the benchmark: its
    truncation error (~1e-10 Ha/atom on the host) is far below the gate.
    reuse 1: the moments pass is skipped on the cycles where mu has settled
    (the benchmark's setting); some cycles must skip it, and the converged
    energy keeps the gate."""
    g = golden(name)
    s = w.config_system(name)
    p = dft.DFT_PREC_FP64 if prec == "fp64" else dft.DFT_PREC_FP16X3
    ctx = dft.Context(s, precision=p, model=dft.DFT_MODEL_NEUTRAL, mixer=dft.DFT_MIX_PULAY, mix_alpha=0.3,
                      kerker_q0=0.8, mix_history=8, cheb_tail_tol=tail, reuse_mu=reuse)
    ctx.overlap_kinetic()
    n = ctx.initial_density()
    stop = 1e-8 if prec == "fp64" else 1e-7
    info = None
    converged = False
    reused = 0
    for it in range(100):
        info = ctx.scf_step(n)
        reused += info.mu_reused
        if it > 0 and abs(info.de_per_atom) < stop and info.residual < 1e-5:
            converged = True
            break
    e = info.e_total / s.n_atoms
    print(f"{name} {prec} tail {tail:.0e} (N_C {info.n_cheb}): {it + 1} cycles ({reused} without the moments pass), "
          f"E/atom {e:.10f} vs oracle {g['E_per_atom']:.10f} ({g['iterations']} cycles), "
          f"|dE| {abs(e - g['E_per_atom']):.2e}")
    assert converged, "the stop criterion was not met in 100 cycles"
    if reuse:
        assert reused > 0
    assert abs(e - g["E_per_atom"]) < 1e-5
    ctx.close()
