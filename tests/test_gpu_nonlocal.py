"""Non-local Kleinman-Bylander pseudopotential V^NL (Eqs. 2.3-2.4, Supp.
A.2.2) and PW92 LDA correlation (Section 4) on the GPU against the FP64
oracle.

The projectors are synthetic (no norm-conserving tables exist here): per
atom one s and three p Gaussians of exponent 1 bohr^-2 with KB energies
1.5 and 0.5 Ha.  V^NL is FP64 on both sides (projections as grid sums over
the windows' intersection, then B^T diag(e) B), so the gate is roundoff;
the SCF step with both terms is held to the FP64 step's gates, and the
converged mixed-precision SCF with both terms to 1e-5 Ha/atom of the
oracle's converged energy (tests/golden/scf_tiny8_nlpw92.json).
"""
import json
import os

import numpy as np
import pytest

import workloads as w
from oracle import pseudo, scf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402

KB = pseudo.KB(zeta=1.0, e_s=1.5, e_p=0.5)
NL = dict(nl_channels=4, nl_zeta=KB.zeta, nl_e_s=KB.e_s, nl_e_p=KB.e_p)
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name,channels", [("tiny8", 4), ("tiny37", 4), ("tiny8", 1)])
def test_nonlocal_matrix_matches_oracle(name, channels):
    s = w.config_system(name)
    kb = pseudo.KB(zeta=KB.zeta, e_s=KB.e_s, e_p=KB.e_p, with_p=channels == 4)
    ref = pseudo.vnl(s, kb)
    ctx = dft.Context(s, **{**NL, "nl_channels": channels})
    ctx.overlap_kinetic()
    V = host(ctx.nonlocal_matrix())
    err = np.max(np.abs(V - ref))
    print(f"{name} V^NL ({channels} projectors per atom): max|dV| {err:.3e} of max {np.max(np.abs(ref)):.3e}")
    assert err < 1e-13 * max(1.0, np.max(np.abs(ref)))
    ctx.close()
    # without projectors the matrix is zero
    c0 = dft.Context(s)
    c0.overlap_kinetic()
    assert float(c0.nonlocal_matrix().abs().max()) == 0.0
    c0.close()


@pytest.mark.parametrize("neutral", [False, True])
def test_hartree_xc_with_pw92(neutral):
    s = w.config_system("tiny8")
    st = scf.setup(s, scf.Model(neutral=neutral, pw92=True))
    n0 = scf.ion_density(s) * 1.3
    v_ref, vh, ex = scf.potential(st, n0)
    ctx = dft.Context(s, model=dft.DFT_MODEL_NEUTRAL if neutral else dft.DFT_MODEL_LITERAL, xc=dft.DFT_XC_PW92)
    v, e = ctx.hartree_xc(dev(n0))
    assert np.max(np.abs(host(v) - v_ref)) < 1e-11 * np.max(np.abs(v_ref))
    h3 = s.grid_h ** 3
    rho = n0 - st.nion
    e_ref = (h3 * np.sum(st.vloc * n0), 0.5 * h3 * np.sum(vh * rho), h3 * np.sum(ex * n0))
    assert np.allclose(e, e_ref, rtol=1e-11, atol=1e-11)
    ctx.close()


def test_scf_step_with_nonlocal_and_pw92():
    """One FP64 SCF cycle with V^NL in the Fock matrix and PW92 in v_xc,
    against the oracle's exact-DM cycle: energies (with the non-local term
    2 Tr[P V^NL] reported apart), potential, density matrix and next density."""
    s = w.config_system("tiny8")
    st = scf.setup(s, scf.Model(nl=KB, pw92=True))
    ctx = dft.Context(s, cheb_tail_tol=1e-11, mix_alpha=0.3, xc=dft.DFT_XC_PW92, **NL)
    ctx.overlap_kinetic()
    n = ctx.initial_density()
    P = ctx.matrix()
    v = ctx.grid_array()
    info = ctx.scf_step(n, v_ks_out=v, P_out=P)
    n0 = scf.ion_density(s)
    r = scf.step(st, n0)
    print(f"tiny8 V^NL + PW92 step: E/atom {info.e_total / s.n_atoms:.10f} vs {r['E']['total'] / s.n_atoms:.10f}, "
          f"E_nl {info.e_nl:.8f} vs {r['E']['nl']:.8f}")
    assert abs(info.e_total - r["E"]["total"]) / s.n_atoms < 1e-7
    assert abs(info.e_nl - r["E"]["nl"]) < 1e-6 and abs(r["E"]["nl"]) > 1e-3
    assert abs(info.e_xc - r["E"]["xc"]) < 1e-9
    assert np.max(np.abs(host(v) - r["v"])) < 1e-10
    assert np.max(np.abs(host(P) - r["P"])) < 1e-7
    nxt = scf.linear_mix(0.3)(n0, r["n_out"])
    assert np.max(np.abs(host(n) - nxt)) < 1e-7
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_converged_scf_with_nonlocal_and_pw92(prec):
    p = os.path.join(GOLD, "scf_tiny8_nlpw92.json")
    if not os.path.exists(p):
        pytest.skip("no oracle golden energy")
    g = json.load(open(p))
    assert g["converged"]
    s = w.config_system("tiny8")
    ctx = dft.Context(s, precision=dft.DFT_PREC_FP64 if prec == "fp64" else dft.DFT_PREC_FP16X3,
                      model=dft.DFT_MODEL_NEUTRAL, mixer=dft.DFT_MIX_PULAY, mix_alpha=0.3, kerker_q0=0.8,
                      mix_history=8, cheb_tail_tol=1e-10 if prec == "fp64" else 1e-6, xc=dft.DFT_XC_PW92, **NL)
    ctx.overlap_kinetic()
    n = ctx.initial_density()
    stop = 1e-8 if prec == "fp64" else 1e-7
    converged = False
    for it in range(100):
        info = ctx.scf_step(n)
        if it > 0 and abs(info.de_per_atom) < stop and info.residual < 1e-5:
            converged = True
            break
    e = info.e_total / s.n_atoms
    print(f"tiny8 V^NL + PW92 {prec}: {it + 1} cycles, E/atom {e:.10f} vs oracle {g['E_per_atom']:.10f}, "
          f"|dE| {abs(e - g['E_per_atom']):.2e}")
    assert converged
    assert abs(e - g["E_per_atom"]) < (1e-7 if prec == "fp64" else 1e-5)
    ctx.close()
