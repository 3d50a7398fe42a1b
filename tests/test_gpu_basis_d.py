"""Contracted spherical Gaussians up to d (Eqs. A.1-A.3, Table A.1) on the
GPU against the FP64 oracle.

The library expands every basis function into Cartesian Gaussian terms
(contraction coefficient times solid-harmonic weight), runs the closed-form
integrals, quadrature and collocation on the terms and contracts the
results (with the functions' normalisation from the overlap).  The oracle
does the same algebra with its own code (basis.expansion) and is pinned
against fine-grid sums, the solid harmonics' orthonormality and closed-form
kinetic values.  FP64 on both sides: roundoff gates.
"""
import numpy as np
import pytest

import workloads as w
from oracle import basis, dm, grid_ops, pseudo, scf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", ["dtiny5", "ctiny5"])
def test_overlap_kinetic_contracted(name):
    s = w.config_system(name)
    S_o, T_o = basis.overlap_kinetic_system(s)
    ctx = dft.Context(s)
    assert ctx.K == s.n_basis
    S, T = ctx.overlap_kinetic()
    print(f"{name}: K {ctx.K}, max|dS| {np.max(np.abs(host(S) - S_o)):.2e}, max|dT| {np.max(np.abs(host(T) - T_o)):.2e}")
    assert np.max(np.abs(host(S) - S_o)) < 1e-13
    assert np.max(np.abs(host(T) - T_o)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("name", ["dtiny5", "ctiny5"])
def test_grid_transforms_contracted(name):
    s = w.config_system(name)
    rng = np.random.default_rng(11)
    shp = tuple(int(t) for t in s.grid_n[::-1])
    v = scf.vloc(s) + 0.1 * rng.normal(size=shp)
    ctx = dft.Context(s)
    V = host(ctx.potential_matrix(dev(v)))
    V_o = grid_ops.potential_matrix(s, v)
    assert np.max(np.abs(V - V_o)) < 1e-12 * max(1.0, np.max(np.abs(V_o)))
    K = s.n_basis
    A = rng.normal(size=(K, K)) * 0.02
    P = A + A.T
    n = host(ctx.density_on_grid(dev(P)))
    n_o = grid_ops.density_on_grid(s, P)
    assert np.max(np.abs(n - n_o)) < 1e-12 * max(1.0, np.max(np.abs(n_o)))
    ctx.close()


def test_scf_step_contracted_d():
    """One FP64 SCF cycle with the contracted d basis against the oracle's
    exact-DM cycle (neutral model, V^NL and PW92 on)."""
    s = w.config_system("dtiny8")
    kb = pseudo.KB(zeta=1.0, e_s=1.5, e_p=0.5)
    st = scf.setup(s, scf.Model(neutral=True, nl=kb, pw92=True))
    ctx = dft.Context(s, cheb_tail_tol=1e-11, mix_alpha=0.3, model=dft.DFT_MODEL_NEUTRAL, xc=dft.DFT_XC_PW92,
                      nl_channels=4, nl_zeta=kb.zeta, nl_e_s=kb.e_s, nl_e_p=kb.e_p)
    ctx.overlap_kinetic()
    assert np.max(np.abs(host(ctx.nonlocal_matrix()) - st.extras["vnl"])) < 1e-13
    n = ctx.initial_density()
    P = ctx.matrix()
    info = ctx.scf_step(n, P_out=P)
    r = scf.step(st, scf.ion_density(s))
    print(f"dtiny8 step: E/atom {info.e_total / s.n_atoms:.10f} vs {r['E']['total'] / s.n_atoms:.10f}")
    assert abs(info.e_total - r["E"]["total"]) / s.n_atoms < 1e-7
    assert np.max(np.abs(host(P) - r["P"])) < 1e-7
    ctx.close()


def test_mixed_density_matrix_contracted_d():
    s = w.config_system("dtiny8")
    st = scf.setup(s, scf.Model(neutral=True))
    F = scf.fock(st, scf.potential(st, scf.ion_density(s))[0])
    ex = dm.dm_exact(F, st.S, s.n_electrons, 1.0 / s.kT)
    ctx = dft.Context(s, precision=dft.DFT_PREC_FP16X3, model=dft.DFT_MODEL_NEUTRAL, cheb_tail_tol=1e-6)
    ctx.overlap_kinetic()
    P, info = ctx.density_matrix(dev(F))
    dP = host(P) - ex["P"]
    e_kin = abs(2 * np.sum(dP * st.T)) / s.n_atoms
    e_band = abs(2 * np.sum(dP * F)) / s.n_atoms
    print(f"dtiny8 fp16x3: max|dP| {np.max(np.abs(dP)):.3e} dEkin/atom {e_kin:.3e} dEband/atom {e_band:.3e}")
    assert np.max(np.abs(dP)) < 1e-4 and e_kin < 1e-5 and e_band < 1e-5
    ctx.close()
