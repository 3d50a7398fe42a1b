"""Local pseudopotential, initial density, energy and the SCF cycle (oracle).

Test infrastructure only; see the package docstring.

SCF cycle (Supp. A.3, Fig. A.3): from an input density n_in,
  v_KS = v_loc + v_H[n_in] + v_xc[n_in]         (Eq. 2.6; v_xc = Slater
                                                 exchange, plus PW92
                                                 correlation when chosen)
  F    = T + V^NL + V^KS[v_KS]                   (Eqs. 2.3-2.5; V^NL = 0
                                                 unless KB projectors are set)
  P    = f_FD(S^-1 F) S^-1                       (Eq. 2.9)
  n_out(r_g) = 2 sum P phi phi                   (Eq. 2.7)
then the energy of n_out and a mixing step give the next n_in.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import basis, dm, grid_ops, poisson, pseudo


def grid_points(sysm):
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    o, h = sysm.grid_origin, sysm.grid_h
    return (o[0] + h * np.arange(nx), o[1] + h * np.arange(ny), o[2] + h * np.arange(nz))


def gaussian_sum(sysm, amp, width):
    """sum_C amp exp(-|r_g - R_C|^2 / width^2) on the grid, (nz, ny, nx)."""
    xs, ys, zs = grid_points(sysm)
    out = np.zeros((len(zs), len(ys), len(xs)))
    for R in sysm.xyz:
        ex = np.exp(-((xs - R[0]) ** 2) / width ** 2)
        ey = np.exp(-((ys - R[1]) ** 2) / width ** 2)
        ez = np.exp(-((zs - R[2]) ** 2) / width ** 2)
        out += amp * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return out


def vloc(sysm, depth=4.0, width=1.5):
    """v_loc(r_g) = sum_C -depth exp(-|r_g - R_C|^2 / width^2)  (Eq. 2.6, the
    workload's purely local pseudopotential)."""
    return gaussian_sum(sysm, -depth, width)


def ion_density(sysm, charge=4.0, width=1.5):
    """Gaussian ionic charge q (pi w^2)^(-3/2) exp(-r^2/w^2) per atom; used by
    the charge-neutral model and as the superposition-of-atoms start."""
    return gaussian_sum(sysm, charge * (np.pi * width * width) ** -1.5, width)


@dataclass
class Model:
    """Run parameters that define the problem (not the numerics)."""
    eta: float = 1e-10                 # window charge cutoff (Eq. A.4)
    vloc_depth: float = 4.0
    vloc_width: float = 1.5
    neutral: bool = False              # add Gaussian ionic charges to the Poisson source
    ion_charge: float = 4.0
    nl: object = None                  # pseudo.KB projectors of V^NL, or None (V^NL = 0)
    pw92: bool = False                 # add PW92 correlation to the Slater exchange


@dataclass
class Setup:
    sysm: object
    model: Model
    S: np.ndarray
    T: np.ndarray
    vloc: np.ndarray
    nion: np.ndarray
    c0: float
    extras: dict = field(default_factory=dict)


def setup(sysm, model=None):
    model = model or Model()
    S, T = basis.overlap_kinetic_system(sysm)
    vl = vloc(sysm, model.vloc_depth, model.vloc_width)
    ni = ion_density(sysm, model.ion_charge, model.vloc_width) if model.neutral else np.zeros_like(vl)
    st = Setup(sysm=sysm, model=model, S=S, T=T, vloc=vl, nion=ni, c0=poisson.cube_inv_r_constant())
    st.extras["vnl"] = pseudo.vnl(sysm, model.nl, model.eta) if model.nl is not None else None
    return st


def xc(st, n):
    """LDA v_xc and eps_xc: Slater exchange, plus PW92 correlation when the
    model asks for it."""
    vx, ex = poisson.slater_exchange(n)
    if st.model.pw92:
        vc, ec = poisson.pw92_correlation(n)
        vx, ex = vx + vc, ex + ec
    return vx, ex


def potential(st, n):
    """v_KS[n] = v_loc + v_H[n - n_ion] + v_x[n]  (Eq. 2.6)."""
    vh = poisson.hartree(st.sysm, n - st.nion, st.c0)
    vx, ex = xc(st, n)
    return st.vloc + vh + vx, vh, ex


def energy(st, P, n):
    """E = 2 Tr[P T] + 2 Tr[P V^NL] + h^3 sum v_loc n + 1/2 h^3 sum v_H[rho] rho
           + h^3 sum eps_xc(n) n,   rho = n - n_ion.
    (The paper names only the change Delta E between cycles, Supp. C; this
    internal energy is the reading taken.)"""
    h3 = st.sysm.grid_h ** 3
    rho = n - st.nion
    vh = poisson.hartree(st.sysm, rho, st.c0)
    _, ex = xc(st, n)
    e_kin = 2.0 * float(np.sum(P * st.T))
    vnl = st.extras.get("vnl")
    e_nl = 2.0 * float(np.sum(P * vnl)) if vnl is not None else 0.0
    e_loc = h3 * float(np.sum(st.vloc * n))
    e_h = 0.5 * h3 * float(np.sum(vh * rho))
    e_x = h3 * float(np.sum(ex * n))
    return dict(total=e_kin + e_nl + e_loc + e_h + e_x, kin=e_kin, nl=e_nl, loc=e_loc, hartree=e_h, xc=e_x)


def fock(st, v):
    """F = T + V^NL + V^KS[v] (Eq. 2.3)."""
    F = st.T + grid_ops.potential_matrix(st.sysm, v, st.model.eta)
    vnl = st.extras.get("vnl")
    return F if vnl is None else F + vnl


def step(st, n_in, dm_fn=None):
    """One SCF cycle from n_in: returns dict(n_out, P, F, E, mu, ...)."""
    sysm = st.sysm
    beta = 1.0 / sysm.kT
    v, _, _ = potential(st, n_in)
    F = fock(st, v)
    if dm_fn is None:
        r = dm.dm_exact(F, st.S, sysm.n_electrons, beta)
    else:
        r = dm_fn(F, st.S)
    P = r["P"]
    n_out = grid_ops.density_on_grid(sysm, P, st.model.eta)
    E = energy(st, P, n_out)
    return dict(n_out=n_out, P=P, F=F, v=v, E=E, mu=r["mu"], dm=r)


def kerker(sysm, q0):
    """Kerker preconditioner G^2 / (G^2 + q0^2) applied to a grid field by
    FFT over the (periodic) box; damps long-wavelength charge sloshing."""
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    h = sysm.grid_h
    gx = 2 * np.pi * np.fft.rfftfreq(nx, h)
    gy = 2 * np.pi * np.fft.fftfreq(ny, h)
    gz = 2 * np.pi * np.fft.fftfreq(nz, h)
    g2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    w = g2 / (g2 + q0 * q0)

    def apply(r):
        rr = r.reshape(nz, ny, nx)
        return np.fft.irfftn(np.fft.rfftn(rr) * w, s=(nz, ny, nx), axes=(0, 1, 2)).reshape(r.shape)
    return apply


class Pulay:
    """Pulay (DIIS) mixing of densities, the paper's SCF accelerator
    (Section 2): minimise |sum_i c_i R_i| with sum c_i = 1 over the last
    `hist` residuals R_i = n_out_i - n_in_i; next n_in = sum c_i (n_in_i +
    alpha K R_i), with K the identity or a Kerker preconditioner."""

    def __init__(self, alpha=0.3, hist=8, precond=None):
        self.alpha, self.hist = alpha, hist
        self.precond = precond
        self.ins, self.res = [], []

    def __call__(self, n_in, n_out):
        self.ins.append(n_in.ravel().copy())
        self.res.append((n_out - n_in).ravel().copy())
        self.ins, self.res = self.ins[-self.hist:], self.res[-self.hist:]
        m = len(self.res)
        B = np.empty((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                B[i, j] = self.res[i] @ self.res[j]
        B[m, :m] = B[:m, m] = -1.0
        B[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
        x = sum(ci * xi for ci, xi in zip(c, self.ins))
        r = sum(ci * ri for ci, ri in zip(c, self.res))
        if self.precond is not None:
            r = self.precond(r)
        nxt = x + self.alpha * r
        return nxt.reshape(n_in.shape)


def linear_mix(alpha):
    def mix(n_in, n_out):
        return (1.0 - alpha) * n_in + alpha * n_out
    return mix


def run(st, n0=None, mixer=None, max_iter=60, tol_e=1e-7, tol_n=1e-6, dm_fn=None, log=None):
    """SCF iterations until |dE|/N_atoms < tol_e and max|n_out - n_in| < tol_n
    (Supp. C: convergence on Delta E = E^SCF - E^{SCF-1})."""
    sysm = st.sysm
    n_in = ion_density(sysm, st.model.ion_charge, st.model.vloc_width) if n0 is None else n0
    mixer = mixer or Pulay()
    e_prev = None
    hist = []
    for it in range(max_iter):
        r = step(st, n_in, dm_fn)
        e = r["E"]["total"]
        res = float(np.max(np.abs(r["n_out"] - n_in)))
        de = None if e_prev is None else (e - e_prev) / sysm.n_atoms
        hist.append(dict(iter=it, E=e, dE_per_atom=de, residual=res, mu=r["mu"]))
        if log:
            log(hist[-1])
        if de is not None and abs(de) < tol_e and res < tol_n:
            r["history"] = hist
            r["converged"] = True
            return r
        e_prev = e
        n_in = mixer(n_in, r["n_out"])
    r["history"] = hist
    r["converged"] = False
    return r
