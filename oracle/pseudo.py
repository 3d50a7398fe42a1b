"""Non-local Kleinman-Bylander pseudopotential matrix V^NL (oracle).

Test infrastructure only; see the package docstring.

The Fock matrix carries a non-local term, F = T + V^NL + V^KS (Eq. 2.3),
V^NL_ab = h^3 sum_g phi_a(r_g) sum_C v_nl^C phi_b(r_g) (Eq. 2.4), with
v_nl^C in the Kleinman-Bylander form (Section 2, footnote on the
pseudopotentials): a separable operator localised around atom C,
  v_nl^C(r, r') = sum_p e_p chi_p(r) chi_p(r'),
built from projectors chi_p centred on R_C.  Supp. A.2.2 evaluates it on the
grid in two stages: psi_Cb(r_g) = sum_{g' in W_b^C} v_nl^C(r_g, r_g')
phi_b(r_g') h^3 on the atom's window W^C, then V^C_ab = sum_{g in W_a^C}
phi_a(r_g) psi_Cb(r_g) h^3, and V^NL = sum_C V^C (Eq. A.7).

Readings (the paper names the form, not its tables; no norm-conserving
pseudopotential tables exist here):
  * synthetic projectors: per atom one s and (optionally) three Cartesian p
    Gaussians, chi(r) = N (x - X)^i (y - Y)^j (z - Z)^k exp(-zeta_nl |r - R|^2)
    normalised to unit continuum norm like the basis functions, with KB
    energies e_s, e_p;
  * the window of a projector is the cube of Eq. A.4 for its own l and
    zeta_nl (the rule of the basis functions), clipped at the box; W^C is
    the union of the atom's projector windows;
  * with a separable v_nl the two stages reduce to the grid projections
    B_pb = h^3 sum_{g in W_p and W_b} chi_p(r_g) phi_b(r_g) and
    V^NL = B^T diag(e) B; both forms are here, and the tests check that they
    agree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import basis


@dataclass
class KB:
    """Synthetic Kleinman-Bylander projectors: Gaussian exponent (bohr^-2),
    energies (Ha) of the s and p channels, and whether p is present."""
    zeta: float = 1.0
    e_s: float = 1.5
    e_p: float = 0.5
    with_p: bool = True


def projectors(sysm, kb):
    """The projectors as a function set in the layout of basis.functions
    (center, zeta, l, pw, norm, atom) plus their energies e."""
    cen, ls, pw, nrm, atm, e = [], [], [], [], [], []
    base = (2.0 * kb.zeta / math.pi) ** 0.75
    for a, R in enumerate(sysm.xyz):
        comps = [(0, (0, 0, 0))]
        if kb.with_p:
            comps += [(1, (1, 0, 0)), (1, (0, 1, 0)), (1, (0, 0, 1))]
        for l, p in comps:
            cen.append(R)
            ls.append(l)
            pw.append(p)
            nrm.append(base if l == 0 else base * 2.0 * math.sqrt(kb.zeta))
            atm.append(a)
            e.append(kb.e_s if l == 0 else kb.e_p)
    n = len(ls)
    return dict(center=np.array(cen).reshape(n, 3), zeta=np.full(n, kb.zeta), l=np.array(ls, dtype=np.int64),
                pw=np.array(pw, dtype=np.int64).reshape(n, 3), norm=np.array(nrm), atom=np.array(atm, dtype=np.int64),
                e=np.array(e))


def projections(sysm, kb, eta=1e-10, windowed=True):
    """B_pb = h^3 sum_{g in W_p and W_b} chi_p(r_g) phi_b(r_g): the grid
    projection of every basis function on every projector, summed point by
    point over each projector's window box.  Contracted functions: the
    projections of their Cartesian terms, times C^T."""
    fn, C = basis.expansion(sysm)
    pj = projectors(sysm, kb)
    tabs = basis.axis_tables(sysm, fn, eta if windowed else None)
    if windowed:
        plo, phi = basis.window_ranges(sysm, pj, eta)
    else:
        plo = np.zeros((len(pj["l"]), 3), dtype=np.int64)
        phi = np.tile(np.asarray(sysm.grid_n, dtype=np.int64) - 1, (len(pj["l"]), 1))
    nx, ny = int(sysm.grid_n[0]), int(sysm.grid_n[1])
    h3 = sysm.grid_h ** 3
    B = np.zeros((len(pj["l"]), len(fn["zeta"])))
    for p in range(len(pj["l"])):
        if np.any(plo[p] > phi[p]):
            continue
        ix, iy, iz = (np.arange(plo[p][d], phi[p][d] + 1) for d in range(3))
        Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
        flat = (Z * ny + Y) * nx + X
        o, h = sysm.grid_origin, sysm.grid_h
        pts = np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel(), o[2] + h * Z.ravel()], axis=1)
        chi = basis.phi_at({k: pj[k][[p]] for k in ("center", "zeta", "pw", "norm")}, pts)[:, 0]
        ph = grid_phi(sysm, tabs, flat.ravel())
        B[p] = h3 * (chi @ ph)
    return (B if C is None else B @ C.T), pj


def grid_phi(sysm, tabs, flat_idx):
    """phi_b at flat grid indices (x fastest) from the windowed tables."""
    nx, ny = int(sysm.grid_n[0]), int(sysm.grid_n[1])
    ix = flat_idx % nx
    iy = (flat_idx // nx) % ny
    iz = flat_idx // (nx * ny)
    return tabs[0][ix] * tabs[1][iy] * tabs[2][iz]


def vnl(sysm, kb, eta=1e-10, windowed=True):
    """V^NL = B^T diag(e) B (Eq. A.7 for the separable KB operator)."""
    B, pj = projections(sysm, kb, eta, windowed)
    return B.T @ (pj["e"][:, None] * B)


def vnl_two_stage(sysm, kb, eta=1e-10):
    """Supp. A.2.2 as written, for small cases: per atom C the operator
    v_nl^C(r_g, r_g') = sum_p e_p chi_p(r_g) chi_p(r_g') on W^C x W^C (each
    projector restricted to its window), psi_Cb = v_nl^C phi_b h^3 on W^C,
    V^C_ab = phi_a . psi_Cb h^3, and V^NL = sum_C V^C."""
    if basis.is_contracted(sysm):
        raise NotImplementedError("written for one-primitive functions")
    fn = basis.functions(sysm)
    pj = projectors(sysm, kb)
    tabs = basis.axis_tables(sysm, fn, eta)
    plo, phi = basis.window_ranges(sysm, pj, eta)
    nx, ny = int(sysm.grid_n[0]), int(sysm.grid_n[1])
    o, h = sysm.grid_origin, sysm.grid_h
    h3 = h ** 3
    K = len(fn["zeta"])
    V = np.zeros((K, K))
    for C in range(sysm.n_atoms):
        ps = np.nonzero(pj["atom"] == C)[0]
        lo = plo[ps].min(axis=0)
        hi = phi[ps].max(axis=0)
        if np.any(lo > hi):
            continue
        ix, iy, iz = (np.arange(lo[d], hi[d] + 1) for d in range(3))
        Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
        Xr, Yr, Zr = X.ravel(), Y.ravel(), Z.ravel()
        pts = np.stack([o[0] + h * Xr, o[1] + h * Yr, o[2] + h * Zr], axis=1)
        vop = np.zeros((len(pts), len(pts)))
        for p in ps:
            inside = ((Xr >= plo[p][0]) & (Xr <= phi[p][0]) & (Yr >= plo[p][1]) & (Yr <= phi[p][1])
                      & (Zr >= plo[p][2]) & (Zr <= phi[p][2]))
            chi = basis.phi_at({k: pj[k][[p]] for k in ("center", "zeta", "pw", "norm")}, pts)[:, 0] * inside
            vop += pj["e"][p] * np.outer(chi, chi)
        ph = grid_phi(sysm, tabs, (Zr * ny + Yr) * nx + Xr)      # phi_b on W^C, zero outside W_b
        psi = vop @ ph * h3                                       # psi_Cb(r_g), g in W^C
        V += ph.T @ psi * h3
    return V


def projections_closed_form(sysm, kb):
    """<chi_p | phi_b> in the continuum (no grid, no windows), from the
    closed-form overlaps of Cartesian Gaussians: the h -> 0 limit of B."""
    if basis.is_contracted(sysm):
        raise NotImplementedError("written for one-primitive functions")
    fn = basis.functions(sysm)
    pj = projectors(sysm, kb)
    both = {k: np.concatenate([pj[k], fn[k]]) for k in ("center", "zeta", "pw", "norm", "l")}
    npj = len(pj["l"])
    S, _ = basis.overlap_kinetic(both, rows=np.arange(npj))
    return S[:, npj:]
