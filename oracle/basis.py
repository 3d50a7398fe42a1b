"""Basis functions, windows and closed-form one-electron integrals (oracle).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


# Table A.1: the real solid harmonics of degree l <= 2 as weights of the
# Cartesian monomials x^i y^j z^k (i + j + k = l), in the table's order of m;
# p keeps the Cartesian order x, y, z (all its weights are 1)
SOLID = {
    0: [[((0, 0, 0), 1.0)]],
    1: [[((1, 0, 0), 1.0)], [((0, 1, 0), 1.0)], [((0, 0, 1), 1.0)]],
    2: [[((2, 0, 0), math.sqrt(3.0) / 2.0), ((0, 2, 0), -math.sqrt(3.0) / 2.0)],   # m = 2
        [((1, 1, 0), math.sqrt(3.0))],                                             # m = 1
        [((2, 0, 0), -0.5), ((0, 2, 0), -0.5), ((0, 0, 2), 1.0)],                  # m = 0
        [((0, 1, 1), math.sqrt(3.0))],                                             # m = -1
        [((1, 0, 1), math.sqrt(3.0))]],                                            # m = -2
}
CART_D = [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def monomial_norm(zeta, l):
    """Normalisation of x^l exp(-zeta r^2): (2 zeta/pi)^(3/4) (4 zeta)^(l/2) / sqrt((2l-1)!!)."""
    dfact = {0: 1.0, 1: 1.0, 2: 3.0}[l]
    return (2.0 * zeta / math.pi) ** 0.75 * (4.0 * zeta) ** (0.5 * l) / math.sqrt(dfact)


def is_contracted(sysm):
    return getattr(sysm, "shell_nprim", None) is not None or bool(np.any(np.asarray(sysm.shell_l) > 1))


def expansion(sysm):
    """Basis functions as sums of Cartesian Gaussian terms (Eqs. A.1-A.3):
    phi_a = N_a sum_{t in a} c_t x^i y^j z^k exp(-zeta_t |r - R|^2), with
    c_t = d_p w^{ijk}_{lm} (contraction coefficient times Table A.1 weight)
    times the monomial's normalisation, and N_a making phi_a of unit norm.
    Returns (terms, C): terms in the layout of functions() (norm = c_t) plus,
    for the window of each term, its function's most diffuse exponent
    ('wzeta') and l ('wl') (Supp. A.1.1); C (K x Kt) with C[a, t] = N_a for
    t in a.  For uncontracted s/p shells C is None and terms are functions()."""
    if not is_contracted(sysm):
        return functions(sysm), None
    nprim = getattr(sysm, "shell_nprim", None)
    off = 0
    cen, zet, ls, pw, nrm, atm, wz, wl, par = [], [], [], [], [], [], [], [], []
    K = 0
    for s in range(len(sysm.shell_l)):
        a = int(sysm.shell_atom[s])
        l = int(sysm.shell_l[s])
        if nprim is None:
            prims = [(float(sysm.shell_exp[s]), 1.0)]
        else:
            n = int(nprim[s])
            prims = list(zip(sysm.prim_exp[off:off + n], sysm.prim_coef[off:off + n]))
            off += n
        zmin = min(z for z, _ in prims)
        comps = SOLID[l] if (l < 2 or sysm.spherical) else [[(c, 1.0)] for c in CART_D]
        for comp in comps:
            for z, d in prims:
                for ijk, wgt in comp:
                    cen.append(sysm.xyz[a])
                    zet.append(z)
                    ls.append(l)
                    pw.append(ijk)
                    nrm.append(d * wgt * monomial_norm(z, l))
                    atm.append(a)
                    wz.append(zmin)
                    wl.append(l)
                    par.append(K)
            K += 1
    terms = dict(center=np.array(cen), zeta=np.array(zet), l=np.array(ls, dtype=np.int64),
                 pw=np.array(pw, dtype=np.int64), norm=np.array(nrm), atom=np.array(atm, dtype=np.int64),
                 wzeta=np.array(wz), wl=np.array(wl, dtype=np.int64), parent=np.array(par, dtype=np.int64))
    M = np.zeros((K, len(par)))
    M[terms["parent"], np.arange(len(par))] = 1.0
    S_t, _ = overlap_kinetic(terms)
    Nrm = 1.0 / np.sqrt(np.einsum("at,ts,as->a", M, S_t, M))
    return terms, Nrm[:, None] * M


def contract(C, A):
    """C A C^T for a term-level matrix A (A itself when C is None)."""
    return A if C is None else C @ A @ C.T


def overlap_kinetic_system(sysm):
    """S and T of the system's basis functions (contracted when it has
    contracted or d shells)."""
    terms, C = expansion(sysm)
    S, T = overlap_kinetic(terms)
    return contract(C, S), contract(C, T)


def functions(sysm):
    """Expand shells into basis functions (Eqs. A.1-A.3 with one primitive).

    Returns a dict of arrays over the K functions:
      center (K,3), zeta (K,), l (K,), pw (K,3) Cartesian powers (i,j,k),
      norm (K,), atom (K,).
    p shells expand in the order x, y, z (Table A.1 lists m = 1, 0, -1 as x, z,
    y; all weights are 1, so only the labels' order differs).
    Normalisation: each primitive has unit self-overlap,
      s: (2 zeta/pi)^(3/4),  p: (2 zeta/pi)^(3/4) * 2 sqrt(zeta).
    """
    cen, zet, ls, pw, nrm, atm = [], [], [], [], [], []
    for s in range(len(sysm.shell_l)):
        a = int(sysm.shell_atom[s])
        l = int(sysm.shell_l[s])
        z = float(sysm.shell_exp[s])
        comps = [(0, 0, 0)] if l == 0 else [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
        for c in comps:
            cen.append(sysm.xyz[a])
            zet.append(z)
            ls.append(l)
            pw.append(c)
            base = (2.0 * z / math.pi) ** 0.75
            nrm.append(base if l == 0 else base * 2.0 * math.sqrt(z))
            atm.append(a)
    return dict(center=np.array(cen), zeta=np.array(zet), l=np.array(ls, dtype=np.int64),
                pw=np.array(pw, dtype=np.int64), norm=np.array(nrm), atom=np.array(atm, dtype=np.int64))


def window_halfwidth(zeta, l, eta):
    """Window half-length L solving c(L sqrt(zeta), l) = 1 - eta (Eq. A.4).

    c(d, l) = int_0^d x^l e^{-x^2} dx / int_0^inf x^l e^{-x^2} dx is the
    regularised lower incomplete gamma function P((l+1)/2, d^2), so
    d^2 = Q^{-1}((l+1)/2, eta) with Q the upper one.
    """
    zeta = np.asarray(zeta, dtype=np.float64)
    l = np.asarray(l)
    d2 = special.gammainccinv((l + 1) / 2.0, eta)
    return np.sqrt(d2) / np.sqrt(zeta)


def _window_params(fn):
    """(zeta, l) that set the window: the function's own, or for the terms of
    a contracted function those of the function (its most diffuse primitive)."""
    if "wzeta" in fn:
        return fn["wzeta"], fn["wl"]
    return fn["zeta"], fn["l"]


def window_ranges(sysm, fn, eta):
    """Grid-index range [lo, hi] per function and axis of the cubic window
    W_alpha (Supp. A.1.1): points with |x_g - R_x| <= L on every axis,
    clipped to the box.  Returns (lo, hi) int arrays of shape (K, 3); an empty
    range has lo > hi.
    """
    L = window_halfwidth(*_window_params(fn), eta)
    o = sysm.grid_origin
    h = sysm.grid_h
    n = sysm.grid_n
    lo = np.ceil((fn["center"] - L[:, None] - o[None, :]) / h).astype(np.int64)
    hi = np.floor((fn["center"] + L[:, None] - o[None, :]) / h).astype(np.int64)
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, n[None, :] - 1)
    return lo, hi


def axis_tables(sysm, fn, eta=None):
    """Separable factors of every function along each axis (Supp. A.1).

    tab[d] has shape (n_d, K): (x_g - R)^i exp(-zeta (x_g - R)^2), zero
    outside the window range when eta is given; the normalisation is folded
    into the x table.  phi_alpha(r_g) = tab[0][ix, a] * tab[1][iy, a] * tab[2][iz, a].
    """
    tabs = []
    if eta is not None:
        lo, hi = window_ranges(sysm, fn, eta)
    for d in range(3):
        nd = int(sysm.grid_n[d])
        x = sysm.grid_origin[d] + sysm.grid_h * np.arange(nd)
        dx = x[:, None] - fn["center"][None, :, d]
        t = dx ** fn["pw"][None, :, d] * np.exp(-fn["zeta"][None, :] * dx * dx)
        if d == 0:
            t = t * fn["norm"][None, :]
        if eta is not None:
            idx = np.arange(nd)[:, None]
            t = np.where((idx >= lo[None, :, d]) & (idx <= hi[None, :, d]), t, 0.0)
        tabs.append(t)
    return tabs


def phi_at(fn, pts):
    """Direct (non-separable, unwindowed) evaluation of every function at
    arbitrary points, Eq. A.3: N (x-X)^i (y-Y)^j (z-Z)^k exp(-zeta |r-R|^2).
    pts (P,3) -> (P,K)."""
    d = pts[:, None, :] - fn["center"][None, :, :]
    r2 = (d * d).sum(-1)
    poly = np.prod(d ** fn["pw"][None, :, :], axis=-1)
    return fn["norm"][None, :] * poly * np.exp(-fn["zeta"][None, :] * r2)


def _os_1d(a, b, A, B, imax, jmax):
    """1D Obara-Saika overlap table S[i][j] for x^i-type primitives about A
    and B with exponents a, b (vectorised over pairs).  Textbook recursion:
      S_00 = sqrt(pi/p) exp(-mu (A-B)^2),
      S_{i+1,j} = X_PA S_ij + (i S_{i-1,j} + j S_{i,j-1}) / 2p,
      S_{i,j+1} = X_PB S_ij + (i S_{i-1,j} + j S_{i,j-1}) / 2p.
    """
    p = a + b
    mu = a * b / p
    P = (a * A + b * B) / p
    xpa = P - A
    xpb = P - B
    S = [[None] * (jmax + 1) for _ in range(imax + 1)]
    S[0][0] = np.sqrt(np.pi / p) * np.exp(-mu * (A - B) ** 2)
    zero = np.zeros_like(S[0][0])

    def g(i, j):
        return zero if (i < 0 or j < 0) else S[i][j]
    for i in range(imax + 1):
        for j in range(jmax + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                S[i][j] = xpa * g(i - 1, j) + ((i - 1) * g(i - 2, j) + j * g(i - 1, j - 1)) / (2 * p)
            else:
                S[i][j] = xpb * g(i, j - 1) + (i * g(i - 1, j - 1) + (j - 1) * g(i, j - 2)) / (2 * p)
    return S


def overlap_kinetic(fn, rows=None):
    """Closed-form overlap S and kinetic T = <-1/2 nabla^2> for normalised
    Cartesian primitives (the continuum limits of Eqs. 2.1 and 2.2; by parts
    1/2 int grad.grad equals <-1/2 lap> for decaying functions).

    1D kinetic: T_ij = -2 b^2 S_{i,j+2} + b (2j+1) S_ij - j(j-1)/2 S_{i,j-2};
    3D: T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz.  rows: optional index array of
    the rows to compute (for sampled checks on large systems).
    """
    K = len(fn["zeta"])
    ri = np.arange(K) if rows is None else np.asarray(rows)
    a = fn["zeta"][ri][:, None]
    b = fn["zeta"][None, :]
    S = np.ones((len(ri), K))
    Sd, Td = [], []
    for d in range(3):
        A = fn["center"][ri, d][:, None]
        B = fn["center"][None, :, d]
        tab = _os_1d(a, b, A, B, 2, 4)
        i = fn["pw"][ri, d][:, None] + np.zeros((1, K), dtype=np.int64)
        j = fn["pw"][None, :, d] + np.zeros((len(ri), 1), dtype=np.int64)
        s_d = np.zeros((len(ri), K))
        t_d = np.zeros((len(ri), K))
        for ii in range(3):
            for jj in range(3):
                m = (i == ii) & (j == jj)
                s_ij = tab[ii][jj]
                t_ij = -2.0 * b * b * tab[ii][jj + 2] + b * (2 * jj + 1) * tab[ii][jj]
                if jj >= 2:
                    t_ij = t_ij - 0.5 * jj * (jj - 1) * tab[ii][jj - 2]
                s_d = np.where(m, np.broadcast_to(s_ij, m.shape), s_d)
                t_d = np.where(m, np.broadcast_to(t_ij, m.shape), t_d)
        Sd.append(s_d)
        Td.append(t_d)
    nn = fn["norm"][ri][:, None] * fn["norm"][None, :]
    S = nn * Sd[0] * Sd[1] * Sd[2]
    T = nn * (Td[0] * Sd[1] * Sd[2] + Sd[0] * Td[1] * Sd[2] + Sd[0] * Sd[1] * Td[2])
    return S, T
