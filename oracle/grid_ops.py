"""Grid <-> basis transforms (oracle): quadrature and collocation.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np

from . import basis


def _slabs(sysm, planes):
    nz = int(sysm.grid_n[2])
    for z0 in range(0, nz, planes):
        yield z0, min(nz, z0 + planes)


def _phi_slab(tabs, z0, z1, sel=None):
    """Phi[g, a] for all points of planes z0..z1-1, g in x-fastest order."""
    tx, ty, tz = tabs
    if sel is not None:
        tx, ty, tz = tx[:, sel], ty[:, sel], tz[:, sel]
    ph = tz[z0:z1, None, None, :] * ty[None, :, None, :] * tx[None, None, :, :]
    return ph.reshape(-1, ph.shape[-1])


def potential_matrix(sysm, v, eta=1e-10, windowed=True, planes=4):
    """V_ab = h^3 sum_{g in W_ab} phi_a(r_g) v(r_g) phi_b(r_g)  (Eq. 2.5 / A.6).

    windowed=True restricts every function to its cubic window W_a (A.1.1),
    so the sum runs over W_a intersect W_b; windowed=False is the plain
    all-points definition.  v has shape (nz, ny, nx).  The overlap on the
    grid (Eq. 2.1) is potential_matrix(v = 1).  Contracted functions (Eq.
    A.1) are sums of Cartesian terms: V = C V_terms C^T (basis.expansion).
    """
    fn, C = basis.expansion(sysm)
    tabs = basis.axis_tables(sysm, fn, eta if windowed else None)
    K = len(fn["zeta"])
    V = np.zeros((K, K))
    vf = np.asarray(v, dtype=np.float64).reshape(int(sysm.grid_n[2]), -1)
    for z0, z1 in _slabs(sysm, planes):
        ph = _phi_slab(tabs, z0, z1)
        w = vf[z0:z1].reshape(-1)
        V += ph.T @ (w[:, None] * ph)
    return basis.contract(C, V * sysm.grid_h ** 3)


def potential_matrix_separable(sysm, factors, eta=1e-10, windowed=True, absolute=False):
    """V_ab of Eq. 2.5 / A.6 for a potential that is a sum of products of
    one-dimensional factors, v(x, y, z) = sum_r fx_r(x) fy_r(y) fz_r(z).

    Each function is a product of one-dimensional tabulated factors inside a
    box window (Supp. A.1), so the grid sum factorises per axis:
    V = h^3 sum_r Vx_r o Vy_r o Vz_r (elementwise product) with
    Vd_r[a, b] = sum_i tab_d[i, a] fd_r[i] tab_d[i, b].  This reaches the
    same V as potential_matrix on the full grid at a cost that stays small
    for thousands of functions.  factors: list of (fx, fy, fz) arrays of
    lengths (nx, ny, nz).  absolute=True sums the absolute values of the
    terms instead, h^3 sum_g |phi_a| |v| |phi_b|: the scale of a rounding-error
    bound on V_ab."""
    fn, C = basis.expansion(sysm)
    tabs = basis.axis_tables(sysm, fn, eta if windowed else None)
    if absolute:
        tabs = [np.abs(t) for t in tabs]
        C = None if C is None else np.abs(C)
        factors = [tuple(np.abs(np.asarray(f, dtype=np.float64)) for f in fr) for fr in factors]
    K = len(fn["zeta"])
    V = np.zeros((K, K))
    for fr in factors:
        # grid lines where a factor vanishes and functions that vanish on
        # every remaining line add exact zeros; leave them out
        rows = [np.nonzero(np.asarray(fr[d]))[0] for d in range(3)]
        live = np.ones(K, dtype=bool)
        for d in range(3):
            live &= np.any(tabs[d][rows[d]] != 0.0, axis=0)
        idx = np.nonzero(live)[0]
        if idx.size == 0:
            continue
        term = None
        for d in range(3):
            f = np.asarray(fr[d], dtype=np.float64)[rows[d]]
            t = tabs[d][np.ix_(rows[d], idx)]
            q = t.T @ (f[:, None] * t)
            term = q if term is None else np.multiply(term, q, out=term)
        V[np.ix_(idx, idx)] += term
    return basis.contract(C, V * sysm.grid_h ** 3)


def density_on_grid(sysm, P, eta=1e-10, windowed=True, planes=4):
    """n(r_g) = 2 sum_ab P_ab phi_a(r_g) phi_b(r_g)  (Eq. 2.7), evaluated as
    the column sum of Eq. A.5: n = sum_a 2 phi_a sum_b phi_b P_ba.
    Returns an (nz, ny, nx) array.  Contracted functions: the same sum over
    their Cartesian terms with P_terms = C^T P C."""
    fn, C = basis.expansion(sysm)
    P = P if C is None else C.T @ P @ C
    tabs = basis.axis_tables(sysm, fn, eta if windowed else None)
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    n = np.zeros(nz * ny * nx)
    for z0, z1 in _slabs(sysm, planes):
        ph = _phi_slab(tabs, z0, z1)
        n[z0 * nx * ny:z1 * nx * ny] = 2.0 * np.einsum("ga,ga->g", ph @ P, ph)
    return n.reshape(nz, ny, nx)


def phi_points(sysm, fn, tabs, flat_idx):
    """Phi at selected flat grid indices (x fastest), from the tables."""
    nx, ny = int(sysm.grid_n[0]), int(sysm.grid_n[1])
    flat_idx = np.asarray(flat_idx)
    ix = flat_idx % nx
    iy = (flat_idx // nx) % ny
    iz = flat_idx // (nx * ny)
    return tabs[0][ix] * tabs[1][iy] * tabs[2][iz]


def density_at(sysm, P, flat_idx, eta=1e-10, windowed=True, absolute=False):
    """n at selected flat grid indices (Eq. 2.7), for sampled checks.
    absolute=True sums the absolute values of the terms,
    2 sum_ab |phi_a| |P_ab| |phi_b|: the scale of a rounding-error bound on n."""
    fn, C = basis.expansion(sysm)
    if C is not None:
        P = (np.abs(C).T @ np.abs(P) @ np.abs(C)) if absolute else C.T @ P @ C
    tabs = basis.axis_tables(sysm, fn, eta if windowed else None)
    ph = phi_points(sysm, fn, tabs, flat_idx)
    if absolute:
        ph, P = np.abs(ph), np.abs(P)
    return 2.0 * np.einsum("ga,ga->g", ph @ P, ph)


def potential_entries(sysm, v, pairs, eta=1e-10, windowed=True):
    """Selected V_ab (Eq. A.6) summed over the intersection box of the two
    windows only, for sampled checks on large systems."""
    if basis.is_contracted(sysm):
        raise NotImplementedError("sampled pair sums are written for one-primitive functions")
    fn = basis.functions(sysm)
    lo, hi = basis.window_ranges(sysm, fn, eta)
    h3 = sysm.grid_h ** 3
    out = []
    vv = np.asarray(v).reshape(int(sysm.grid_n[2]), int(sysm.grid_n[1]), int(sysm.grid_n[0]))
    for a, b in pairs:
        l = np.maximum(lo[a], lo[b]) if windowed else np.zeros(3, np.int64)
        u = np.minimum(hi[a], hi[b]) if windowed else np.asarray(sysm.grid_n) - 1
        if np.any(l > u):
            out.append(0.0)
            continue
        xs = [sysm.grid_origin[d] + sysm.grid_h * np.arange(l[d], u[d] + 1) for d in range(3)]
        Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        sub = {k: fn[k][[a, b]] for k in fn}
        ph = basis.phi_at(sub, pts)
        w = vv[l[2]:u[2] + 1, l[1]:u[1] + 1, l[0]:u[0] + 1].ravel()
        out.append(h3 * float(np.sum(ph[:, 0] * w * ph[:, 1])))
    return np.array(out)
