"""Free-space Hartree potential and LDA exchange on the grid (oracle).

Test infrastructure only; see the package docstring.

The paper solves Poisson's equation by a reciprocal-space method for
isolated systems (Section 2, Supp. A.3).  The oracle uses the Hockney
zero-padded convolution with the Coulomb kernel, which solves the same
free-space problem: v_H(r_g) = h^3 sum_g' G(r_g - r_g') rho(r_g'),
G(r) = 1/|r|, and G(0) the cell average of 1/|r| over one grid cube.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def cube_inv_r_constant():
    """c = int_{[-1/2,1/2]^3} d^3u / |u|, by quadrature.

    Splitting the cube into 24 pyramids (octant x which axis is largest) and
    scaling the two smaller coordinates by the largest one gives
    c = 3 int_0^1 int_0^1 ds dt / sqrt(1 + s^2 + t^2)."""
    val, _ = integrate.dblquad(lambda t, s: 1.0 / math.sqrt(1.0 + s * s + t * t), 0.0, 1.0, 0.0, 1.0,
                               epsabs=1e-14, epsrel=1e-14)
    return 3.0 * val


def fft_size(n):
    """Smallest 2^a 3^b 5^c 7^d >= n."""
    m = n
    while True:
        k = m
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


def hartree(sysm, rho, c0=None):
    """v_H = h^3 (G * rho) on the grid, by circular convolution on a grid of
    at least 2n points per axis (so no image overlaps the box).  rho is the
    charge density (nz, ny, nx) in electrons/bohr^3 (electrons positive)."""
    h = sysm.grid_h
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    Nx, Ny, Nz = fft_size(2 * nx), fft_size(2 * ny), fft_size(2 * nz)
    if c0 is None:
        c0 = cube_inv_r_constant()

    def img(n, N):
        i = np.arange(N)
        return np.minimum(i, N - i).astype(np.float64)
    X = img(nx, Nx)[None, None, :]
    Y = img(ny, Ny)[None, :, None]
    Z = img(nz, Nz)[:, None, None]
    r = h * np.sqrt(X * X + Y * Y + Z * Z)
    with np.errstate(divide="ignore"):
        G = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), c0 / h)
    pad = np.zeros((Nz, Ny, Nx))
    pad[:nz, :ny, :nx] = rho
    v = np.fft.irfftn(np.fft.rfftn(pad) * np.fft.rfftn(G), s=(Nz, Ny, Nx), axes=(0, 1, 2))
    return h ** 3 * v[:nz, :ny, :nx]


def hartree_direct(sysm, rho, c0=None):
    """Brute-force O(N^2) sum of the same discrete convolution (small grids)."""
    h = sysm.grid_h
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    if c0 is None:
        c0 = cube_inv_r_constant()
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * h
    q = np.asarray(rho).ravel()
    out = np.zeros(len(q))
    for i in range(len(q)):
        d = np.sqrt(((pts - pts[i]) ** 2).sum(1))
        g = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), c0 / h)
        out[i] = h ** 3 * (g @ q)
    return out.reshape(nz, ny, nx)


CX = (3.0 / math.pi) ** (1.0 / 3.0)


def slater_exchange(n, floor=1e-30):
    """LDA exchange (Dirac-Slater): v_x = -(3 n / pi)^(1/3),
    eps_x = -(3/4) (3 n / pi)^(1/3); points with n <= floor give 0.
    (The paper uses PW92 LDA, Section 2; exchange alone is the workload's
    functional.)"""
    n = np.asarray(n, dtype=np.float64)
    pos = n > floor
    c = np.where(pos, np.cbrt(np.where(pos, n, 0.0)), 0.0) * CX
    return -c, -0.75 * c


# Perdew-Wang 1992 parametrisation of the spin-unpolarised correlation energy
# per electron of the uniform gas (the paper's LDA, Section 4),
#   eps_c(r_s) = -2 A (1 + a1 r_s) ln(1 + 1 / (2 A (b1 r_s^1/2 + b2 r_s + b3 r_s^3/2 + b4 r_s^2))),
# r_s = (3 / (4 pi n))^(1/3); the published constants for the unpolarised gas:
PW92_A, PW92_A1 = 0.031091, 0.21370
PW92_B = (7.5957, 3.5876, 1.6382, 0.49294)


def pw92_correlation(n, floor=1e-30):
    """PW92 LDA correlation: eps_c(n) and v_c = d(n eps_c)/dn =
    eps_c - (r_s / 3) d eps_c / d r_s; points with n <= floor give 0.
    Returns (v_c, eps_c) like slater_exchange."""
    n = np.asarray(n, dtype=np.float64)
    pos = n > floor
    rs = np.where(pos, (3.0 / (4.0 * math.pi * np.where(pos, n, 1.0))) ** (1.0 / 3.0), 1.0)
    b1, b2, b3, b4 = PW92_B
    sr = np.sqrt(rs)
    q0 = -2.0 * PW92_A * (1.0 + PW92_A1 * rs)
    q1 = 2.0 * PW92_A * (b1 * sr + b2 * rs + b3 * rs * sr + b4 * rs * rs)
    dq1 = PW92_A * (b1 / sr + 2.0 * b2 + 3.0 * b3 * sr + 4.0 * b4 * rs)
    lg = np.log1p(1.0 / q1)
    eps = q0 * lg
    deps = -2.0 * PW92_A * PW92_A1 * lg - q0 * dq1 / (q1 * q1 + q1)
    v = eps - rs / 3.0 * deps
    return np.where(pos, v, 0.0), np.where(pos, eps, 0.0)
