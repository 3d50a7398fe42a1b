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
