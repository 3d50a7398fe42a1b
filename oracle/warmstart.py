"""Atom-centred learned warm start (oracle, FP64).

Test infrastructure only; see the package docstring.  The paper starts the
SCF cycle from a sum of atomic densities (Supp. A.3); this workload adds a
small network that predicts a correction to the starting potential.  The
definitions below are the reference for the CUDA kernels:

  descriptor  G_Ak = sum_{B != A, r_AB < r_c} exp(-(r_AB - m_k)^2 / (2 s^2)) f_c(r_AB),
              m_k = k r_c / 31 (k = 0..31), s = r_c / 31, r_c = 8 bohr,
              f_c(r) = (cos(pi r / r_c) + 1) / 2
  network     x = G_A / 4; h1 = silu(W1 x + b1); h2 = silu(W2 h1 + b2);
              h3 = silu(W3 h2 + b3); c_A = W4 h3 + b4   (32-128-128-128-16)
  potential   v0(r_g) = v_start(r_g) + sum_A sum_k c_Ak exp(-|r_g - R_A|^2 / w_k^2)
              over atoms with |r_g - R_A| < 12 bohr, w_k = 0.5 * 6^(k/15)
  loss        L = h^3 sum_g (v0 - v*)^2 over the grid (v* a converged v_KS)

Parity status: pinned by tests/test_oracle_warmstart.py (closed-form
descriptor of a dimer, finite differences of the whole chain, the adjoint
identity of the potential assembly).
"""
from __future__ import annotations

import math

import numpy as np

R_C = 8.0
N_DESC = 32
N_HID = 128
N_OUT = 16
R_CUT = 12.0
SIZES = [(N_HID, N_DESC), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID)]


def widths():
    return 0.5 * 6.0 ** (np.arange(N_OUT) / 15.0)


def n_params():
    return sum(o * i + o for o, i in SIZES)


def unpack(theta):
    """Flat parameter vector -> [(W1, b1), ..., (W4, b4)] (W row-major out x in)."""
    out, p = [], 0
    for o, i in SIZES:
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


def init_params(seed=0, scale_out=0.0):
    """He-style initial weights; the output layer starts at zero unless asked."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (o, i) in enumerate(SIZES):
        std = math.sqrt(2.0 / i) if li < 3 else scale_out / math.sqrt(i)
        parts.append(rng.normal(0.0, 1.0, o * i) * std)
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def descriptors(xyz):
    """G (n_atoms, 32) as defined in the module docstring."""
    d = np.sqrt(((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1))
    n = len(xyz)
    mk = R_C * np.arange(N_DESC) / 31.0
    s = R_C / 31.0
    G = np.zeros((n, N_DESC))
    for a in range(n):
        for b in range(n):
            r = d[a, b]
            if a == b or r >= R_C:
                continue
            fc = 0.5 * (math.cos(math.pi * r / R_C) + 1.0)
            G[a] += np.exp(-(r - mk) ** 2 / (2 * s * s)) * fc
    return G


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def forward(theta, G):
    """Per-atom coefficients c (n_atoms, 16) and the cache for backward."""
    L = unpack(theta)
    x = G / 4.0
    cache = [x]
    zs = []
    for li, (W, b) in enumerate(L):
        z = x @ W.T + b
        zs.append(z)
        x = silu(z) if li < 3 else z
        cache.append(x)
    return x, (cache, zs)


def backward(theta, cache, dc):
    """dL/dtheta from dL/dc (n_atoms, 16)."""
    L = unpack(theta)
    acts, zs = cache
    grads = [None] * 4
    g = dc
    for li in range(3, -1, -1):
        W, b = L[li]
        if li < 3:
            g = g * dsilu(zs[li])
        grads[li] = (g.T @ acts[li], g.sum(0))
        g = g @ W
    return np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])


def assemble(sysm, coeffs):
    """sum_A sum_k c_Ak exp(-|r - R_A|^2 / w_k^2), |r - R_A| < R_CUT, on the grid."""
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    o, h = sysm.grid_origin, sysm.grid_h
    xs, ys, zs = o[0] + h * np.arange(nx), o[1] + h * np.arange(ny), o[2] + h * np.arange(nz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    out = np.zeros((nz, ny, nx))
    w = widths()
    for a, R in enumerate(sysm.xyz):
        r2 = (X - R[0]) ** 2 + (Y - R[1]) ** 2 + (Z - R[2]) ** 2
        inside = r2 < R_CUT * R_CUT
        val = np.zeros_like(r2)
        for k in range(N_OUT):
            val += coeffs[a, k] * np.exp(-r2 / (w[k] * w[k]))
        out += np.where(inside, val, 0.0)
    return out


def assemble_adjoint(sysm, resid):
    """d/dc_Ak of sum_g resid_g * assemble(c)_g (the transpose of assemble)."""
    nx, ny, nz = (int(t) for t in sysm.grid_n)
    o, h = sysm.grid_origin, sysm.grid_h
    xs, ys, zs = o[0] + h * np.arange(nx), o[1] + h * np.arange(ny), o[2] + h * np.arange(nz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    w = widths()
    dc = np.zeros((len(sysm.xyz), N_OUT))
    for a, R in enumerate(sysm.xyz):
        r2 = (X - R[0]) ** 2 + (Y - R[1]) ** 2 + (Z - R[2]) ** 2
        inside = r2 < R_CUT * R_CUT
        for k in range(N_OUT):
            dc[a, k] = np.sum(np.where(inside, resid * np.exp(-r2 / (w[k] * w[k])), 0.0))
    return dc


def loss_and_grad(theta, sysm, v_start, v_target):
    """L = h^3 sum (v0 - v*)^2 and dL/dtheta for one system."""
    G = descriptors(sysm.xyz)
    c, cache = forward(theta, G)
    v0 = v_start + assemble(sysm, c)
    r = v0 - v_target
    h3 = sysm.grid_h ** 3
    L = h3 * float(np.sum(r * r))
    dc = 2.0 * h3 * assemble_adjoint(sysm, r)
    return L, backward(theta, cache, dc)


def round_fp16(theta):
    """The network's weights as the GPU stores them (FP16)."""
    return np.asarray(theta, dtype=np.float16).astype(np.float64)
