"""Pins for oracle.warmstart: closed-form dimer descriptor, the adjoint
identity of the potential assembly, and finite differences of the whole
loss chain (descriptor -> network -> potential -> loss)."""
import math

import numpy as np

import workloads as w
from oracle import warmstart as ws


def small_system():
    xyz = np.array([[0.0, 0.0, 0.0], [2.3, 0.4, -1.1], [-1.2, 2.5, 0.7]])
    return w.make_system(xyz, h=0.6, pad=4.0)


def test_dimer_descriptor_closed_form():
    r = 3.7
    G = ws.descriptors(np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]))
    mk = 8.0 * np.arange(32) / 31.0
    s = 8.0 / 31.0
    ref = np.exp(-(r - mk) ** 2 / (2 * s * s)) * 0.5 * (math.cos(math.pi * r / 8.0) + 1)
    assert np.max(np.abs(G[0] - ref)) < 1e-15 and np.max(np.abs(G[1] - ref)) < 1e-15
    far = ws.descriptors(np.array([[0.0, 0.0, 0.0], [8.5, 0.0, 0.0]]))
    assert np.all(far == 0.0)


def test_silu_derivative():
    z = np.linspace(-6, 6, 25)
    fd = (ws.silu(z + 1e-6) - ws.silu(z - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - ws.dsilu(z))) < 1e-8


def test_assembly_adjoint_identity():
    s = small_system()
    rng = np.random.default_rng(0)
    c = rng.normal(size=(3, 16))
    r = rng.normal(size=tuple(int(t) for t in s.grid_n[::-1]))
    lhs = float(np.sum(r * ws.assemble(s, c)))
    rhs = float(np.sum(ws.assemble_adjoint(s, r) * c))
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)


def test_zero_output_layer_gives_start_potential():
    s = small_system()
    theta = ws.init_params(1, scale_out=0.0)
    c, _ = ws.forward(theta, ws.descriptors(s.xyz))
    assert np.all(c == 0.0)


def test_gradient_matches_central_differences():
    s = small_system()
    rng = np.random.default_rng(2)
    theta = ws.init_params(3, scale_out=0.5)
    shp = tuple(int(t) for t in s.grid_n[::-1])
    v_start = 0.1 * rng.normal(size=shp)
    v_target = 0.1 * rng.normal(size=shp)
    L, g = ws.loss_and_grad(theta, s, v_start, v_target)
    for idx in rng.integers(0, ws.n_params(), 12):
        e = np.zeros_like(theta)
        e[idx] = 1e-5
        Lp, _ = ws.loss_and_grad(theta + e, s, v_start, v_target)
        Lm, _ = ws.loss_and_grad(theta - e, s, v_start, v_target)
        fd = (Lp - Lm) / 2e-5
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_assembly_of_one_radial_gaussian():
    """One atom with a single nonzero coefficient c_k = 1 contributes
    exp(-r^2 / w_k^2) inside the 12-bohr cut and nothing beyond it."""
    import workloads as w
    s = w.make_system(np.array([[0.0, 0.0, 0.0]]), h=0.5, pad=13.0)
    k = 9
    c = np.zeros((1, ws.N_OUT))
    c[0, k] = 1.0
    v = ws.assemble(s, c)
    nx, ny, nz = (int(t) for t in s.grid_n)
    o, h = s.grid_origin, s.grid_h
    Z, Y, X = np.meshgrid(o[2] + h * np.arange(nz), o[1] + h * np.arange(ny), o[0] + h * np.arange(nx), indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    wk = ws.widths()[k]
    ref = np.where(r2 < 144.0, np.exp(-r2 / (wk * wk)), 0.0)
    assert np.max(np.abs(v - ref)) < 1e-15
    assert abs(wk - 0.5 * 6.0 ** (k / 15)) < 1e-15
