"""GB300 Chebyshev density-matrix DFT (arXiv 2108.13478), Python side.

`_binding` mirrors the C ABI of include/dft.h one function per entry point.
`Context` below bundles the descriptors and the device workspace so that a
caller can go from atoms and shells to SCF steps in a few lines; it only
marshals arguments, every step runs in libdft's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _binding as B
from ._binding import (  # noqa: F401
    DftError, dft_basis_desc, dft_grid_desc, dft_info, dft_params,
    DFT_PREC_FP64, DFT_PREC_BF16X3, DFT_PREC_FP16X3, DFT_MODEL_LITERAL, DFT_MODEL_NEUTRAL, DFT_MIX_LINEAR, DFT_MIX_KERKER, DFT_MIX_PULAY,
    DFT_XC_SLATER, DFT_XC_PW92, dft_nonlocal_matrix, DFT_PRECOND_BLOCK_JACOBI, DFT_PRECOND_NONE, dft_columns_info,
    dft_workspace_bytes, dft_init_basis, dft_overlap_kinetic, dft_density_matrix, dft_density_on_grid,
    dft_potential_matrix, dft_hartree_xc, dft_scf_step, dft_initial_density, dft_destroy, dft_last_error,
    dft_version, dft_kernel_launches, dft_spectral_bounds_static, dft_scf_step_batched,
    dft_density_from_potential, dft_warmstart_state_bytes, dft_warmstart_param_count, dft_warmstart_init,
    dft_warmstart_potential, dft_warmstart_accumulate, dft_warmstart_adam, dft_warmstart_read,
)


def make_params(*, kT, n_electrons, eta=1e-10, cheb_tail_tol=1e-10, cheb_order=0, precision=DFT_PREC_FP64,
                e_min=0.0, e_max=0.0, lanczos_steps=64, model=DFT_MODEL_LITERAL, vloc_depth=4.0, vloc_width=1.5,
                ion_charge=4.0, mixer=DFT_MIX_LINEAR, mix_alpha=0.3, kerker_q0=0.8, mix_history=8,
                seed=1234, skip_correction=0, reuse_mu=0, nl_channels=0, nl_zeta=1.0, nl_e_s=0.0, nl_e_p=0.0,
                xc=DFT_XC_SLATER) -> dft_params:
    p = dft_params()
    p.beta = 1.0 / kT
    p.n_electrons = n_electrons
    p.eta = eta
    p.cheb_tail_tol = cheb_tail_tol
    p.cheb_order = cheb_order
    p.precision = precision
    p.e_min, p.e_max = e_min, e_max
    p.lanczos_steps = lanczos_steps
    p.model = model
    p.vloc_depth, p.vloc_width, p.ion_charge = vloc_depth, vloc_width, ion_charge
    p.mixer, p.mix_alpha, p.kerker_q0, p.mix_history = mixer, mix_alpha, kerker_q0, mix_history
    p.seed = seed
    p.skip_correction = int(skip_correction)
    p.reuse_mu = int(reuse_mu)
    p.nl_channels, p.nl_zeta, p.nl_e_s, p.nl_e_p = int(nl_channels), nl_zeta, nl_e_s, nl_e_p
    p.xc = int(xc)
    return p


def device_f64(t, numel, name, inout=False):
    """Check that t has the layout the C ABI expects for a K x K matrix or a
    grid: a float64 CUDA tensor of numel elements, contiguous (in-place
    arguments must already be, so that the library writes into t itself).
    A host or wrongly typed buffer handed to the kernels would be read as
    device memory, so it is refused here.  Returns the contiguous tensor."""
    import torch
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, not {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if not t.is_contiguous():
        if inout:
            raise ValueError(f"{name} is written in place and must be contiguous")
        t = t.contiguous()
    return t


class Context:
    """One system on one GPU: descriptors, workspace and the libdft context.

    system: any object with xyz (n,3), shell_atom, shell_l, shell_exp,
    grid_origin (3,), grid_h, grid_n (3,) (nx, ny, nz), n_electrons, kT, and
    optionally contracted shells (shell_nprim, prim_exp, prim_coef) and
    spherical (d shells as the five solid harmonics).
    """

    def __init__(self, system, device="cuda", stream=None, **param_kw):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self._xyz = np.ascontiguousarray(system.xyz, dtype=np.float64)
        self._sa = np.ascontiguousarray(system.shell_atom, dtype=np.int32)
        self._sl = np.ascontiguousarray(system.shell_l, dtype=np.int32)
        self._se = np.ascontiguousarray(system.shell_exp, dtype=np.float64)
        b = dft_basis_desc()
        b.n_atoms = int(self._xyz.shape[0])
        b.xyz = self._xyz.ctypes.data_as(C.POINTER(C.c_double))
        b.n_shells = int(self._sa.shape[0])
        b.shell_atom = self._sa.ctypes.data_as(C.POINTER(C.c_int))
        b.shell_l = self._sl.ctypes.data_as(C.POINTER(C.c_int))
        b.shell_exp = self._se.ctypes.data_as(C.POINTER(C.c_double))
        if getattr(system, "shell_nprim", None) is not None:
            self._np = np.ascontiguousarray(system.shell_nprim, dtype=np.int32)
            self._pe = np.ascontiguousarray(system.prim_exp, dtype=np.float64)
            self._pc = np.ascontiguousarray(system.prim_coef, dtype=np.float64)
            b.shell_nprim = self._np.ctypes.data_as(C.POINTER(C.c_int))
            b.prim_exp = self._pe.ctypes.data_as(C.POINTER(C.c_double))
            b.prim_coef = self._pc.ctypes.data_as(C.POINTER(C.c_double))
        b.spherical = 1 if getattr(system, "spherical", False) else 0
        g = dft_grid_desc()
        for d in range(3):
            g.origin[d] = float(system.grid_origin[d])
            g.n[d] = int(system.grid_n[d])
        g.h = float(system.grid_h)
        param_kw.setdefault("kT", system.kT)
        param_kw.setdefault("n_electrons", system.n_electrons)
        self.params = make_params(**param_kw)
        self.basis, self.grid = b, g
        nbytes = dft_workspace_bytes(b, g, self.params)
        if nbytes == 0:
            raise DftError(B.DFT_EINVAL, "invalid system description")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws = self.workspace[off:off + nbytes]
        self.ctx = dft_init_basis(b, g, self.params, self._ws, stream)
        per_l = {0: 1, 1: 3, 2: 5 if b.spherical else 6}
        self.K = int(sum(per_l[int(l)] for l in self._sl))
        self.grid_shape = (int(g.n[2]), int(g.n[1]), int(g.n[0]))
        self.n_atoms = b.n_atoms

    def close(self):
        if getattr(self, "ctx", None) is not None:
            dft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # allocation helpers (device memory through torch)
    def matrix(self):
        return self.torch.zeros((self.K, self.K), dtype=self.torch.float64, device=self.device)

    def grid_array(self):
        return self.torch.zeros(self.grid_shape, dtype=self.torch.float64, device=self.device)

    def overlap_kinetic(self, stream=None):
        S, T = self.matrix(), self.matrix()
        dft_overlap_kinetic(self.ctx, S, T, stream)
        return S, T

    def _mat(self, t, name, inout=False):
        return device_f64(t, self.K * self.K, name, inout)

    def _grid(self, t, name, inout=False):
        return device_f64(t, int(np.prod(self.grid_shape)), name, inout)

    def density_matrix(self, F, stream=None):
        P = self.matrix()
        info = dft_density_matrix(self.ctx, self._mat(F, "F"), P, stream)
        return P, info

    def density_matrix_columns(self, F, cols, mu, e_min, e_max, n_cheb, thresh=0.0,
                               precond=B.DFT_PRECOND_BLOCK_JACOBI, pcg_tol=1e-10, pcg_maxit=2000, stream=None):
        """P[:, cols] (K x len(cols)) by the sparse-operator route: the
        Chebyshev recurrence on the unit columns with S^-1 by PCG on the
        thresholded sparse S (see include/dft.h)."""
        torch = self.torch
        cols = [int(x) for x in np.asarray(cols).ravel()]
        if not cols:
            raise ValueError("cols is empty")
        if any(x < 0 or x >= self.K for x in cols):
            raise ValueError(f"column indices must lie in [0, {self.K})")
        F = self._mat(F, "F").reshape(self.K, self.K)
        out = torch.empty((self.K, len(cols)), dtype=torch.float64, device=self.device)
        info = B.dft_density_matrix_columns(self.ctx, F, cols, mu, e_min, e_max, n_cheb, thresh,
                                            precond, pcg_tol, pcg_maxit, out, stream)
        return out, info

    def nonlocal_matrix(self, stream=None):
        """V^NL (K x K), formed by overlap_kinetic (zeros without projectors)."""
        V = self.matrix()
        dft_nonlocal_matrix(self.ctx, V, stream)
        return V

    def spectral_bounds_static(self, F, stream=None):
        """(E_min, E_max) of S^-1 F from the allocation-free entry point."""
        return dft_spectral_bounds_static(self.ctx, self._mat(F, "F"), stream)

    def density_on_grid(self, P, stream=None):
        n = self.grid_array()
        dft_density_on_grid(self.ctx, self._mat(P, "P"), n, stream)
        return n

    def potential_matrix(self, v, stream=None):
        V = self.matrix()
        dft_potential_matrix(self.ctx, self._grid(v, "v"), V, stream)
        return V

    def hartree_xc(self, n, stream=None):
        v = self.grid_array()
        e = dft_hartree_xc(self.ctx, self._grid(n, "n"), v, stream)
        return v, e

    def initial_density(self, stream=None):
        n = self.grid_array()
        dft_initial_density(self.ctx, n, stream)
        return n

    def scf_step(self, n_in_out, v_ks_out=None, P_out=None, stream=None):
        n_in_out = self._grid(n_in_out, "n_in_out", inout=True)
        if v_ks_out is not None:
            v_ks_out = self._grid(v_ks_out, "v_ks_out", inout=True)
        if P_out is not None:
            P_out = self._mat(P_out, "P_out", inout=True)
        return dft_scf_step(self.ctx, n_in_out, v_ks_out, P_out, stream)
