"""ctypes binding of libdft (include/dft.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory
and the current stream.  Importing this module fails loudly when the shared
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdft.so")

DFT_OK, DFT_EINVAL, DFT_ENOMEM, DFT_ECUDA, DFT_ESPECTRUM, DFT_ENOTCONV, DFT_ETIMEOUT, DFT_EINTERNAL, \
    DFT_EUNSUPPORTED = range(9)
STATUS_NAMES = {0: "DFT_OK", 1: "DFT_EINVAL", 2: "DFT_ENOMEM", 3: "DFT_ECUDA", 4: "DFT_ESPECTRUM",
                5: "DFT_ENOTCONV", 6: "DFT_ETIMEOUT", 7: "DFT_EINTERNAL", 8: "DFT_EUNSUPPORTED"}
DFT_PREC_FP64, DFT_PREC_BF16X3, DFT_PREC_FP16X3 = 0, 1, 2
DFT_MODEL_LITERAL, DFT_MODEL_NEUTRAL = 0, 1
DFT_MIX_LINEAR, DFT_MIX_KERKER, DFT_MIX_PULAY = 0, 1, 2
DFT_XC_SLATER, DFT_XC_PW92 = 0, 1
DFT_PRECOND_BLOCK_JACOBI, DFT_PRECOND_NONE = 0, 1


class dft_basis_desc(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("xyz", C.POINTER(C.c_double)), ("n_shells", C.c_int),
                ("shell_atom", C.POINTER(C.c_int)), ("shell_l", C.POINTER(C.c_int)),
                ("shell_exp", C.POINTER(C.c_double)), ("shell_nprim", C.POINTER(C.c_int)),
                ("prim_exp", C.POINTER(C.c_double)), ("prim_coef", C.POINTER(C.c_double)), ("spherical", C.c_int)]


class dft_grid_desc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("h", C.c_double), ("n", C.c_int * 3)]


class dft_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("n_electrons", C.c_double), ("eta", C.c_double),
                ("cheb_tail_tol", C.c_double), ("cheb_order", C.c_int), ("precision", C.c_int),
                ("e_min", C.c_double), ("e_max", C.c_double), ("lanczos_steps", C.c_int), ("model", C.c_int),
                ("vloc_depth", C.c_double), ("vloc_width", C.c_double), ("ion_charge", C.c_double),
                ("mixer", C.c_int), ("mix_alpha", C.c_double), ("kerker_q0", C.c_double),
                ("mix_history", C.c_int), ("seed", C.c_ulonglong), ("skip_correction", C.c_int),
                ("reuse_mu", C.c_int), ("nl_channels", C.c_int), ("nl_zeta", C.c_double),
                ("nl_e_s", C.c_double), ("nl_e_p", C.c_double), ("xc", C.c_int)]


class dft_info(C.Structure):
    _fields_ = [("mu", C.c_double), ("e_min", C.c_double), ("e_max", C.c_double), ("n_e_trace", C.c_double),
                ("e_total", C.c_double), ("e_kin", C.c_double), ("e_loc", C.c_double), ("e_hartree", C.c_double),
                ("e_xc", C.c_double), ("de_per_atom", C.c_double), ("residual", C.c_double),
                ("n_cheb", C.c_int), ("iter", C.c_int), ("spectrum_ok", C.c_int), ("mu_reused", C.c_int),
                ("ms_stage", C.c_float * 8), ("mu_correction", C.c_double), ("n_e_uncorrected", C.c_double),
                ("e_band_correction", C.c_double), ("e_nl", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_stage"}
        d["ms_stage"] = list(self.ms_stage)
        return d


class dft_columns_info(C.Structure):
    _fields_ = [("nnz_s", C.c_longlong), ("nnz_f", C.c_longlong), ("pcg_solves", C.c_longlong),
                ("pcg_iterations", C.c_longlong), ("max_rel_residual", C.c_double), ("not_converged", C.c_int),
                ("block_cols", C.c_int), ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) for every entry point of include/dft.h
_P = C.c_void_p
SIGNATURES = [
    ("dft_workspace_bytes", C.c_size_t, [C.POINTER(dft_basis_desc), C.POINTER(dft_grid_desc), C.POINTER(dft_params)]),
    ("dft_init_basis", C.c_int, [C.POINTER(_P), C.POINTER(dft_basis_desc), C.POINTER(dft_grid_desc),
                                 C.POINTER(dft_params), _P, C.c_size_t, _P]),
    ("dft_overlap_kinetic", C.c_int, [_P, _P, _P, _P]),
    ("dft_density_matrix", C.c_int, [_P, _P, _P, C.POINTER(dft_info), _P]),
    ("dft_nonlocal_matrix", C.c_int, [_P, _P, _P]),
    ("dft_density_matrix_columns", C.c_int, [_P, _P, C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int, _P,
                                             C.POINTER(dft_columns_info), _P]),
    ("dft_density_on_grid", C.c_int, [_P, _P, _P, _P]),
    ("dft_potential_matrix", C.c_int, [_P, _P, _P, _P]),
    ("dft_hartree_xc", C.c_int, [_P, _P, _P, C.POINTER(C.c_double), _P]),
    ("dft_scf_step", C.c_int, [_P, _P, _P, _P, C.POINTER(dft_info), _P]),
    ("dft_initial_density", C.c_int, [_P, _P, _P]),
    ("dft_scf_step_batched", C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(dft_info), _P]),
    ("dft_density_from_potential", C.c_int, [_P, _P, _P, C.POINTER(dft_info), _P]),
    ("dft_warmstart_state_bytes", C.c_size_t, []),
    ("dft_warmstart_param_count", C.c_int, []),
    ("dft_warmstart_init", C.c_int, [_P, C.POINTER(C.c_float), _P]),
    ("dft_warmstart_potential", C.c_int, [_P, _P, _P, _P, _P]),
    ("dft_warmstart_accumulate", C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double), _P]),
    ("dft_warmstart_adam", C.c_int, [_P, C.c_float, C.c_int, _P]),
    ("dft_warmstart_read", C.c_int, [_P, C.POINTER(C.c_float), C.POINTER(C.c_float), _P]),
    ("dft_destroy", C.c_int, [_P]),
    ("dft_last_error", C.c_char_p, [_P]),
    ("dft_version", C.c_char_p, []),
    ("dft_kernel_launches", C.c_ulonglong, []),
    ("dft_spectral_bounds_static", C.c_int, [_P, _P, C.POINTER(C.c_double), _P]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libdft.so is not built ({path}); run __graft_entry__.build() or "
                          "python paper_2108_13478_gb300/build.py")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class DftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---- thin wrappers with the ABI's names (torch tensors in, status checked) ----

def _check(ctx, st):
    if st != DFT_OK:
        msg = lib.dft_last_error(ctx).decode() if ctx else ""
        raise DftError(st, msg)


def dft_workspace_bytes(basis, grid, params) -> int:
    return int(lib.dft_workspace_bytes(C.byref(basis), C.byref(grid), C.byref(params)))


def dft_init_basis(basis, grid, params, workspace, stream=None):
    ctx = C.c_void_p()
    st = lib.dft_init_basis(C.byref(ctx), C.byref(basis), C.byref(grid), C.byref(params),
                            _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    if st != DFT_OK:
        msg = lib.dft_last_error(ctx).decode() if ctx.value else ""
        if ctx.value:
            lib.dft_destroy(ctx)
        raise DftError(st, msg)
    return ctx


def dft_overlap_kinetic(ctx, S=None, T=None, stream=None):
    _check(ctx, lib.dft_overlap_kinetic(ctx, _ptr(S), _ptr(T), _stream(stream)))


def dft_nonlocal_matrix(ctx, VNL, stream=None):
    _check(ctx, lib.dft_nonlocal_matrix(ctx, _ptr(VNL), _stream(stream)))


def dft_density_matrix(ctx, F, P, stream=None) -> dft_info:
    info = dft_info()
    _check(ctx, lib.dft_density_matrix(ctx, _ptr(F), _ptr(P), C.byref(info), _stream(stream)))
    return info


def _square_f64(F, name):
    import torch
    if not getattr(F, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if F.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, not {F.dtype}")
    if F.dim() != 2 or F.shape[0] != F.shape[1]:
        raise ValueError(f"{name} must be a square matrix")
    if not F.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def dft_density_matrix_columns(ctx, F, cols, mu, e_min, e_max, n_cheb, thresh, precond, pcg_tol, pcg_maxit, out,
                               stream=None) -> dft_columns_info:
    """The kernels read K x K doubles from F's pointer and write K x len(cols)
    doubles to out's: both must be contiguous float64 CUDA tensors of those
    sizes (Context.density_matrix_columns also checks that F is K x K)."""
    import torch
    _square_f64(F, "F")
    n = len(cols)
    if not getattr(out, "is_cuda", False) or out.dtype != torch.float64 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor")
    if out.numel() != F.shape[0] * n:
        raise ValueError(f"out has {out.numel()} elements, expected {F.shape[0]} x {n}")
    info = dft_columns_info()
    carr = (C.c_int * n)(*[int(x) for x in cols])
    _check(ctx, lib.dft_density_matrix_columns(ctx, _ptr(F), carr, n, float(mu), float(e_min), float(e_max),
                                               int(n_cheb), float(thresh), int(precond), float(pcg_tol),
                                               int(pcg_maxit), _ptr(out), C.byref(info), _stream(stream)))
    return info


def dft_density_on_grid(ctx, P, n_grid, stream=None):
    _check(ctx, lib.dft_density_on_grid(ctx, _ptr(P), _ptr(n_grid), _stream(stream)))


def dft_potential_matrix(ctx, v_grid, V, stream=None):
    _check(ctx, lib.dft_potential_matrix(ctx, _ptr(v_grid), _ptr(V), _stream(stream)))


def dft_hartree_xc(ctx, n_grid, v_ks, stream=None):
    e = (C.c_double * 3)()
    _check(ctx, lib.dft_hartree_xc(ctx, _ptr(n_grid), _ptr(v_ks), e, _stream(stream)))
    return tuple(e)


def dft_scf_step(ctx, n_in_out, v_ks_out=None, P_out=None, stream=None) -> dft_info:
    info = dft_info()
    _check(ctx, lib.dft_scf_step(ctx, _ptr(n_in_out), _ptr(v_ks_out), _ptr(P_out), C.byref(info), _stream(stream)))
    return info


def dft_scf_step_batched(ctxs, n_in_out, stream=None):
    """One SCF step for several contexts; returns their dft_info results."""
    import torch
    n = len(ctxs)
    if len(n_in_out) != n:
        raise ValueError("one density per context")
    for q, t in enumerate(n_in_out):
        if not (getattr(t, "is_cuda", False) and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError(f"density {q} must be a contiguous float64 CUDA tensor (it is updated in place)")
    carr = (_P * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    narr = (_P * n)(*[t.data_ptr() for t in n_in_out])
    infos = (dft_info * n)()
    st = lib.dft_scf_step_batched(carr, n, narr, infos, _stream(stream))
    if st != DFT_OK:
        raise DftError(st, lib.dft_last_error(carr[0]).decode())
    return list(infos)


def dft_density_from_potential(ctx, v_grid, n_out, stream=None) -> dft_info:
    info = dft_info()
    _check(ctx, lib.dft_density_from_potential(ctx, _ptr(v_grid), _ptr(n_out), C.byref(info), _stream(stream)))
    return info


def dft_warmstart_state_bytes() -> int:
    return int(lib.dft_warmstart_state_bytes())


def dft_warmstart_param_count() -> int:
    return int(lib.dft_warmstart_param_count())


def _fptr(a):
    import numpy as np
    if a is None:
        return None
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_float))


def dft_warmstart_init(state, params=None, stream=None):
    _check(None, lib.dft_warmstart_init(_ptr(state), _fptr(params), _stream(stream)))


def dft_warmstart_potential(ctx, state, v_start, v0, stream=None):
    _check(ctx, lib.dft_warmstart_potential(ctx, _ptr(state), _ptr(v_start), _ptr(v0), _stream(stream)))


def dft_warmstart_accumulate(ctx, state, v_start, v_target, stream=None) -> float:
    loss = C.c_double()
    _check(ctx, lib.dft_warmstart_accumulate(ctx, _ptr(state), _ptr(v_start), _ptr(v_target), C.byref(loss),
                                             _stream(stream)))
    return loss.value


def dft_warmstart_adam(state, lr, step, stream=None):
    _check(None, lib.dft_warmstart_adam(_ptr(state), C.c_float(lr), int(step), _stream(stream)))


def dft_warmstart_read(state, params=None, grads=None, stream=None):
    _check(None, lib.dft_warmstart_read(_ptr(state), _fptr(params), _fptr(grads), _stream(stream)))


def dft_initial_density(ctx, n_grid, stream=None):
    _check(ctx, lib.dft_initial_density(ctx, _ptr(n_grid), _stream(stream)))


def dft_destroy(ctx):
    lib.dft_destroy(ctx)


def dft_last_error(ctx) -> str:
    return lib.dft_last_error(ctx).decode()


def dft_version() -> str:
    return lib.dft_version().decode()


def dft_spectral_bounds_static(ctx, F, stream=None):
    """Lanczos bounds of S^-1 F through the allocation-free entry point
    (K <= 768); returns (E_min, E_max).  F must be a contiguous square
    float64 CUDA matrix (Context.spectral_bounds_static also checks that it
    is K x K): the kernels read K x K doubles from its pointer."""
    _square_f64(F, "F")
    b = (C.c_double * 2)()
    _check(ctx, lib.dft_spectral_bounds_static(ctx, _ptr(F), b, _stream(stream)))
    return b[0], b[1]


def dft_kernel_launches() -> int:
    return int(lib.dft_kernel_launches())
