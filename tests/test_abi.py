"""Host-side checks of the C ABI: the library loads, exports every entry
point declared in include/dft.h, and sizes workspaces without a GPU."""
import ctypes
import os
import re
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return os.path.join(ROOT, "paper_2108_13478_gb300", "libdft.so")


def header_functions():
    src = open(os.path.join(ROOT, "include", "dft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dft_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("dft_init_basis", "dft_overlap_kinetic", "dft_density_matrix", "dft_density_on_grid",
              "dft_potential_matrix", "dft_scf_step", "dft_workspace_bytes", "dft_destroy", "dft_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for n in header_functions():
        assert hasattr(lib, n), n


def test_binding_covers_header(built):
    from paper_2108_13478_gb300 import _binding
    declared = set(header_functions())
    bound = {s[0] for s in _binding.SIGNATURES}
    assert declared == bound


def test_struct_sizes_match_header(built):
    """The ctypes mirrors have the C layout (checked against offsets that a
    C compiler computes from the header)."""
    import subprocess
    import tempfile
    from paper_2108_13478_gb300 import _binding as B
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "dft.h"
int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dft_basis_desc), sizeof(dft_grid_desc),
 sizeof(dft_params), sizeof(dft_info), offsetof(dft_params, seed), offsetof(dft_info, ms_stage),
 offsetof(dft_params, kerker_q0) + offsetof(dft_params, mix_history) * 1000, sizeof(dft_columns_info),
 offsetof(dft_columns_info, ms));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    got = [ctypes.sizeof(B.dft_basis_desc), ctypes.sizeof(B.dft_grid_desc), ctypes.sizeof(B.dft_params),
           ctypes.sizeof(B.dft_info), B.dft_params.seed.offset, B.dft_info.ms_stage.offset,
           B.dft_params.kerker_q0.offset + B.dft_params.mix_history.offset * 1000,
           ctypes.sizeof(B.dft_columns_info), B.dft_columns_info.ms.offset]
    assert got == out


def test_workspace_bytes_and_invalid_input(built):
    import paper_2108_13478_gb300 as dft
    import workloads as w
    s = w.config_system("tiny8")
    xyz = np.ascontiguousarray(s.xyz)
    sa = np.ascontiguousarray(s.shell_atom, np.int32)
    sl = np.ascontiguousarray(s.shell_l, np.int32)
    se = np.ascontiguousarray(s.shell_exp)
    b = dft.dft_basis_desc()
    b.n_atoms, b.n_shells = s.n_atoms, len(sa)
    b.xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    b.shell_atom = sa.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.shell_l = sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.shell_exp = se.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g = dft.dft_grid_desc()
    for d in range(3):
        g.origin[d] = s.grid_origin[d]
        g.n[d] = int(s.grid_n[d])
    g.h = s.grid_h
    p = dft.make_params(kT=s.kT, n_electrons=s.n_electrons)
    nb = dft.dft_workspace_bytes(b, g, p)
    K = s.n_basis
    assert nb > 11 * K * K * 8 + 5 * s.n_grid * 8
    assert nb < 64 * K * K * 8 + 64 * s.n_grid * 8 + (1 << 30)
    # f shells are not supported; a d shell is, and adds its functions
    sl_bad = sl.copy()
    sl_bad[0] = 3
    b.shell_l = sl_bad.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    assert dft.dft_workspace_bytes(b, g, p) == 0
    sl_d = sl.copy()
    sl_d[0] = 2
    b.shell_l = sl_d.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    assert dft.dft_workspace_bytes(b, g, p) > nb
    b.shell_l = sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    # contracted shells need their primitive arrays; non-positive exponents are refused
    npr = np.full(len(sa), 2, np.int32)
    b.shell_nprim = npr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    assert dft.dft_workspace_bytes(b, g, p) == 0
    pe = np.repeat(se, 2)
    pc = np.tile([0.6, 0.5], len(sa))
    b.prim_exp = pe.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    b.prim_coef = pc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert dft.dft_workspace_bytes(b, g, p) > nb
    pe[3] = -1.0
    assert dft.dft_workspace_bytes(b, g, p) == 0
    b.shell_nprim = None
    b.prim_exp = None
    b.prim_coef = None
    p.beta = -1.0
    assert dft.dft_workspace_bytes(b, g, p) == 0
    assert "sm_103a" in dft.dft_version()


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2108_13478_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f


def _desc(dft, s):
    """Descriptors of a workload system; the arrays are kept alive on the returned tuple."""
    arrs = (np.ascontiguousarray(s.xyz), np.ascontiguousarray(s.shell_atom, np.int32),
            np.ascontiguousarray(s.shell_l, np.int32), np.ascontiguousarray(s.shell_exp))
    b = dft.dft_basis_desc()
    b.n_atoms, b.n_shells = s.n_atoms, len(arrs[1])
    b.xyz = arrs[0].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    b.shell_atom = arrs[1].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.shell_l = arrs[2].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.shell_exp = arrs[3].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g = dft.dft_grid_desc()
    for d in range(3):
        g.origin[d] = s.grid_origin[d]
        g.n[d] = int(s.grid_n[d])
    g.h = s.grid_h
    return b, g, arrs


@pytest.mark.parametrize("name,lo_gb,hi_gb", [("sphere25", 2.0, 4.0), ("sphere40", 25.0, 64.0)])
def test_workspace_of_the_large_workloads_fits_one_gpu(built, name, lo_gb, hi_gb):
    """The mixed-precision workspace (K x K FP64 matrices, 16-bit operand
    pairs padded to 256, rho pairs, grids and the padded FFT grid) of the
    465- and 1963-atom spheres: a few GB and a few tens of GB of the
    GPU's 284 GB (host-side sizing, no device needed)."""
    import paper_2108_13478_gb300 as dft
    import workloads as w
    s = w.config_system(name)
    b, g, _keep = _desc(dft, s)
    p = dft.make_params(kT=s.kT, n_electrons=s.n_electrons, precision=dft.DFT_PREC_FP16X3)
    nb = dft.dft_workspace_bytes(b, g, p)
    K = s.n_basis
    Kp = -(-K // 256) * 256
    assert nb >= 8 * K * K * 8 + 4 * Kp * Kp * 2      # at least the FP64 matrices and the operand pairs
    assert lo_gb * 1e9 < nb < hi_gb * 1e9


class Dev:
    """Stands in for a CUDA tensor on a host without a GPU."""
    is_cuda = True

    def __init__(self, n, dtype=None, contiguous=True):
        import torch
        self.n, self.dtype, self.c = n, torch.float64 if dtype is None else dtype, contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.c

    def contiguous(self):
        return Dev(self.n, self.dtype, True)


def test_context_refuses_buffers_the_kernels_cannot_read(built):
    """The Python side checks what the C ABI cannot: a host tensor, another
    dtype or a wrong size would be read by the kernels as device memory."""
    import torch
    import paper_2108_13478_gb300 as dft

    with pytest.raises(ValueError, match="CUDA"):
        dft.device_f64(torch.zeros(16, dtype=torch.float64), 16, "F")
    with pytest.raises(ValueError, match="float64"):
        dft.device_f64(Dev(16, torch.float32), 16, "F")
    with pytest.raises(ValueError, match="elements"):
        dft.device_f64(Dev(15), 16, "F")
    with pytest.raises(ValueError, match="in place"):
        dft.device_f64(Dev(16, contiguous=False), 16, "n_in_out", inout=True)
    t = Dev(16)
    assert dft.device_f64(t, 16, "F") is t
    assert dft.device_f64(Dev(16, contiguous=False), 16, "F").is_contiguous()


def test_batched_step_refuses_host_densities(built):
    import torch
    import paper_2108_13478_gb300 as dft
    with pytest.raises(ValueError, match="CUDA"):
        dft.dft_scf_step_batched([None], [torch.zeros(8, dtype=torch.float64)])
    with pytest.raises(ValueError, match="one density"):
        dft.dft_scf_step_batched([None, None], [torch.zeros(8, dtype=torch.float64)])


def test_context_methods_check_each_argument(built, monkeypatch):
    """Every Context method sends matrices and grids through the check with
    its own size (K x K or the grid), and in-place SCF arguments must be
    contiguous; the library calls are replaced by recorders."""
    import torch
    import paper_2108_13478_gb300 as dft
    c = object.__new__(dft.Context)
    c.torch, c.device, c.K, c.grid_shape, c.ctx = torch, torch.device("cpu"), 4, (2, 3, 5), None
    calls = []
    for name in ("dft_density_matrix", "dft_density_on_grid", "dft_potential_matrix", "dft_hartree_xc",
                 "dft_scf_step"):
        monkeypatch.setattr(dft, name, lambda *a, _n=name: calls.append(_n))
    mat, grid = Dev(16), Dev(30)
    c.density_matrix(mat)
    c.density_on_grid(mat)
    c.potential_matrix(grid)
    c.hartree_xc(grid)
    c.scf_step(grid, grid, mat)
    c.scf_step(grid)
    assert calls == ["dft_density_matrix", "dft_density_on_grid", "dft_potential_matrix", "dft_hartree_xc",
                     "dft_scf_step", "dft_scf_step"]
    for bad in (lambda: c.density_matrix(grid), lambda: c.density_on_grid(torch.zeros(16, dtype=torch.float64)),
                lambda: c.potential_matrix(mat), lambda: c.hartree_xc(Dev(30, torch.float32)),
                lambda: c.scf_step(Dev(30, contiguous=False)), lambda: c.scf_step(grid, None, grid)):
        with pytest.raises(ValueError):
            bad()
    assert len(calls) == 6


def test_static_bounds_refuse_buffers_the_kernels_cannot_read(built, monkeypatch):
    """The allocation-free bounds call reads K x K doubles from F's pointer:
    the binding refuses host, non-float64, non-square or non-contiguous
    tensors, and the Context method also a size other than K x K, before the
    library is called."""
    import torch
    import paper_2108_13478_gb300 as dft
    from paper_2108_13478_gb300 import _binding as B

    class Mat(Dev):
        def __init__(self, shape, dtype=None, contiguous=True):
            super().__init__(int(np.prod(shape)), dtype, contiguous)
            self.shape = shape

        def dim(self):
            return len(self.shape)

    called = []
    monkeypatch.setattr(B, "lib", types.SimpleNamespace(
        dft_spectral_bounds_static=lambda *a: called.append(a) or 0, dft_last_error=lambda c: b""))
    monkeypatch.setattr(B, "_stream", lambda s=None: None)
    monkeypatch.setattr(B, "_ptr", lambda t: None)
    with pytest.raises(ValueError, match="CUDA"):
        dft.dft_spectral_bounds_static(None, torch.zeros((4, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        dft.dft_spectral_bounds_static(None, Mat((4, 4), torch.float32))
    with pytest.raises(ValueError, match="square"):
        dft.dft_spectral_bounds_static(None, Mat((4, 5)))
    with pytest.raises(ValueError, match="contiguous"):
        dft.dft_spectral_bounds_static(None, Mat((4, 4), contiguous=False))
    c = object.__new__(dft.Context)
    c.torch, c.device, c.K, c.grid_shape, c.ctx = torch, torch.device("cpu"), 4, (2, 3, 5), None
    with pytest.raises(ValueError, match="elements"):
        c.spectral_bounds_static(Mat((3, 3)))
    assert called == []
    c.spectral_bounds_static(Mat((4, 4)))
    assert len(called) == 1


def test_columns_call_checks_its_arguments(built, monkeypatch):
    """dft_density_matrix_columns refuses a null context in the library, and
    the Context method refuses out-of-range columns and a wrong-size F
    before the library is called."""
    import torch
    import paper_2108_13478_gb300 as dft
    from paper_2108_13478_gb300 import _binding as B
    lib = ctypes.CDLL(built)
    lib.dft_density_matrix_columns.restype = ctypes.c_int
    cols = (ctypes.c_int * 1)(0)
    st = lib.dft_density_matrix_columns(None, None, cols, 1, ctypes.c_double(0.0), ctypes.c_double(-1.0),
                                        ctypes.c_double(1.0), 8, ctypes.c_double(0.0), 0, ctypes.c_double(1e-10),
                                        100, None, None, None)
    assert st == B.DFT_EINVAL
    c = object.__new__(dft.Context)
    c.torch, c.device, c.K, c.grid_shape, c.ctx = torch, torch.device("cpu"), 4, (2, 3, 5), None
    calls = []
    monkeypatch.setattr(B, "dft_density_matrix_columns", lambda *a: calls.append(a))
    with pytest.raises(ValueError, match="column"):
        c.density_matrix_columns(Dev(16), [0, 4], 0.0, -1.0, 1.0, 8)
    with pytest.raises(ValueError, match="empty"):
        c.density_matrix_columns(Dev(16), [], 0.0, -1.0, 1.0, 8)
    with pytest.raises(ValueError):
        c.density_matrix_columns(Dev(30), [0], 0.0, -1.0, 1.0, 8)
    assert calls == []


def test_columns_binding_refuses_buffers_the_kernels_cannot_use(built, monkeypatch):
    """The low-level column-route binding reads K x K doubles from F and
    writes K x len(cols) doubles to out: host, non-float64, non-square or
    non-contiguous F, and an out of the wrong type or size, are refused
    before the library is called."""
    import torch
    from paper_2108_13478_gb300 import _binding as B

    class Mat(Dev):
        def __init__(self, shape, dtype=None, contiguous=True):
            super().__init__(int(np.prod(shape)), dtype, contiguous)
            self.shape = shape

        def dim(self):
            return len(self.shape)

    called = []
    monkeypatch.setattr(B, "lib", types.SimpleNamespace(
        dft_density_matrix_columns=lambda *a: called.append(a) or 0, dft_last_error=lambda c: b""))
    monkeypatch.setattr(B, "_stream", lambda s=None: None)
    monkeypatch.setattr(B, "_ptr", lambda t: None)
    args = (0.0, -1.0, 1.0, 8, 0.0, B.DFT_PRECOND_BLOCK_JACOBI, 1e-10, 100)
    good_F, good_out = Mat((4, 4)), Mat((4, 2))
    for F, out, msg in ((torch.zeros((4, 4), dtype=torch.float64), good_out, "CUDA"),
                        (Mat((4, 4), torch.float32), good_out, "float64"),
                        (Mat((4, 5)), good_out, "square"),
                        (Mat((4, 4), contiguous=False), good_out, "contiguous"),
                        (good_F, Mat((4, 2), torch.float32), "out must be"),
                        (good_F, Mat((4, 3)), "elements")):
        with pytest.raises(ValueError, match=msg):
            B.dft_density_matrix_columns(None, F, [0, 3], *args, out)
    assert called == []
    B.dft_density_matrix_columns(None, good_F, [0, 3], *args, good_out)
    assert len(called) == 1
