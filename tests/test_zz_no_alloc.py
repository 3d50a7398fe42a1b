"""The allocation-free spectral-bounds entry point against dft_density_matrix.

dft_spectral_bounds_static serves callers that cannot call cudaMalloc (a
host framework's fixed memory pool, pre-planned execution): its scratch is a
file-scope device array instead of an allocation.  It must return the same
Lanczos bounds that dft_density_matrix computes for the same Fock matrix, on
every call, although all calls share (and overwrite) the one array.  This
file is named to run last, so a failure here leaves every other test run.
"""
import numpy as np
import pytest

import workloads as w
from oracle import scf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402


def fock(name):
    s = w.config_system(name)
    st = scf.setup(s)
    v, _, _ = scf.potential(st, scf.ion_density(s))
    return s, torch.from_numpy(np.ascontiguousarray(scf.fock(st, v))).cuda()


@pytest.mark.parametrize("name", ["tiny8", "cluster64"])
def test_static_bounds_match_density_matrix(name):
    s, F = fock(name)
    ctx = dft.Context(s, cheb_order=200)
    ctx.overlap_kinetic()
    _, info = ctx.density_matrix(F)
    width = info.e_max - info.e_min
    for _ in range(2):   # two calls in a row reuse the same static scratch
        lo, hi = ctx.spectral_bounds_static(F)
        assert abs(lo - info.e_min) <= 1e-12 * width
        assert abs(hi - info.e_max) <= 1e-12 * width
    ctx.close()


def test_static_bounds_fixed_in_the_parameters():
    """A context with fixed bounds (e_max > e_min) skips Lanczos in
    dft_density_matrix; the allocation-free call returns the same bounds."""
    s, F = fock("tiny8")
    ctx = dft.Context(s, cheb_order=200, e_min=3.5, e_max=13.5)   # the spectrum is [4.24, 12.61]
    ctx.overlap_kinetic()
    _, info = ctx.density_matrix(F)
    assert (info.e_min, info.e_max) == (3.5, 13.5)
    assert ctx.spectral_bounds_static(F) == (3.5, 13.5)
    ctx.close()


def test_static_bounds_mixed_precision_context():
    """A mixed-precision context forms F~ by split-FP16 products inside
    dft_density_matrix; the allocation-free call's FP64 F~ gives the same
    padded bounds to that rounding."""
    s, F = fock("cluster64")
    ctx = dft.Context(s, cheb_order=200, precision=dft.DFT_PREC_FP16X3)
    ctx.overlap_kinetic()
    _, info = ctx.density_matrix(F)
    width = info.e_max - info.e_min
    for _ in range(2):
        lo, hi = ctx.spectral_bounds_static(F)
        assert abs(lo - info.e_min) <= 1e-5 * width
        assert abs(hi - info.e_max) <= 1e-5 * width
    ctx.close()


def test_static_bounds_reject_large_k():
    s = w.config_system("sphereR14")        # K = 870 > 768
    ctx = dft.Context(s, cheb_order=200)
    F = ctx.matrix()
    with pytest.raises(dft.DftError) as e:
        ctx.spectral_bounds_static(F)
    assert e.value.status == dft._binding.DFT_EINVAL
    assert "768" in str(e.value)
    ctx.close()
