"""Mixed-precision (tensor-core, split 16-bit) path against the FP64 oracle.

The Chebyshev products run on tcgen05 with operands split into hi + lo
16-bit pairs and FP32 accumulation; the recurrence result rho is summed in
FP64.  The errors are reported per result; the gates are the ones the method
needs: P within 2e-5 max-abs and energy-like traces within 1e-5 Ha/atom.
"""
import numpy as np
import pytest

import workloads as w
from oracle import dm, grid_ops, scf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(name, neutral=True):
    s = w.config_system(name)
    st = scf.setup(s, scf.Model(neutral=neutral))
    n0 = scf.ion_density(s)
    v, _, _ = scf.potential(st, n0)
    F = scf.fock(st, v)
    eps = dm.geneig(F, st.S)[0]
    W = eps[-1] - eps[0]
    lo, hi = eps[0] - 0.02 * W, eps[-1] + 0.02 * W
    beta = 1.0 / s.kT
    n_c = dm.cheb_order(0.5 * (lo + hi), beta, lo, hi, 1e-10)
    ref = dm.dm_cheb(F, st.S, s.n_electrons, beta, lo, hi, n_c)
    return s, st, F, lo, hi, n_c, ref


@pytest.mark.parametrize("name,prec,tol_p,tol_e", [
    ("tiny8", "fp16x3", 1e-4, 1e-5),
    ("cluster64", "fp16x3", 1e-4, 1e-5),
    ("tiny8", "bf16x3", 2e-3, 1e-3),
])
def test_mixed_density_matrix(name, prec, tol_p, tol_e):
    s, st, F, lo, hi, n_c, ref = case(name)
    p = dft.DFT_PREC_FP16X3 if prec == "fp16x3" else dft.DFT_PREC_BF16X3
    ctx = dft.Context(s, precision=p, e_min=lo, e_max=hi, cheb_order=n_c, model=dft.DFT_MODEL_NEUTRAL)
    ctx.overlap_kinetic()
    P, info = ctx.density_matrix(dev(F))
    P = P.cpu().numpy()
    dP = P - ref["P"]
    err = float(np.max(np.abs(dP)))
    e_kin = abs(2 * np.sum(dP * st.T)) / s.n_atoms
    e_band = abs(2 * np.sum(dP * F)) / s.n_atoms
    print(f"{name} {prec}: max|dP| {err:.3e}  dEkin/atom {e_kin:.3e}  dEband/atom {e_band:.3e}  "
          f"N_e {info.n_e_trace:.8f}  mu {info.mu:.8f} vs {ref['mu']:.8f}")
    assert info.spectrum_ok == 1
    assert err < tol_p
    assert e_kin < tol_e and e_band < tol_e
    ctx.close()


def test_mixed_grid_kernels_fp32():
    """FP32-arithmetic collocation and quadrature against the FP64 oracle."""
    s = w.config_system("cluster64")
    st = scf.setup(s)
    rng = np.random.default_rng(5)
    v = st.vloc + 0.1 * rng.normal(size=tuple(int(t) for t in s.grid_n[::-1]))
    ctx = dft.Context(s, precision=dft.DFT_PREC_FP16X3)
    V = ctx.potential_matrix(dev(v)).cpu().numpy()
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, s.n_basis, (40, 2))]
    ref = grid_ops.potential_entries(s, v, pairs)
    got = np.array([V[a, b] for a, b in pairs])
    assert np.max(np.abs(got - ref)) < 2e-6 * max(1.0, np.max(np.abs(ref)))
    K = s.n_basis
    A = rng.normal(size=(K, K)) * 0.01
    P = A + A.T
    n = ctx.density_on_grid(dev(P)).cpu().numpy().ravel()
    pick = rng.integers(0, n.size, 200)
    refn = grid_ops.density_at(s, P, pick)
    assert np.max(np.abs(n[pick] - refn)) < 1e-5 * max(1.0, np.max(np.abs(refn)))
    ctx.close()


SHAPES = ["32,0,256", "64,0,256", "32,1,256", "64,1,256", "32,0,128", "32,2,128", "32,0,256,1", "64,0,256,1",
          "32,0,256,0,0,0,1", "64,0,256,0,0,0,1", "16,0,256", "16,0,256,1", "16,0,256,0,0,0,1"]


@pytest.mark.parametrize("name", ["tiny37", "cluster64"])
def test_mixed_launch_shapes(name, monkeypatch):
    """Every tensor-core launch shape (k-block width, persistent grid, 256- or
    128-wide tiles with one or two CTAs per SM, stream-K chunk ranges) gives
    the oracle's density matrix; K = 370 leaves a ragged row and column tile,
    K = 640 a padded one.  Stream-K runs 5 CTAs on 10 chunks at K = 370 (no
    tile cut) and 16 CTAs on 33 chunks at K = 640, where most tiles are cut
    between two CTAs and finished from handed-over partial sums.  The dataflow
    shapes run each pass as one launch: with 5 (K = 370) or 11 (K = 640)
    tiles per step, the grid holds items of many consecutive steps at once,
    so almost every chunk load waits on the block counters of the step
    before and every epilogue on the readers of the block it overwrites.  The
    16-wide k-block shapes use a 9-stage ring with 32-byte swizzled operands
    and keep three of their four mirror buffers inside the ring."""
    s, st, F, lo, hi, n_c, ref = case(name)
    Ps = []
    for shape in SHAPES:
        monkeypatch.setenv("DFT_TC_SHAPE", shape)
        ctx = dft.Context(s, precision=dft.DFT_PREC_FP16X3, e_min=lo, e_max=hi, cheb_order=n_c,
                          model=dft.DFT_MODEL_NEUTRAL)
        ctx.overlap_kinetic()
        P, info = ctx.density_matrix(dev(F))
        P = P.cpu().numpy()
        ctx.close()
        dP = P - ref["P"]
        err = float(np.max(np.abs(dP)))
        e_kin = abs(2 * np.sum(dP * st.T)) / s.n_atoms
        print(f"{name} shape {shape}: max|dP| {err:.3e} dEkin/atom {e_kin:.3e}")
        assert info.spectrum_ok == 1
        assert err < 1e-4 and e_kin < 1e-5
        Ps.append(P)
    # the shapes differ in the order of the moment partial sums and possibly in
    # the tensor core's FP32 rounding inside a chunk
    for shape, P in zip(SHAPES[1:], Ps[1:]):
        d = float(np.max(np.abs(P - Ps[0])))
        print(f"{name} shape {shape} vs {SHAPES[0]}: max|dP| {d:.3e}")
        assert d < 1e-5


def test_expired_waits_return_timeout_and_leave_the_context_usable(monkeypatch):
    """The dataflow launch's block-counter waits are bounded (1 s of the
    GPU's global timer).  With DFT_TEST_EXPIRE_WAITS set, every producer wait
    asks for one write more than any tile makes, so the waits run out: the
    CTAs record FLAG_TIMEOUT, drain their copies and MMAs, free tensor memory
    and return, and the call reports DFT_ETIMEOUT within seconds.  The same
    context then computes the oracle's density matrix."""
    import time
    s, st, F, lo, hi, n_c, ref = case("tiny37")
    monkeypatch.setenv("DFT_TC_SHAPE", "32,0,256,0,0,0,1")
    ctx = dft.Context(s, precision=dft.DFT_PREC_FP16X3, e_min=lo, e_max=hi, cheb_order=n_c,
                      model=dft.DFT_MODEL_NEUTRAL)
    ctx.overlap_kinetic()
    monkeypatch.setenv("DFT_TEST_EXPIRE_WAITS", "1")
    t0 = time.time()
    with pytest.raises(dft.DftError) as e:
        ctx.density_matrix(dev(F))
    took = time.time() - t0
    print(f"expired waits: {e.value} after {took:.1f} s")
    assert e.value.status == dft._binding.DFT_ETIMEOUT
    assert took < 60.0
    monkeypatch.delenv("DFT_TEST_EXPIRE_WAITS")
    P, info = ctx.density_matrix(dev(F))
    dP = P.cpu().numpy() - ref["P"]
    e_kin = abs(2 * np.sum(dP * st.T)) / s.n_atoms
    assert info.spectrum_ok == 1
    assert float(np.max(np.abs(dP))) < 1e-4 and e_kin < 1e-5
    ctx.close()
