"""Parity at full size: the 465-atom silicon sphere (K = 4650, 147^3 grid)
in the mixed precision and the dataflow launch shape that the benchmark times.

Inputs come from the oracle and the seeded geometry only.  The Fock matrix is
F = T + V[v_loc]: the closed-form kinetic matrix plus the quadrature (Eq. 2.5)
of the bare local pseudopotential v_loc = sum_A -4 exp(-|r - R_A|^2 / 1.5^2),
the Hamiltonian of the workload without the density-dependent terms.  Each
well is a product of three one-dimensional factors, so the oracle sums V per
atom in separable form (the plain grid sum over 3.2 M points for 4650
functions is out of reach on the host); the factors are cut where they fall
below 1e-18, and the grid potential handed to the CUDA path is built from the
same cut factors.  At this size its spectrum, occupation and the order N_C
the tail rule picks (about 2900) are those of the first SCF cycle of the
benchmark.

Tolerances:
* S, T: FP64 closed forms on both sides, roundoff (as at K = 640).
* P: the mixed-precision gates of the smaller systems, max|dP| < 1e-4 and
  |2 Tr[dP T]|, |2 Tr[dP F]| < 1e-5 Ha per atom, against the exact
  P = C f(eps) C^T (Eq. 2.9) of one generalised eigensolve.
* V and n (FP32 arithmetic on the mixed path): the rounding-error bound of
  the kernels' summation, (m + 12) u sum|terms| with u = 2^-24 and m the
  longest FP32 sum: 512 points of one grid tile per pair for V (tiles meet
  in 2^-48 fixed point, at most 2^-49 each); for n, up to K terms per
  function plus 32 per chunk.  V is
  compared entry by entry over the whole matrix, n at 300 sampled points and
  through its sum over the grid.
"""
import numpy as np
import pytest

import workloads as w
from oracle import basis, dm, grid_ops, scf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402

FLOW = "32,0,256,0,0,0,1"      # one cooperative launch per recurrence pass
U32 = 2.0 ** -24


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _well(x, c):
    e = np.exp(-(x - c) ** 2 / 1.5 ** 2)
    return np.where(e > 1e-18, e, 0.0)


@pytest.fixture(scope="module")
def sphere():
    s = w.config_system("sphere25")
    fn = basis.functions(s)
    S, T = basis.overlap_kinetic(fn)
    xs, ys, zs = scf.grid_points(s)
    factors = [(-4.0 * _well(xs, R[0]), _well(ys, R[1]), _well(zs, R[2])) for R in s.xyz]
    V = grid_ops.potential_matrix_separable(s, factors)
    F = T + V
    ex = dm.dm_exact(F, S, s.n_electrons, 1.0 / s.kT)
    # the same potential on the grid: each cut well is a product over a sub-box
    nx, ny, nz = (int(t) for t in s.grid_n)
    v = np.zeros((nz, ny, nx))
    for fx, fy, fz in factors:
        ix, iy, iz = (np.nonzero(f)[0] for f in (fx, fy, fz))
        v[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1] += (
            fz[iz][:, None, None] * fy[iy][None, :, None] * fx[ix][None, None, :])
    return dict(s=s, S=S, T=T, V=V, F=F, ex=ex, factors=factors, v=v)


@pytest.fixture(scope="module")
def ctx(sphere):
    mp = pytest.MonkeyPatch()
    mp.setenv("DFT_TC_SHAPE", FLOW)
    c = dft.Context(sphere["s"], precision=dft.DFT_PREC_FP16X3, model=dft.DFT_MODEL_NEUTRAL,
                    cheb_tail_tol=1e-10)
    yield c
    c.close()
    mp.undo()


def test_overlap_kinetic(sphere, ctx):
    S, T = ctx.overlap_kinetic()
    assert np.max(np.abs(host(S) - sphere["S"])) < 1e-13
    assert np.max(np.abs(host(T) - sphere["T"])) < 1e-12


def test_density_matrix(sphere, ctx):
    s, ex, F, T = sphere["s"], sphere["ex"], sphere["F"], sphere["T"]
    ctx.overlap_kinetic()
    P, info = ctx.density_matrix(dev(F))
    P = host(P)
    dP = P - ex["P"]
    err = float(np.max(np.abs(dP)))
    e_kin = abs(2 * np.sum(dP * T)) / s.n_atoms
    e_band = abs(2 * np.sum(dP * F)) / s.n_atoms
    n_e = 2 * np.sum(P * sphere["S"])
    print(f"sphere25 fp16x3 {FLOW}: N_C {info.n_cheb}  max|dP| {err:.3e} (max|P| {np.max(np.abs(ex['P'])):.3f})  "
          f"dEkin/atom {e_kin:.3e}  dEband/atom {e_band:.3e}  2Tr[PS] {n_e:.6f}  "
          f"mu {info.mu:.8f} vs {ex['mu']:.8f}")
    assert info.spectrum_ok == 1
    assert abs(n_e - s.n_electrons) < 1e-5 * s.n_electrons
    assert err < 1e-4
    assert e_kin < 1e-5 and e_band < 1e-5


@pytest.mark.parametrize("skip", [0, 1])
def test_density_matrix_at_the_benchmark_order(sphere, skip):
    """The benchmark runs the mixed path with the Chebyshev tail 1e-5 (about
    half the steps of 1e-10; the oracle's truncated expansion against its
    exact eigensolve gives 9e-10 Ha/atom here, and the K = 640 case is
    pinned in tests/test_oracle_truncation.py): the same gates hold, with
    the FP64 electron-count correction after the recurrence (skip = 0, the
    default) and without it."""
    s, ex, F, T = sphere["s"], sphere["ex"], sphere["F"], sphere["T"]
    mp = pytest.MonkeyPatch()
    mp.setenv("DFT_TC_SHAPE", FLOW)
    c = dft.Context(s, precision=dft.DFT_PREC_FP16X3, model=dft.DFT_MODEL_NEUTRAL, cheb_tail_tol=1e-5,
                    skip_correction=skip)
    try:
        c.overlap_kinetic()
        P, info = c.density_matrix(dev(F))
        P = host(P)
    finally:
        c.close()
        mp.undo()
    dP = P - ex["P"]
    err = float(np.max(np.abs(dP)))
    e_kin = abs(2 * np.sum(dP * T)) / s.n_atoms
    e_band = abs(2 * np.sum(dP * F)) / s.n_atoms
    n_e = 2 * np.sum(P * sphere["S"])
    print(f"sphere25 fp16x3 tail 1e-5 {'without' if skip else 'with'} correction: N_C {info.n_cheb}  "
          f"max|dP| {err:.3e}  dEkin/atom {e_kin:.3e}  dEband/atom {e_band:.3e}  2Tr[PS] {n_e:.6f}  "
          f"dmu {info.mu_correction:+.3e}  stages {[round(x, 1) for x in info.ms_stage]}")
    assert info.spectrum_ok == 1
    assert abs(n_e - s.n_electrons) < 1e-5 * s.n_electrons
    assert err < 1e-4
    assert e_kin < 1e-5 and e_band < 1e-5


def test_potential_matrix(sphere, ctx):
    Vg = host(ctx.potential_matrix(dev(sphere["v"])))
    A = grid_ops.potential_matrix_separable(sphere["s"], sphere["factors"], absolute=True)
    err = np.abs(Vg - sphere["V"])
    # plus the quadrature's fixed-point accumulation across tiles: each tile's
    # contribution is rounded to a multiple of 2^-48, and two functions share
    # at most ~10^3 tiles (windows up to ~29 bohr, 8^3-point tiles at 0.4 bohr)
    bound = (512 + 12) * U32 * A + 1e-13 * np.max(A) + 1e3 * 2.0 ** -49
    print(f"sphere25 V (FP32 quadrature): max|dV| {err.max():.3e}  max|dV|/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


def test_density_on_grid(sphere, ctx):
    s, P = sphere["s"], sphere["ex"]["P"]
    n = host(ctx.density_on_grid(dev(P))).ravel()
    pick = np.random.default_rng(25).integers(0, n.size, 300)
    ref = grid_ops.density_at(s, P, pick)
    A = grid_ops.density_at(s, P, pick, absolute=True)
    err = np.abs(n[pick] - ref)
    bound = (s.n_basis + 32 + 12) * U32 * A + 1e-14
    print(f"sphere25 n (FP32 collocation): max|dn| {err.max():.3e} of max n {ref.max():.3e}  "
          f"max|dn|/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
    # every point at once: h^3 sum_g n = 2 Tr[P S_grid] with the same windows
    # (Eq. 2.1 and Eq. 2.7), within the summed rounding bound of the points
    ones = [tuple(np.ones(int(k)) for k in s.grid_n)]
    Sg = grid_ops.potential_matrix_separable(s, ones)
    Sa = grid_ops.potential_matrix_separable(s, ones, absolute=True)
    total = s.grid_h ** 3 * n.sum()
    tol = (s.n_basis + 32 + 12) * U32 * 2 * np.sum(np.abs(P) * Sa) + 1e-9 * s.n_electrons
    print(f"sphere25 h^3 sum n {total:.6f} vs 2Tr[P S_grid] {2 * np.sum(P * Sg):.6f} (bound {tol:.3e})")
    assert abs(total - 2 * np.sum(P * Sg)) <= tol
