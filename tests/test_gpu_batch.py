"""Batched SCF steps of ragged systems (one persistent tensor-core launch per
recurrence step for all systems) against the same steps run one system at a
time.  Each tile's arithmetic is the same in both; the quadrature's FP64
atomics leave differences at the 1e-16 level, which two SCF cycles carry to
about 1e-11 in the density."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2108_13478_gb300 as dft  # noqa: E402

NAMES = ["sphereR10", "tiny8", "cluster64", "tiny5"]


def make(name):
    ctx = dft.Context(w.config_system(name), precision=dft.DFT_PREC_FP16X3, model=dft.DFT_MODEL_NEUTRAL,
                      mixer=dft.DFT_MIX_LINEAR, mix_alpha=0.3, cheb_tail_tol=1e-10)
    ctx.overlap_kinetic()
    return ctx


@pytest.mark.parametrize("shape", [None, "32,0,256,0,0,0,1"])
def test_batched_equals_one_by_one(shape, monkeypatch):
    """Tuned launch shape, and the dataflow shape (each pass one launch over
    all systems' tiles, block counters per system, fixed-point moments)."""
    if shape:
        monkeypatch.setenv("DFT_TC_SHAPE", shape)
    solo = [make(n) for n in NAMES]
    dens_solo = [c.initial_density() for c in solo]
    batch = [make(n) for n in NAMES]
    dens_batch = [c.initial_density() for c in batch]
    for step in range(2):
        infos_s = [c.scf_step(d) for c, d in zip(solo, dens_solo)]
        infos_b = dft.dft_scf_step_batched([c.ctx for c in batch], dens_batch)
        for name, a, b, ds, db in zip(NAMES, infos_s, infos_b, dens_solo, dens_batch):
            assert a.n_cheb == b.n_cheb, name
            assert abs(a.e_total - b.e_total) <= 1e-10 * abs(a.e_total), name
            assert abs(a.mu - b.mu) <= 1e-9, name
            assert float((ds - db).abs().max()) <= 1e-9 * float(ds.abs().max()), name
    for c in solo + batch:
        c.close()


def test_batched_rejects_fp64_and_duplicates():
    a = make("tiny8")
    f = dft.Context(w.config_system("tiny5"))
    f.overlap_kinetic()
    n = a.initial_density()
    with pytest.raises(dft.DftError):
        dft.dft_scf_step_batched([a.ctx, f.ctx], [n, f.initial_density()])
    with pytest.raises(dft.DftError):
        dft.dft_scf_step_batched([a.ctx, a.ctx], [n, n])
    a.close()
    f.close()
