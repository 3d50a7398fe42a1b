"""Training and use of the learned SCF warm start (orchestration only).

The network, its gradients and Adam run in libdft's kernels
(dft_warmstart_*); this module drives them: it generates training targets
with the library's own SCF (converged Kohn-Sham potentials of seeded
clusters), trains, and starts SCF cycles from the predicted potential.
"""
from __future__ import annotations

import math

import numpy as np

from . import _binding as B
from . import Context, make_params  # noqa: F401


def init_params(seed=0, scale_out=0.0):
    """He-style random hidden layers, zero output layer (the untrained
    network reproduces the superposition-of-atoms start)."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 32), (128, 128), (128, 128), (16, 128)]
    parts = []
    for li, (o, i) in enumerate(sizes):
        std = math.sqrt(2.0 / i) if li < 3 else scale_out / math.sqrt(i)
        parts.append(rng.normal(0.0, 1.0, o * i) * std)
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


class WarmStart:
    """Device state of the network (FP32 master, gradient, Adam moments, FP16 copy)."""

    def __init__(self, params=None, device="cuda"):
        import torch
        self.torch = torch
        self.state = torch.empty(B.dft_warmstart_state_bytes(), dtype=torch.uint8, device=device)
        p = init_params() if params is None else np.ascontiguousarray(params, dtype=np.float32)
        B.dft_warmstart_init(self.state, p)
        self.step = 0

    def params(self):
        out = np.empty(B.dft_warmstart_param_count(), dtype=np.float32)
        B.dft_warmstart_read(self.state, params=out)
        return out

    def grads(self):
        out = np.empty(B.dft_warmstart_param_count(), dtype=np.float32)
        B.dft_warmstart_read(self.state, grads=out)
        return out

    def potential(self, ctx, v_start):
        """v0 = v_start (None: zero) + the network's correction, on ctx's grid."""
        v0 = ctx.grid_array()
        if v_start is not None:
            v_start = ctx._grid(v_start, "v_start")
        B.dft_warmstart_potential(ctx.ctx, self.state, v_start, v0)
        return v0

    def accumulate(self, ctx, v_start, v_target):
        return B.dft_warmstart_accumulate(ctx.ctx, self.state, ctx._grid(v_start, "v_start"),
                                          ctx._grid(v_target, "v_target"))

    def adam(self, lr):
        self.step += 1
        B.dft_warmstart_adam(self.state, lr, self.step)


def scf_context(system, **kw):
    kw.setdefault("precision", B.DFT_PREC_FP16X3)
    kw.setdefault("model", B.DFT_MODEL_NEUTRAL)
    kw.setdefault("mixer", B.DFT_MIX_PULAY)
    kw.setdefault("mix_alpha", 0.3)
    kw.setdefault("kerker_q0", 0.8)
    kw.setdefault("mix_history", 8)
    kw.setdefault("cheb_tail_tol", 1e-10)
    ctx = Context(system, **kw)
    ctx.overlap_kinetic()
    return ctx


def start_potential(ctx):
    """v_KS of the superposition-of-atoms density."""
    n0 = ctx.initial_density()
    v, _ = ctx.hartree_xc(n0)
    return v


def run_scf(ctx, v_first, max_iter=80, tol_e=1e-8, tol_n=1e-5, e_ref=None, e_tol=1e-5, timings=None):
    """SCF cycle that starts from a potential: n_1 = n[v_first], then Pulay
    cycles.  Returns (cycles, final info, converged v_KS, cycles to reach
    |E - e_ref| / atom < e_tol if e_ref is given).  timings (a dict, if
    given) receives the GPU seconds (CUDA events) of the start and of every
    cycle, and the seconds until e_tol was reached."""
    torch = ctx.torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    n = ctx.grid_array()
    B.dft_density_from_potential(ctx.ctx, ctx._grid(v_first, "v_first"), n)
    ev[1].record()
    ev[1].synchronize()
    t = ev[0].elapsed_time(ev[1]) / 1000.0
    if timings is not None:
        timings.update(start_s=t, cycle_s=[], hit_s=None, e_per_atom=[], residual=[])
    v = ctx.grid_array()
    hit = None
    info = None
    for it in range(max_iter):
        ev[0].record()
        info = ctx.scf_step(n, v_ks_out=v)
        ev[1].record()
        ev[1].synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1000.0
        t += dt
        if timings is not None:
            timings["cycle_s"].append(dt)
            timings["e_per_atom"].append(info.e_total / ctx.n_atoms)
            timings["residual"].append(info.residual)
        if e_ref is not None and hit is None and abs(info.e_total / ctx.n_atoms - e_ref) < e_tol:
            hit = it + 1
            if timings is not None:
                timings["hit_s"] = t
        if it > 0 and abs(info.de_per_atom) < tol_e and info.residual < tol_n:
            return it + 1, info, v, hit
    return max_iter, info, v, hit


def training_set(systems, **kw):
    """(context, v_start, converged v_KS) for each system, from the library's SCF."""
    data = []
    for s in systems:
        ctx = scf_context(s, **kw)
        v_start = start_potential(ctx)
        _, _, v_star, _ = run_scf(ctx, v_start)
        data.append((ctx, v_start, v_star))
    return data


def train(ws, data, epochs=60, lr=3e-3, log=None):
    """Full-batch Adam on sum over systems of h^3 sum (v0 - v*)^2."""
    hist = []
    for ep in range(epochs):
        loss = 0.0
        for ctx, v_start, v_star in data:
            loss += ws.accumulate(ctx, v_start, v_star)
        ws.adam(lr)
        hist.append(loss)
        if log:
            log(ep, loss)
    return hist


def compare_starts(ws, system, max_iter=150, **kw):
    """SCF from the superposition-of-atoms potential and from the network's
    potential on one system: cycles and GPU seconds to 1e-5 Ha/atom of the
    converged energy (from a tight run of the atomic start) and to full
    convergence."""
    ref = scf_context(system, **kw)
    n_ref, info, _, _ = run_scf(ref, start_potential(ref), max_iter=max_iter + 80, tol_e=1e-9, tol_n=1e-6)
    e_ref = info.e_total / system.n_atoms
    ref.close()
    out = {"n_atoms": system.n_atoms, "n_basis": int(system.n_basis), "e_ref_per_atom": e_ref,
           "reference_cycles": n_ref, "reference_converged": n_ref < max_iter + 80,
           "reference_last_dE_per_atom": info.de_per_atom, "reference_last_residual": info.residual}
    for key, warm in (("atoms", False), ("warm", True)):
        ctx = scf_context(system, **kw)
        v0 = start_potential(ctx)
        if warm:
            v0 = ws.potential(ctx, v0)
        tm = {}
        n_conv, _, _, hit = run_scf(ctx, v0, max_iter=max_iter, e_ref=e_ref, timings=tm)
        out[key] = {"cycles_to_1e-5": hit, "seconds_to_1e-5": tm["hit_s"], "cycles_to_convergence": n_conv,
                    "converged": n_conv < max_iter, "seconds_to_convergence": tm["start_s"] + sum(tm["cycle_s"]),
                    "dE_per_atom_trace": [float("%.2e" % (e - e_ref)) for e in tm["e_per_atom"]],
                    "residual_trace": [float("%.2e" % r) for r in tm["residual"]]}
        ctx.close()
    return out


def main(argv=None):
    """Train on seeded spheres with the library's own converged potentials and
    compare the two starts on a larger sphere; prints one JSON record."""
    import argparse
    import json
    import os
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as w
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20, help="training spheres")
    ap.add_argument("--rmin", type=float, default=10.0)
    ap.add_argument("--rmax", type=float, default=20.0)
    ap.add_argument("--test-radius", type=float, default=25.0)
    ap.add_argument("--epochs", type=int, default=120)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--cheb-tail", type=float, default=1e-6)
    a = ap.parse_args(argv)
    kw = dict(cheb_tail_tol=a.cheb_tail, reuse_mu=1)
    t0 = time.time()
    radii = np.random.default_rng(a.seed).uniform(a.rmin, a.rmax, a.train)
    systems = [w.config_system(f"sphereR{r:.3f}", seed=a.seed + i) for i, r in enumerate(radii)]
    data = training_set(systems, **kw)
    t_data = time.time() - t0
    ws = WarmStart(init_params(seed=1))
    hist = train(ws, data, epochs=a.epochs, lr=a.lr)
    for c, _, _ in data:
        c.close()
    test = w.config_system(f"sphereR{a.test_radius:g}", seed=99)
    res = compare_starts(ws, test, **kw)
    rec = {"train_spheres": a.train, "train_radii": [round(float(r), 3) for r in radii],
           "train_atoms": [s.n_atoms for s in systems], "epochs": a.epochs, "loss_first": hist[0],
           "loss_last": hist[-1], "test_radius": a.test_radius, "test": res, "targets_s": t_data,
           "wall_s": time.time() - t0}
    print(json.dumps(rec), flush=True)
    return rec


if __name__ == "__main__":
    main()
