"""The benchmark's multi-rank bookkeeping on CPU ranks (gloo, world size 2).

With N GPUs the benchmark runs one replica of the workload per rank (the
path needs no collective); the job is timed by its slowest rank and its
throughput is the units of all ranks over that time.  The reference arm runs
on rank 0 only.  These are the host-side parts of the N > 1 path, exercised
here with two gloo ranks on 127.0.0.1.
"""
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(local_ms[rank], world, "cpu")
        q.put((rank, m, bench.job_throughput(world, 4650, 3, m)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_are_timed_by_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [1200.0, 955.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 1200.0
        assert v == pytest.approx(2 * 4650 * 3 / 1.2)


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_throughput(1, 640, 2, 500.0) == pytest.approx(2560.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import workloads as w
    args = types.SimpleNamespace(warmup=0, steps=1, cpu_budget=1.0, gpus=2)
    bench.run_reference(args, w.config_system("tiny8"), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(capsys):
    """Rank 0 prints one JSON line with the contract's keys: the oracle's
    throughput, its time per step, a CPU-baseline record and an end-to-end
    record without host-device copies."""
    import json
    import workloads as w
    s = w.config_system("tiny8")
    args = types.SimpleNamespace(warmup=1, steps=2, cpu_budget=1.0, gpus=1)
    bench.run_reference(args, s, rank=0, world=1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    # a step is one bounded sample: its wall time, with the projected time of a
    # whole oracle SCF step (the basis of value) beside it
    assert d["value"] > 0 and d["projected_ms_per_scf_step"] == pytest.approx(1000.0 * s.n_basis / d["value"])
    assert 0 < d["ms_per_step"] < 60000.0 and d["value_kind"].startswith("projected")
    assert len(d["cpu_baseline"]["sample"]) <= 120
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "tiny8"


def test_chebyshev_tail_defaults():
    """FP64 keeps the 1e-10 tail its 1e-9 parity needs; the mixed precisions
    take 1e-5 (see tests/test_oracle_truncation.py); an explicit --cheb-tail
    wins."""
    ns = lambda p, t=None: types.SimpleNamespace(precision=p, cheb_tail=t)
    assert bench.cheb_tail(ns("fp64")) == 1e-10
    assert bench.cheb_tail(ns("fp16x3")) == 1e-5 and bench.cheb_tail(ns("bf16x3")) == 1e-5
    assert bench.cheb_tail(ns("fp16x3", 1e-8)) == 1e-8


def test_clock_samples_summarised():
    """The clock record of the bench line from nvidia-smi's CSV rows (index,
    clocks.sm, clocks.max.sm, power.draw, active-reasons mask, then the
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown and sw_power_cap
    flags): median SM clock under load, the maximum clock, and every reason
    seen Active in any sample; short or non-numeric rows are skipped."""
    rows = ["0, 2070, 2070, 1180.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1950, 2070, 1398.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    c = bench.ClockSampler.summarise(rows)
    assert c == {"sm_mhz": 1995.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.ClockSampler.summarise(["0, 1500, 2070, 900, 0x8, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.ClockSampler.summarise([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_upper_triangle_tile_count():
    """Tiles of the tensor-core step: 128 x 256 output tiles that reach the
    upper triangle, counted against a brute-force scan of their elements."""
    import numpy as np
    for K in (80, 370, 640, 1000):
        mt, nt = -(-K // 128), -(-K // 256)
        brute = 0
        for i in range(mt):
            for j in range(nt):
                r = np.arange(i * 128, i * 128 + 128)[:, None]
                c = np.arange(j * 256, j * 256 + 256)[None, :]
                brute += bool(np.any(c >= r))
        assert bench.tc_tiles(K) == brute
