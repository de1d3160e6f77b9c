"""bench.py's algorithmic-work constants equal the oracle's count, and the
reference arm prints the contract's JSON line (CPU only)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_constants_match_oracle_count(oracle_mod):
    sys.path.insert(0, ROOT)
    import bench
    from oracle import count_work
    w = count_work.work()
    assert bench.ALGO["fp64_flops_per_subgrid_stage"] == w["fp64_flops_per_subgrid_stage"]
    assert bench.ALGO["bytes_per_subgrid_stage"] == w["bytes_per_subgrid_stage"]


@pytest.mark.slow
def test_reference_arm_json_line(oracle_mod):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "cpu_baseline", "e2e", "config", "higher_is_better"):
        assert k in line


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # per-rank timings of a replicated step: the slowest rank sets the job's time
        got = bench.max_over_ranks({"t_dev": 1.0 + 0.5 * rank, "t_e2e": 3.0 - rank, "t_graph": 2.0})
        dist.barrier()
        q.put((rank, got, bench.job_rate(262144 * 20, world, got["t_dev"])))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    """The N>1 path (independent replicas, one per rank): every rank sees the
    largest time of each timing, and the whole-job value counts the units
    of all ranks over that time."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in out:
        assert got == {"t_dev": 1.5, "t_e2e": 3.0, "t_graph": 2.0}
        assert rate == pytest.approx(262144 * 20 * 2 / 1.5)


def test_single_process_timings_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks({"t_dev": 0.25}) == {"t_dev": 0.25}
    assert bench.job_rate(100.0, 1, 0.5) == 200.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_sampler_summary_and_missing_tool():
    """The clocks record: median SM clock, max clock, active throttle reasons;
    without nvidia-smi (this CPU host) the sampler records no samples."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.out = ("2070, 2070, 900.1, Not Active, Not Active, Not Active, Active\n"
             "1980, 2070, 1300, Not Active, Not Active, Not Active, Not Active\n"
             "2050, 2070, 1200, Not Active, Not Active, Not Active, Not Active\n")
    sm = c.summary()
    assert sm == {"sm_mhz": 2050.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    import shutil
    if shutil.which("nvidia-smi") is None:
        with bench.ClockSampler(0) as c2:
            pass
        assert c2.summary()["samples"] == 0


def test_contact_block_reports_cost_against_unsteepened(monkeypatch):
    """The contact-steepening block: each precision's RK3 step with
    steepening on, as run_form reports it, against the same form without it
    from the run; a form measured without its unsteepened partner reports
    no ratio.  run_form itself (GPU) is replaced by a stand-in."""
    import types

    import torch
    sys.path.insert(0, ROOT)
    import bench
    calls = []

    def fake_run_form(args, H, dev, prec, flush, indicator=None, fused=False, contact=False, workload="polytrope",
                      steps=None, state=None):
        calls.append((prec, fused, contact, workload))
        return {"t_dev": 0.030 if prec == 0 else 0.015, "t_graph": 0.014, "kern_s": 0.0005, "status": 0,
                "rho": torch.full((4,), 1.1), "n": 512, "cells": 512 * 512, "steps": 20}

    monkeypatch.setattr(bench, "run_form", fake_run_form)
    H = types.SimpleNamespace(HYDRO_PREC_MIXED=1, HYDRO_PREC_FP64=0)
    args = types.SimpleNamespace(steps=20)
    res = {"mixed_separate": {"t_dev": 0.012, "kern_s": 0.0004, "rho": torch.ones(4), "steps": 20}}
    out = bench.contact_measure(args, H, None, None, res)
    assert calls == [(1, False, True, "sedov"), (0, False, True, "sedov")]
    m, f = out["mixed"], out["fp64"]
    assert m["value"] == pytest.approx(512 * 512 * 20 / 0.015)
    assert m["ms_per_step"] == pytest.approx(0.75)
    assert m["step_cost_vs_unsteepened"] == pytest.approx(1.25)
    assert m["kernel_cost_vs_unsteepened"] == pytest.approx(1.25)
    assert m["max_rel_density_diff_vs_unsteepened"] == pytest.approx(0.1, rel=1e-6)
    assert "step_cost_vs_unsteepened" not in f and f["device_status"] == 0
    json.dumps(out)
