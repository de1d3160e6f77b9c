"""Benchmark of the hydro hot path on one GB300 (cell-updates/s).

Headline workload: the rotating n = 1.5 polytrope on a uniform octree level
of 32,768 sub-grids of 8^3 cells (256^3 cells on [-1,1]^3, the size of the
paper's Sedov and rotating-star runs, Sec. V and VI), rotating frame
Omega = 0.2, its static gravitational field as an input array, ambient
density 1e-10, outflow boundaries, 10 FP64 fields, gamma = 5/3.  One
benchmark step is one full SSP-RK3 time step: three hydro stages (ghost fill,
step, update) plus the CFL time step from the first stage's amax, all through
the C ABI on the device.  The headline runs it in mixed precision as the
fused step (hydro_rk3_step with the descriptor's fused flag: one persistent
launch per time step); the same step as separate launches, the plain FP64
form and the forms with the learned indicator are reported beside it, and
the accuracy of the forms (L1 density error after 100 steps) with them.
Extras: the Sedov blast on 512 sub-grids (64^3, the pure-hydro problem of
Sec. IV-A), the adaptive Sedov-shell mesh (~4,096 leaves at levels 3-6) and
contact steepening.
value = cells x time steps / s (the paper's "cells processed per second").

--impl reference times the FP64 CPU oracle on the host cores instead (on a
bounded sample of the same workload: the central 4x4x4 sub-grids), in a
process of its own; the cpu_baseline leg of the GPU arm runs the same
timing in a child process of the same kind.
Multi-GPU (torchrun): every rank runs an independent replica of the workload
(the step has no cross-GPU exchange in this build); value sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hydro cell-updates/s on 1 GB300: plain FP64 vs batched/mixed at fixed L1 err"
UNIT = "cell-updates/s (cells x RK3 time steps / s)"
GAMMA = 5.0 / 3.0
N = 8
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (an FMA counts as two flops)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 80.5: SMs x FP32 lanes x FMA x max clock
# FP32 FFMA throughput measured on this GPU by a probe kernel (3.48e13 FFMA/s)
FP32_PROBE_TFLOPS = 69.6

# Workloads (uniform octree levels of nb^3 sub-grids of 8^3 on [-1,1]^3).
WORKLOADS = {
    "polytrope": {"nb": 32, "omega": 0.2,
                  "desc": "rotating n=1.5 polytrope, 32,768 sub-grids of 8^3 (256^3 on [-1,1]^3), static gravity "
                          "field input, rotating frame omega=0.2, ambient rho 1e-10, outflow, 10 FP64 fields, "
                          "one step = one full RK3 time step (3 stages)"},
    "polytrope128": {"nb": 16, "omega": 0.2,
                     "desc": "rotating n=1.5 polytrope cut at 128^3: 4,096 sub-grids of 8^3 on [-1,1]^3 (h = 1/64), "
                             "static gravity field input, rotating frame omega=0.2, ambient rho 1e-10, outflow; the "
                             "headline's workload at an eighth of its size, for profiler captures"},
    "sedov": {"nb": 8, "omega": 0.0,
              "desc": "Sedov blast, uniform octree level of 512 sub-grids of 8^3 (64^3 on [-1,1]^3), outflow, "
                      "10 FP64 fields, one step = one full RK3 time step (3 stages)"},
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


def max_over_ranks(values: dict, device=None) -> dict:
    """Each timing's largest value over the ranks of the job (the slowest
    rank sets the job's time); unchanged for a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dict(values)
    keys = sorted(values)
    t = torch.tensor([float(values[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return dict(zip(keys, t.tolist()))


def job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return units_per_rank * world_size / seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms around the
    timed work (the sampler's first sample is in before the work starts)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = len(self.lines)  # samples taken before the work
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.thread.join(timeout=5)
            self.out = "".join(self.lines[max(self.skip - 1, 0):])

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Algorithmic work of one hydro_step launch per sub-grid, as counted by the
# oracle's operation-counting scalar (``python -m oracle.count_work``; a CPU
# test keeps these constants equal to that count): unique PPM line
# evaluations (13 lines per interior cell, 9 per face-adjacent ghost cell,
# 10 fields) at the average cost per evaluation on random discontinuous data,
# 15,552 point fluxes, face sums, divergence and sources.  Bytes: the padded
# state read once and dU/dt written once.
ALGO = {"fp64_flops_per_subgrid_stage": 6565962.0, "bytes_per_subgrid_stage": 260520}
# DRAM bytes per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# by form and workload: the hydro_step launch of each precision form, and the
# fused RK3 step (three stages per launch).  Captures on the 256^3 polytrope
# are taken on its 128^3 cut (4,096 sub-grids) and scaled by 8 (traffic
# grows with the sub-grids processed).  None until captured for the current
# kernel.
# Sedov: the mean over the 42 (fused: 14) launches of one ncu launch list of
# `--workload sedov --precision both --steps 3 --warmup 3`; polytrope: one
# full capture at 128^3.
TRAFFIC_PER_LAUNCH = {"fp64_sedov": 1503850831.0 + 1085510120.0, "mixed_sedov": 142870894.0 + 93039927.0,
                      "fused_sedov": 342275310.0 + 444961573.0,
                      "fp64_polytrope": None, "mixed_polytrope": None,
                      "fused_polytrope": 8 * (3430653e3 + 3719836e3)}


def algorithmic_work():
    return dict(ALGO, dram_bytes_per_launch_scaled=TRAFFIC_PER_LAUNCH)


_HOST_STATES = {}


def host_state(workload: str):
    """Seeded initial interiors, gravity, origins and h of a workload (cached)."""
    from paper_2107_10987_gb300 import workloads as W
    if workload not in _HOST_STATES:
        nb = WORKLOADS[workload]["nb"]
        if workload.startswith("polytrope"):
            Ui, g, o, h, _ = W.rotating_polytrope(nb, GAMMA)
        else:
            Ug, h, lo = W.sedov_box(nb * N, GAMMA)
            Ui, g = W.box_to_subgrids(Ug, N), None
            o, hh = W.uniform_mesh(nb, N)
            assert abs(hh - h) < 1e-15
        _HOST_STATES[workload] = (Ui, g, o, h)
    return _HOST_STATES[workload]


def make_state(dev, H, workload: str):
    """Device state of a workload: ghost-padded sub-grids (interiors set, ghost
    layers left to the first ghost fill), origins, cell widths, gravity."""
    import torch
    wl = WORKLOADS[workload]
    nb = wl["nb"]
    Ui, g, o, h = host_state(workload)
    n = nb ** 3
    U = torch.zeros((n, 10, N + 6, N + 6, N + 6), dtype=torch.float64, device=dev)
    origin = torch.tensor(o, device=dev)
    hv = torch.full((n,), h, dtype=torch.float64, device=dev)
    gt = torch.tensor(g, device=dev) if g is not None else None
    ctx = H.Context(GAMMA, wl["omega"])
    H.hydro_scatter_interior(ctx, H.make_batch(U, origin, hv), torch.tensor(Ui, device=dev))
    torch.cuda.synchronize()
    ctx.close()
    return {"U": U, "origin": origin, "h": hv, "g": gt, "nb": nb, "n": n, "cells": n * N ** 3,
            "omega": wl["omega"], "hval": h}


def train_indicator(dev):
    """Train the learned smoothness indicator from seeded runs (Sedov blasts at
    random energy and centre, Sod planes at random orientation; none of them
    the benchmark's own problem) on the GPU's own kernels; threshold for
    99.99% recall of limiter-active cells.  Outside the timed region."""
    from paper_2107_10987_gb300 import gate as GT
    t0 = time.perf_counter()
    # 16 runs on 64^3 meshes, 3 snapshots each: 12.6M labelled cells
    X, y, ch = GT.collect(range(0, 16), n=64, snapshots=(6, 16, 30), device=dev)
    params, hist = GT.train(X, y, iters=2000, batch=16384, lr=3e-3)
    thr = GT.choose_threshold(params, X, y, ch, recall=0.9999)
    Xh, yh, chh = GT.collect(range(1000, 1004), n=64, snapshots=(6, 16, 30), device=dev)
    ev = GT.evaluate(params, thr, Xh, yh, chh)
    ev["train_s"] = time.perf_counter() - t0
    ev["final_loss"] = hist[-1][1]
    return params, thr, ev


def run_form(args, H, dev, precision, flush, indicator=None, fused=False, contact=False, workload="polytrope", spin=False,
             steps=None, state=None):
    """Warm-up, then `steps` timed RK3 steps of one precision form on a
    workload; returns timings and the final density.  Separate launches: the
    sequence hydro_rk3_step enqueues (per stage ghost fill, hydro_step,
    hydro_update; the first stage writes the second state buffer, so no copy
    of the step's initial state is made), issued entry point by entry point
    so that the step kernel can be timed alone.  fused: hydro_rk3_step with
    the descriptor's fused flag (one persistent launch per time step, mixed
    precision).  contact: PPM contact steepening on (hydro_mode_t.contact).
    spin: the spin feedback on (hydro_mode_t.spin).
    state: a make_state() result to start from (it is advanced in place)."""
    import torch
    steps = args.steps if steps is None else steps
    stream = torch.cuda.current_stream()
    st = state if state is not None else make_state(dev, H, workload)
    nb, n, cells = st["nb"], st["n"], st["cells"]
    ctx = H.Context(GAMMA, st["omega"])
    H.hydro_set_mode(ctx, precision, 0.4, contact=1 if contact else 0, spin=1 if spin else 0)
    if indicator is not None:
        H.hydro_set_indicator(ctx, indicator[0], indicator[1])
    Ua, origin, hv, g = st["U"], st["origin"], st["h"], st["g"]
    Ub = torch.zeros_like(Ua)
    bufs = [Ua, Ub]
    dU = torch.empty((n, 10, N, N, N), dtype=torch.float64, device=dev)
    am = torch.empty(n, dtype=torch.float64, device=dev)
    dt = torch.empty(1, dtype=torch.float64, device=dev)
    batches = [H.make_batch(Ua, origin, hv, g), H.make_batch(Ub, origin, hv, g)]
    cur = [0]
    fdesc = H.make_rk3_desc(Ua, Ub, origin, hv, (nb, nb, nb), H.HYDRO_BC_OUTFLOW, dU, am, dt, 0.4, g=g, fused=True)

    def rk3_step(step_events=None):
        x = cur[0]
        if fused:
            if step_events is not None:
                step_events[0][0].record(stream)
            H.hydro_rk3_step(ctx, fdesc, x)
            if step_events is not None:
                step_events[0][1].record(stream)
            cur[0] = 1 - x
            return
        X, Y = batches[x], batches[1 - x]
        for k in range(3):
            B = X if k == 0 else Y
            H.hydro_fill_ghosts_uniform(ctx, B, nb, nb, nb, H.HYDRO_BC_OUTFLOW)
            if step_events is not None:
                step_events[k][0].record(stream)
            H.hydro_step(ctx, B, 0.0, dU, am)
            if step_events is not None:
                step_events[k][1].record(stream)
            if k == 0:
                H.hydro_dt(ctx, am, hv, n, 0.4, dt)
            H.hydro_update(ctx, B, bufs[x], dU, dt_dev=dt, stage=k, U_out=bufs[1 - x] if k == 0 else None)
        cur[0] = 1 - x

    for _ in range(args.warmup):
        rk3_step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(1 if fused else 3)]
           for _ in range(steps)]
    for i in range(steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        rk3_step(kev[i])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    out = {"t_dev": sum(a.elapsed_time(b) for a, b in ev) / 1e3,
           "kern_s": float(np.mean([a.elapsed_time(b) for st_ in kev for a, b in st_])) / 1e3,
           "status": H.hydro_status(ctx), "n": n, "cells": cells, "steps": steps}
    rho_now = lambda: bufs[cur[0]][:, 0, 3:-3, 3:-3, 3:-3].clone()  # noqa: E731
    out["rho"] = rho_now()

    # the same step replayed as a captured CUDA graph (continuing the run)
    desc = H.make_rk3_desc(bufs[cur[0]], bufs[1 - cur[0]], origin, hv, (nb, nb, nb), H.HYDRO_BC_OUTFLOW, dU, am, dt,
                           0.4, g=g, fused=fused)
    graph = H.hydro_rk3_graph_create(ctx, desc)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        gev[i][0].record(stream)
        H.hydro_rk3_graph_launch(graph)
        gev[i][1].record(stream)
    torch.cuda.synchronize()
    out["t_graph"] = sum(a.elapsed_time(b) for a, b in gev) / 1e3
    if H.hydro_rk3_graph_state(graph) == 1:  # the state now lives in the descriptor's second buffer
        cur[0] = 1 - cur[0]
    H.hydro_rk3_graph_destroy(graph)

    # end to end, with the state living on the host: every step moves it in
    # from pinned memory (the N^3 interiors of every sub-grid, the evolved
    # variables), runs one RK3 step and moves the new state out, which is the
    # next step's input.  The library's scatter and gather kernels read and
    # write the pinned host buffers directly over the host link (no staging
    # copy).  The run continues from the evolved state of the timed steps.
    dev_I = torch.empty((n, 10, N, N, N), dtype=torch.float64, device=dev)
    H.hydro_gather_interior(ctx, batches[cur[0]], dev_I)
    host_I = [dev_I.cpu().pin_memory(), torch.empty(dev_I.shape, dtype=torch.float64).pin_memory()]
    del dev_I
    hio = [0]

    def e2e_step():
        H.hydro_scatter_interior(ctx, batches[cur[0]], host_I[hio[0]])
        rk3_step()
        H.hydro_gather_interior(ctx, batches[cur[0]], host_I[1 - hio[0]])
        hio[0] ^= 1

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    out["t_e2e"] = e0.elapsed_time(e1) / 1e3
    out["bytes_step"] = host_I[0].numel() * 8
    if cur[0] == 1:  # leave the state in the caller's buffer
        Ua.copy_(Ub)
    del host_I, Ub, bufs, batches
    ctx.close()
    torch.cuda.empty_cache()
    return out


def amr_measure(args, H, dev, flush, precision, steps, indicator=None):
    """The batched adaptive configuration: ~4,096 leaves at levels 3-6 around a
    blast shell, leaf order shuffled.  Times one RK3 step (direct launches and
    graph replay) and the step kernel alone as one persistent launch over all
    levels (default grid, then the autotuned grid) against one launch per
    level on a level-sorted copy."""
    import torch
    from paper_2107_10987_gb300 import workloads as W
    from paper_2107_10987_gb300.amr import AMRRun
    lev, ijk, theta = W.amr_shell_mesh()
    U = W.amr_shell_state(lev, ijk, GAMMA)
    cells = len(lev) * 512
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, precision, 0.4)
    if indicator is not None:
        H.hydro_set_indicator(ctx, indicator[0], indicator[1])
    stream = torch.cuda.current_stream()
    out = {"leaves": len(lev), "cells": cells, "levels": {int(l): int((lev == l).sum()) for l in np.unique(lev)}}

    def timed(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for i in range(n):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    run = AMRRun(ctx, U, lev, ijk)
    for _ in range(2):
        run.step()
    out["rk3_step_ms_direct"] = timed(run.step, steps)
    grun = AMRRun(ctx, U, lev, ijk)
    grun.step(use_graph=True)
    grun.step(use_graph=True)
    out["rk3_step_ms_graph"] = timed(lambda: grun.step(use_graph=True), steps)
    grun.close()
    out["value_graph"] = cells / (out["rk3_step_ms_graph"] / 1e3)
    # the step kernel alone on the current state
    B = H.make_batch(run.U, run.origin, run.h)
    H.hydro_fill_ghosts_amr(ctx, B, run.mesh)
    dU, am = torch.empty_like(run.dU), torch.empty_like(run.am)
    H.hydro_step(ctx, B, 0.0, dU, am)
    out["step_ms_one_launch"] = timed(lambda: H.hydro_step(ctx, B, 0.0, dU, am), steps)
    order = torch.tensor(np.argsort(lev, kind="stable"), device=dev)
    Us, os_, hs = run.U[order].contiguous(), run.origin[order].contiguous(), run.h[order].contiguous()
    lv = np.sort(lev)
    batches = []
    start = 0
    for l in np.unique(lv):
        cnt = int((lv == l).sum())
        batches.append((H.make_batch(Us[start:start + cnt], os_[start:start + cnt], hs[start:start + cnt]),
                        dU[start:start + cnt], am[start:start + cnt]))
        start += cnt

    def per_level():
        for Bl, d, a in batches:
            H.hydro_step(ctx, Bl, 0.0, d, a)

    per_level()
    out["step_ms_per_level_launches"] = timed(per_level, steps)
    out["autotuned_slots"] = H.hydro_autotune_step(ctx, B, dU, am)
    out["step_ms_one_launch_autotuned"] = timed(lambda: H.hydro_step(ctx, B, 0.0, dU, am), steps)
    out["status"] = H.hydro_status(ctx)
    run.close()
    ctx.close()
    return out


def contact_measure(args, H, dev, flush, res):
    """PPM contact steepening (hydro_mode_t.contact = 1) on the Sedov mesh of
    512 sub-grids: the mixed and the FP64 RK3 step as separate launches (so
    that the step kernel is timed alone), each beside the same form without
    steepening (res: sedov_mixed_separate, sedov_fp64) when that was
    measured.  Values are this GPU's (the block runs on rank 0)."""
    out = {"workload": WORKLOADS["sedov"]["desc"],
           "note": "separate launches (ghost fill, hydro_step, hydro_update per stage; dt); the step kernel "
                   "steepens the density and species lines"}
    for name, prec, plain in (("mixed", H.HYDRO_PREC_MIXED, "mixed_separate"), ("fp64", H.HYDRO_PREC_FP64, "fp64")):
        r = run_form(args, H, dev, prec, flush, contact=True, workload="sedov")
        cells = r["cells"]
        ent = {"value": cells * r["steps"] / r["t_dev"], "ms_per_step": 1e3 * r["t_dev"] / r["steps"],
               "graph_replay": cells * r["steps"] / r["t_graph"], "kernel_ms": 1e3 * r["kern_s"],
               "device_status": r["status"]}
        if plain in res:
            p = res[plain]
            ent["step_cost_vs_unsteepened"] = (r["t_dev"] / r["steps"]) / (p["t_dev"] / p["steps"])
            ent["kernel_cost_vs_unsteepened"] = r["kern_s"] / p["kern_s"]
            if p["steps"] == r["steps"]:
                ent["max_rel_density_diff_vs_unsteepened"] = ((r["rho"] - p["rho"]).abs().max().item() /
                                                              p["rho"].abs().max().item())
        out[name] = ent
    return out


def spin_measure(args, H, dev, flush, res):
    """The spin feedback (hydro_mode_t.spin = 1) on the Sedov mesh of 512
    sub-grids: the fused mixed step, the mixed step as separate launches and
    the FP64 step, each beside the same form without it (res) when that was
    measured.  The spin starts at zero and grows from the torques of the face
    fluxes as the blast expands."""
    out = {"workload": WORKLOADS["sedov"]["desc"],
           "note": "each cell's spin fed back into the velocity at its quadrature points (rigid-rotation "
                   "reading); the spin starts at zero and builds up from the face torques"}
    for name, prec, fused in (("mixed", H.HYDRO_PREC_MIXED, True), ("mixed_separate", H.HYDRO_PREC_MIXED, False),
                              ("fp64", H.HYDRO_PREC_FP64, False)):
        r = run_form(args, H, dev, prec, flush, fused=fused, spin=True, workload="sedov")
        cells = r["cells"]
        ent = {"value": cells * r["steps"] / r["t_dev"], "ms_per_step": 1e3 * r["t_dev"] / r["steps"],
               "kernel_ms": 1e3 * r["kern_s"], "device_status": r["status"]}
        if name in res:
            p = res[name]
            ent["step_cost_vs_without"] = (r["t_dev"] / r["steps"]) / (p["t_dev"] / p["steps"])
            if p["steps"] == r["steps"]:
                ent["max_rel_density_diff_vs_without"] = ((r["rho"] - p["rho"]).abs().max().item() /
                                                          p["rho"].abs().max().item())
        out[name] = ent
    return out


def sedov_measure(args, H, dev, flush):
    """The Sedov blast on 512 sub-grids (64^3, the pure-hydro problem of Sec.
    IV-A at the 8^3 sub-grid size): the fused mixed step, the mixed step as
    separate launches and the plain FP64 step."""
    res = {}
    out = {"workload": WORKLOADS["sedov"]["desc"]}
    for name, prec, fused in (("mixed", H.HYDRO_PREC_MIXED, True), ("mixed_separate", H.HYDRO_PREC_MIXED, False),
                              ("fp64", H.HYDRO_PREC_FP64, False)):
        r = run_form(args, H, dev, prec, flush, fused=fused, workload="sedov")
        res[name] = r
        cells = r["cells"]
        out[name] = {"value": cells * r["steps"] / r["t_dev"], "ms_per_step": 1e3 * r["t_dev"] / r["steps"],
                     "graph_replay": cells * r["steps"] / r["t_graph"],
                     "e2e": cells * r["steps"] / r["t_e2e"], "kernel_ms": 1e3 * r["kern_s"],
                     "device_status": r["status"]}
    out["speedup_mixed_vs_fp64"] = (res["fp64"]["t_dev"] / res["fp64"]["steps"]) / \
        (res["mixed"]["t_dev"] / res["mixed"]["steps"])
    return out, res


def polytrope_measure(args, H, dev, flush, indicator=None):
    """Beside the headline on the rotating polytrope: the old hydro module
    (fluxes at the face centres only, Sec. III-B; the paper compares the new
    module with it on a rotating star, Sec. VI) timed on the same 32,768
    sub-grids in both precisions (graph replay); then every form runs
    --polytrope-steps steps on --polytrope-nb^3 sub-grids from the same
    initial state, and each reports the L1 density error against that state,
    the drift of the total angular momentum about z and of the mass.  With an
    indicator, the forms with the learned smoothness indicator ("gated",
    "fp64_gated") run beside them."""
    import torch
    from paper_2107_10987_gb300 import workloads as W
    from paper_2107_10987_gb300.uniform import UniformRun
    stream = torch.cuda.current_stream()
    omega = WORKLOADS["polytrope"]["omega"]
    forms = (("mixed", H.HYDRO_PREC_MIXED), ("fp64", H.HYDRO_PREC_FP64))
    if indicator is not None:
        forms = forms + (("gated", H.HYDRO_PREC_MIXED), ("fp64_gated", H.HYDRO_PREC_FP64))
    forms = forms + (("mixed_old", H.HYDRO_PREC_MIXED), ("fp64_old", H.HYDRO_PREC_FP64))

    def context(name, prec):
        c = H.Context(GAMMA, omega)
        H.hydro_set_mode(c, prec, 0.4, flux_points=1 if name.endswith("_old") else 9)
        if name in ("gated", "fp64_gated"):
            H.hydro_set_indicator(c, indicator[0], indicator[1])
        return c

    out = {"workload": WORKLOADS["polytrope"]["desc"], "omega": omega}

    def timed(run, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for i in range(n):
            flush.zero_()
            ev[i][0].record(stream)
            run.step(use_graph=True)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev])) / 1e3

    nb = WORKLOADS["polytrope"]["nb"]
    Ui, g, o, h = host_state("polytrope")
    cells = Ui.shape[0] * 512
    for name, prec in (("mixed_old", H.HYDRO_PREC_MIXED), ("fp64_old", H.HYDRO_PREC_FP64)):
        ctx = context(name, prec)
        run = UniformRun(ctx, Ui, o, h, nb, H.HYDRO_BC_OUTFLOW, g, fused=not name.startswith("fp64"))
        steps = max(2, args.steps // 10) if name.startswith("fp64") else args.steps
        for _ in range(2):
            run.step(use_graph=True)
        t = timed(run, steps)
        out[name] = {"value": cells / t, "ms_per_step": 1e3 * t, "steps_timed": steps,
                     "status": H.hydro_status(ctx)}
        run.close()
        del run
        ctx.close()
        torch.cuda.empty_cache()

    nb = args.polytrope_nb
    Ui, g, o, h, _ = W.rotating_polytrope(nb, GAMMA)
    rho_ic = Ui[:, 0]
    acc = {"sub_grids": nb ** 3, "cells": nb ** 3 * 512, "steps": args.polytrope_steps}
    for name, prec in forms:
        ctx = context(name, prec)
        run = UniformRun(ctx, Ui, o, h, nb, H.HYDRO_BC_OUTFLOW, g, fused=not name.startswith("fp64"))
        c0 = run.sums()
        t = 0.0
        for _ in range(args.polytrope_steps):
            run.step(use_graph=True)
            t += run.last_dt()
        c1 = run.sums()
        rho = run.interior()[:, 0].cpu().numpy()
        acc[name] = {"t": t, "l1_density": W.density_l1(rho, rho_ic, h),
                     "angular_momentum_drift": float((c1[10] - c0[10]) / c0[10]),
                     "mass_drift": float((c1[0] - c0[0]) / c0[0]), "status": H.hydro_status(ctx)}
        run.close()
        del run
        ctx.close()
        torch.cuda.empty_cache()
    acc["l1_mixed_over_fp64"] = acc["mixed"]["l1_density"] / acc["fp64"]["l1_density"]
    # the paper's comparison: the old module's error over the new one's
    acc["l1_old_over_new_fp64"] = acc["fp64_old"]["l1_density"] / acc["fp64"]["l1_density"]
    acc["l1_old_over_new_mixed"] = acc["mixed_old"]["l1_density"] / acc["mixed"]["l1_density"]
    if indicator is not None:
        acc["l1_gated_over_fp64"] = acc["gated"]["l1_density"] / acc["fp64"]["l1_density"]
        acc["l1_fp64_gated_over_fp64"] = acc["fp64_gated"]["l1_density"] / acc["fp64"]["l1_density"]
    out["accuracy"] = acc
    return out


def subgrid16_measure(args, H, dev, flush):
    """The headline's rotating polytrope at 256^3 cut into 4,096 sub-grids of
    16^3 (the paper's best-performing sub-grid size, Sec. V), replayed from a
    CUDA graph: the mixed RK3 step fused into one launch (each octant of a
    sub-grid a work unit) and as separate launches, and plain FP64 (the step
    kernels run the octants of each sub-grid in place)."""
    import torch
    from paper_2107_10987_gb300 import workloads as W
    from paper_2107_10987_gb300.uniform import UniformRun
    stream = torch.cuda.current_stream()
    omega = WORKLOADS["polytrope"]["omega"]
    nb = 16
    Ui, g, o, h, _ = W.rotating_polytrope(nb, GAMMA, N=16)
    cells = Ui.shape[0] * 16 ** 3
    out = {"workload": "rotating n=1.5 polytrope, 4,096 sub-grids of 16^3 (256^3 on [-1,1]^3), as the headline"}
    for name, prec, fused in (("mixed", H.HYDRO_PREC_MIXED, True), ("mixed_separate", H.HYDRO_PREC_MIXED, False),
                              ("fp64", H.HYDRO_PREC_FP64, False)):
        ctx = H.Context(GAMMA, omega, N=16)
        H.hydro_set_mode(ctx, prec, 0.4)
        run = UniformRun(ctx, Ui, o, h, nb, H.HYDRO_BC_OUTFLOW, g, fused=fused)
        steps = max(2, args.steps // 10) if name == "fp64" else args.steps
        for _ in range(2):
            run.step(use_graph=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            run.step(use_graph=True)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        t = float(np.mean([a.elapsed_time(b) for a, b in ev])) / 1e3
        out[name] = {"value": cells / t, "ms_per_step": 1e3 * t, "steps_timed": steps, "status": H.hydro_status(ctx)}
        run.close()
        del run
        ctx.close()
        torch.cuda.empty_cache()
    return out


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    from paper_2107_10987_gb300 import hydro as H

    ws, rk, lr = dist_env()
    dev = torch.device("cuda", lr)
    torch.cuda.set_device(dev)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    # precision and launch form of each measured form; the headline is last.
    # The FP64 forms take ~2 s per step on the full mesh: they time fewer steps.
    forms = {"fp64": (H.HYDRO_PREC_FP64, False), "fp64_gated": (H.HYDRO_PREC_FP64, False),
             "gated": (H.HYDRO_PREC_MIXED, True), "mixed_separate": (H.HYDRO_PREC_MIXED, False),
             "mixed": (H.HYDRO_PREC_MIXED, True)}
    order = {"all": ["fp64", "fp64_gated", "gated", "mixed_separate", "mixed"],
             "both": ["fp64", "mixed_separate", "mixed"]}.get(args.precision, [args.precision])
    wl = args.workload
    fp64_steps = max(2, args.steps // 10) if wl == "polytrope" else args.steps
    indicator = ind_eval = None
    if "gated" in order or "fp64_gated" in order:
        params, thr, ind_eval = train_indicator(dev)
        indicator = (params, thr)
    res = {}
    for name in order:
        if ws > 1:
            dist.barrier()
        ind = indicator if name in ("gated", "fp64_gated") else None
        prec, fused = forms[name]
        steps = fp64_steps if name.startswith("fp64") else args.steps
        if name == order[-1]:
            with ClockSampler(lr) as clk:
                t0 = time.perf_counter()
                res[name] = run_form(args, H, dev, prec, flush, ind, fused, workload=wl, steps=steps)
                res[name]["wall"] = time.perf_counter() - t0
            res[name]["clocks"] = clk.summary()
        else:
            res[name] = run_form(args, H, dev, prec, flush, ind, fused, workload=wl, steps=steps)
        res[name].update(max_over_ranks({k: res[name][k] for k in ("t_dev", "t_e2e", "t_graph")}, dev))

    if rk == 0:
        work = algorithmic_work()
        pk = peaks()
        head = order[-1]
        r = res[head]
        n, cells, K = r["n"], r["cells"], r["steps"]

        def rate(x, key="t_dev"):
            return job_rate(cells * x["steps"], ws, x[key])

        def per_step_ms(x, key="t_dev"):
            return 1e3 * x[key] / x["steps"]

        head_fused = forms[head][1]
        flops = work["fp64_flops_per_subgrid_stage"] * n  # one stage of the mesh
        bytes_launch = work["bytes_per_subgrid_stage"] * n
        # the timed kernel: the fused step does three stages per launch and
        # reads the state once and writes the new state once (interiors)
        k_flops = 3 * flops if head_fused else flops
        k_bytes = 2 * n * 10 * N ** 3 * 8 if head_fused else bytes_launch
        k_name = "hydro_rk3_fused_kernel (one launch per RK3 step)" if head_fused else f"hydro_step_{head} (avg launch)"
        peak = FP64_PEAK_TFLOPS if head.startswith("fp64") else FP32_PEAK_TFLOPS
        achieved = k_flops / r["kern_s"] / 1e12
        traffic_key = ("fused" if head_fused else ("fp64" if head.startswith("fp64") else "mixed")) + "_" + wl
        line = {
            "metric": METRIC, "value": rate(r), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_ms(r),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head.startswith("fp64") else "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl]["desc"], "sub_grids": n, "cells": cells,
                       "precision": "mixed: FP32 reconstruction/fluxes, FP64 dual-energy recovery, accumulation "
                                    "and update" if not head.startswith("fp64") else "fp64 (plain)",
                       "launch": ("fused: one persistent launch per RK3 step" if head_fused
                                  else "separate: ten launches per RK3 step"),
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed (256 MB write) between timed steps, outside the timed events; the padded "
                             "state (7.2 GB at 256^3) is larger than L2 anyway"},
            "cell_stage_updates_per_s": 3 * rate(r),
            "graph_replay": {"value": rate(r, "t_graph"), "ms_per_step": per_step_ms(r, "t_graph"),
                             "note": "the same RK3 step captured once into a CUDA graph (hydro_rk3_graph_*)"},
            "wall_s_timed_region": r["wall"],
            "kernel_ms": {k_name: 1e3 * r["kern_s"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": work.get("dram_bytes_per_launch_scaled", {}).get(traffic_key),
                         "peak_source": ("FP32: 152 SMs x 128 lanes x 2 flops x 2070 MHz (profiling recipe units)"
                                         if not head.startswith("fp64") else "nominal GB300 FP64 from the profiling "
                                                                             "recipe"),
                         "flops_counted": "algorithmic ops of the method (oracle count), each op one flop",
                         "hbm_frac": (k_bytes / r["kern_s"] / 1e9) / pk["hbm_gbs"] if "hbm_gbs" in pk else None},
            "e2e": {"value": rate(r, "t_e2e"), "unit": UNIT,
                    "h2d_bytes_per_step": r["bytes_step"], "d2h_bytes_per_step": r["bytes_step"]},
            "gpu_launches": (1 if head_fused else 10) * K,
            "clocks": r["clocks"],
            "device_status": r["status"],
        }
        if not head.startswith("fp64"):
            line["roofline"]["peak_measured_fp32_probe"] = FP32_PROBE_TFLOPS
            line["roofline"]["frac_of_measured_fp32_probe"] = achieved / FP32_PROBE_TFLOPS
        if "mixed_separate" in res and head != "mixed_separate":
            m = res["mixed_separate"]
            am = flops / m["kern_s"] / 1e12
            line["separate_launches"] = {
                "note": "the same mixed RK3 step as ten launches (per stage ghost fill, hydro_step, hydro_update; "
                        "dt), hydro_rk3_step without the fused flag",
                "value": rate(m), "ms_per_step": per_step_ms(m), "graph_replay": rate(m, "t_graph"),
                "e2e": rate(m, "t_e2e"),
                "kernel_ms": {"hydro_step_mixed (avg launch)": 1e3 * m["kern_s"]},
                "roofline": {"bound": "alu", "achieved": am, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": am / FP32_PEAK_TFLOPS,
                             "traffic": work.get("dram_bytes_per_launch_scaled", {}).get("mixed_" + wl)},
                "max_rel_density_diff_vs_fused": (m["rho"] - r["rho"]).abs().max().item() / r["rho"].abs().max().item()
                if m["steps"] == r["steps"] else None}
        if "fp64" in res and head != "fp64":
            f = res["fp64"]
            a64 = flops / f["kern_s"] / 1e12
            line["plain_fp64"] = {
                "value": rate(f), "ms_per_step": per_step_ms(f), "steps_timed": f["steps"],
                "kernel_ms": 1e3 * f["kern_s"], "e2e": rate(f, "t_e2e"), "graph_replay": rate(f, "t_graph"),
                "roofline": {"bound": "alu", "achieved": a64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a64 / FP64_PEAK_TFLOPS,
                             "traffic": work.get("dram_bytes_per_launch_scaled", {}).get("fp64_" + wl)}}
            line["speedup_vs_plain_fp64"] = per_step_ms(f) / per_step_ms(r)
        if "fp64_gated" in res and "fp64" in res:
            fg, f = res["fp64_gated"], res["fp64"]
            line["plain_fp64_with_indicator"] = {
                "value": rate(fg), "ms_per_step": per_step_ms(fg), "kernel_ms": 1e3 * fg["kern_s"],
                "speedup_vs_plain_fp64": per_step_ms(f) / per_step_ms(fg)}
        if "gated" in res:
            gr = res["gated"]
            line["mixed_with_indicator"] = {
                "value": rate(gr), "ms_per_step": per_step_ms(gr), "kernel_ms": 1e3 * gr["kern_s"],
                "speedup_vs_mixed": per_step_ms(r) / per_step_ms(gr) if head == "mixed" else None,
                "indicator_held_out": ind_eval}
            if wl == "polytrope":
                line["mixed_with_indicator"]["note"] = (
                    "off by design on this workload: by the method's own labels the limiter acts on ~99.8 % of "
                    "its cells (the thin infalling ambient gas carries oscillations above the label threshold), so "
                    "the indicator finds nothing to skip and its evaluation is pure cost; it pays on the Sedov mesh, "
                    "where ~98 % of cells sit in uniform neighbourhoods")
        if args.polytrope and wl == "polytrope":
            line["rotating_polytrope"] = polytrope_measure(args, H, dev, flush, indicator)
            acc = line["rotating_polytrope"]["accuracy"]
            line["equal_accuracy"] = {
                "note": f"L1 density error against the initial state after {acc['steps']} RK3 steps on "
                        f"{acc['sub_grids']} sub-grids ({round(acc['cells'] ** (1 / 3))}^3), each form from the same "
                        "state (Sec. VI's measure with an absolute value)",
                "l1_fp64": acc["fp64"]["l1_density"], "l1_mixed": acc["mixed"]["l1_density"],
                "l1_mixed_over_fp64": acc["l1_mixed_over_fp64"]}
        if args.subgrid16 and wl == "polytrope":
            line["subgrid16"] = subgrid16_measure(args, H, dev, flush)
            sg = line["subgrid16"]
            sg["mixed_vs_8cubed_fused"] = line["ms_per_step"] / sg["mixed"]["ms_per_step"] if head_fused else None
            sg["separate_vs_8cubed_separate"] = (
                line["separate_launches"]["ms_per_step"] / sg["mixed_separate"]["ms_per_step"]
                if "separate_launches" in line else None)
        if args.sedov:
            line["sedov_512"], sres = sedov_measure(args, H, dev, flush)
        else:
            sres = {}
        if args.amr:
            line["amr_batched"] = {"workload": "adaptive octree, ~4,096 leaves of 8^3 at levels 3-6 refined around a "
                                               "blast shell of radius 0.3, leaf order shuffled (seed 1234; the kernels take the leaves along their Morton curve), outflow",
                                   "mixed": amr_measure(args, H, dev, flush, H.HYDRO_PREC_MIXED, args.steps),
                                   "fp64": amr_measure(args, H, dev, flush, H.HYDRO_PREC_FP64, max(2, args.steps // 5))}
            if indicator is not None:
                line["amr_batched"]["gated"] = amr_measure(args, H, dev, flush, H.HYDRO_PREC_MIXED, args.steps,
                                                           indicator)
                line["amr_batched"]["fp64_gated"] = amr_measure(args, H, dev, flush, H.HYDRO_PREC_FP64,
                                                                max(2, args.steps // 5), indicator)
        if args.contact:
            try:
                line["contact_steepening"] = contact_measure(args, H, dev, flush, sres)
            except Exception as e:  # an optional block: it never costs the headline line
                line["contact_steepening"] = {"error": f"{type(e).__name__}: {e}"}
        if args.spin and args.sedov:  # beside the Sedov forms it is compared with
            try:
                line["spin_feedback"] = spin_measure(args, H, dev, flush, sres)
            except Exception as e:  # an optional block: it never costs the headline line
                line["spin_feedback"] = {"error": f"{type(e).__name__}: {e}"}
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, wl)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def oracle_sample(workload: str):
    """The central 4x4x4 sub-grids of a workload (32^3 cells, same h), with
    their gravity; the sample's own boundary is outflow.  The polytrope's
    sample is generated on its own cell centres by the workload's formulas
    (the same values as in the full mesh, without building the full mesh)."""
    from paper_2107_10987_gb300 import workloads as W
    nb = WORKLOADS[workload]["nb"]
    k0 = nb // 2 - 2
    if workload.startswith("polytrope"):
        o, h = W.uniform_mesh(nb, N)
        lo = tuple(o[(k0 * nb + k0) * nb + k0])
        model = W.polytrope_model(1.5, 0.5)
        x = lo[0] + (np.arange(4 * N) + 0.5) * h
        y = lo[1] + (np.arange(4 * N) + 0.5) * h
        z = lo[2] + (np.arange(4 * N) + 0.5) * h
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        rho, v, p, g = W.polytrope_point(model, X, Y, Z, 0.2, 1e-10)
        Ug = W.conserved_from_primitive(rho, v, p, GAMMA)
        gs = np.ascontiguousarray(W.box_to_subgrids(np.ascontiguousarray(g), N))
        return Ug, gs, h, lo
    Ug, h, lo = W.sedov_box(nb * N, GAMMA)
    c = slice(k0 * N, (k0 + 4) * N)
    return Ug[:, c, c, c].copy(), None, h, (lo[0] + k0 * N * h, lo[1] + k0 * N * h, lo[2] + k0 * N * h)


def oracle_timing(workload: str, steps: int, warmup: int, budget_s: float = 0.0, threads: int = 0) -> dict:
    """The FP64 oracle as it stands, timed on the host cores: `warmup` RK3
    steps, then `steps` timed RK3 steps (or as many as fit in budget_s when it
    is positive) of the workload's central 4x4x4 sub-grids, OpenMP over
    sub-grids on `threads` cores (0: all).  The reference arm and the
    cpu_baseline leg both run this, each in a process of its own that has not
    loaded torch or the GPU library."""
    from oracle import core, mesh
    core.build()
    Ug, g, h, lo = oracle_sample(workload)
    P = core.OracleParams(gamma=GAMMA, omega=WORKLOADS[workload]["omega"])
    run = mesh.BoxRun(P, Ug, h, lo, "outflow", g=g, nthreads=threads)
    for _ in range(warmup):
        run.step(0.4)
    t0 = time.perf_counter()
    n = 0
    while (n < steps) if budget_s <= 0 else (time.perf_counter() - t0 < budget_s or n == 0):
        run.step(0.4)
        n += 1
    dt = time.perf_counter() - t0
    cells = Ug[0].size
    return {"value": cells * n / dt, "steps": n, "seconds": dt, "cells": cells,
            "cores": threads if threads > 0 else os.cpu_count()}


def _oracle_child(workload: str, steps: int, warmup: int, budget_s: float, threads: int) -> dict:
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_timing(%r, %d, %d, %r, %d)))" % (ROOT, workload, steps, warmup,
                                                                          float(budget_s), threads))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True)
    return json.loads(p.stdout.strip().splitlines()[-1])


def cpu_baseline(budget_s: float, workload: str = "polytrope"):
    """The oracle as it stands, on all host cores and on one, on a bounded
    sample of the workload, in child processes (the reference arm's protocol:
    one warm-up step, then RK3 steps for about budget_s seconds)."""
    r = _oracle_child(workload, 0, 1, budget_s, 0)
    out = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
           "sample": f"{r['steps']} RK3 steps of the central 4x4x4 sub-grids ({r['cells']} cells) of the workload, "
                     f"{r['seconds']:.1f} s, OpenMP over sub-grids on all host cores, in a child process without "
                     f"torch (the reference arm's protocol)"}
    r1 = _oracle_child(workload, 0, 1, budget_s / 4, 1)
    out["single_core"] = {"value": r1["value"], "unit": UNIT, "cores": 1,
                          "sample": f"{r1['steps']} RK3 steps of the same sample, {r1['seconds']:.1f} s"}
    return out


def reference_arm(args):
    ws, rk, lr = dist_env()
    if rk != 0:
        return
    r = oracle_timing(args.workload, args.steps, args.warmup)
    v = r["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / r["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"] + "; oracle sample: its central 4x4x4 "
                                   "sub-grids (32^3 cells, same h), outflow at the sample's boundary",
                       "cells": r["cells"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": f"{r['steps']} RK3 steps of 32^3 cells on all host cores"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-amr", dest="amr", action="store_false", help="skip the batched adaptive-mesh measurement")
    ap.add_argument("--no-polytrope", dest="polytrope", action="store_false",
                    help="skip the rotating-polytrope measurement")
    ap.add_argument("--no-contact", dest="contact", action="store_false",
                    help="skip the contact-steepening measurement")
    ap.add_argument("--no-spin", dest="spin", action="store_false",
                    help="skip the spin-feedback measurement")
    ap.add_argument("--no-sedov", dest="sedov", action="store_false",
                    help="skip the 512-sub-grid Sedov measurement")
    ap.add_argument("--no-subgrid16", dest="subgrid16", action="store_false",
                    help="skip the 16^3-sub-grid measurement")
    ap.add_argument("--workload", default="polytrope", choices=sorted(WORKLOADS),
                    help="the headline workload (polytrope: 32,768 sub-grids; sedov: 512 sub-grids)")
    ap.add_argument("--polytrope-nb", type=int, default=16,
                    help="sub-grids per axis of the polytrope accuracy runs (32: the full 256^3 mesh)")
    ap.add_argument("--polytrope-steps", type=int, default=100)
    ap.add_argument("--precision", default="all",
                    choices=["all", "both", "mixed", "mixed_separate", "fp64", "gated", "fp64_gated"],
                    help="all: time the plain FP64 form, the FP64 and mixed forms with the learned indicator, "
                         "then the mixed form (reported as value); both: FP64 then mixed")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ws, rk, _ = dist_env()
        if rk != 0 or ws > 1:
            args.cpu_baseline = args.cpu_baseline and rk == 0 and ws == 1
        gpu_arm(args)


if __name__ == "__main__":
    main()
