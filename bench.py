"""Benchmark of the hydro hot path on one GB300 (cell-updates/s).

Workload: the Sedov-Taylor blast on a uniform octree level of 512 sub-grids
of 8^3 cells (64^3 cells on [-1,1]^3), outflow boundaries, 10 FP64 fields,
gamma = 5/3 -- the paper's pure-hydro benchmark problem (Sec. IV-A) at the
sub-grid size 8^3.  One benchmark step is one full SSP-RK3 time step: three
hydro stages (ghost fill, step, update) plus the CFL time step from the first
stage's amax, all through the C ABI on the device.  The headline runs it in
mixed precision as the fused step (hydro_rk3_step with the descriptor's
fused flag: one persistent launch per time step); the same step as separate
launches and the plain FP64 form are reported beside it.
value = cells x time steps / s (the paper's "cells processed per second").

--impl reference times the FP64 CPU oracle on the host cores instead (on a
bounded sample of the same workload: the central 4x4x4 sub-grids).
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
NB = 8  # 8^3 sub-grids
N = 8
CELLS = (NB * N) ** 3
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (an FMA counts as two flops)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 80.5: SMs x FP32 lanes x FMA x max clock


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
# DRAM bytes per launch on this workload from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum): the hydro_step launch of each precision form, and
# the fused RK3 step (three stages per launch); None until captured for the
# current kernel.
TRAFFIC_PER_LAUNCH = {"fp64": 204584192.0, "mixed": 254990848.0, "fused": 838170112.0}


def algorithmic_work():
    return dict(ALGO, dram_bytes_per_launch_scaled=TRAFFIC_PER_LAUNCH)


def make_state(dev):
    import torch
    from paper_2107_10987_gb300 import workloads as W
    Ug, h, lo = W.sedov_box(NB * N, GAMMA)
    # ghost-padded sub-grids; the first ghost fill of every stage overwrites the ghosts
    sub = np.zeros((NB ** 3, 10, N + 6, N + 6, N + 6))
    sub[:, :, 3:-3, 3:-3, 3:-3] = W.box_to_subgrids(Ug, N)
    o, hh = W.uniform_mesh(NB, N)
    assert abs(hh - h) < 1e-15
    U = torch.tensor(sub, device=dev)
    origin = torch.tensor(o, device=dev)
    hv = torch.full((NB ** 3,), h, dtype=torch.float64, device=dev)
    return U, origin, hv, sub


def train_indicator(dev):
    """Train the learned smoothness indicator from seeded runs (Sedov blasts at
    random energy and centre, Sod planes at random orientation; none of them
    the benchmark's own problem) on the GPU's own kernels; threshold for
    99.95% recall of limiter-active cells.  Outside the timed region."""
    from paper_2107_10987_gb300 import gate as GT
    t0 = time.perf_counter()
    X, y, ch = GT.collect(range(0, 8), n=32, snapshots=(6, 16, 30), device=dev)
    params, hist = GT.train(X, y, iters=600, batch=16384, lr=3e-3)
    thr = GT.choose_threshold(params, X, y, ch, recall=0.9995)
    Xh, yh, chh = GT.collect(range(1000, 1004), n=32, snapshots=(6, 16, 30), device=dev)
    ev = GT.evaluate(params, thr, Xh, yh, chh)
    ev["train_s"] = time.perf_counter() - t0
    ev["final_loss"] = hist[-1][1]
    return params, thr, ev


def run_form(args, H, dev, precision, flush, indicator=None, fused=False, contact=False):
    """Warm-up, then K timed RK3 steps of one precision form; returns timings
    and the final state.  Separate launches: the sequence hydro_rk3_step
    enqueues (per stage ghost fill, hydro_step, hydro_update; the first stage
    writes the second state buffer, so no copy of the step's initial state is
    made), issued entry point by entry point so that the step kernel can be
    timed alone.  fused: hydro_rk3_step with the descriptor's fused flag (one
    persistent launch per time step, mixed precision).  contact: PPM contact
    steepening on (hydro_mode_t.contact)."""
    import torch
    stream = torch.cuda.current_stream()
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, precision, 0.4, contact=1 if contact else 0)
    if indicator is not None:
        H.hydro_set_indicator(ctx, indicator[0], indicator[1])
    Ua, origin, hv, _ = make_state(dev)
    Ub = torch.zeros_like(Ua)
    bufs = [Ua, Ub]
    n = Ua.shape[0]
    dU = torch.empty((n, 10, N, N, N), dtype=torch.float64, device=dev)
    am = torch.empty(n, dtype=torch.float64, device=dev)
    dt = torch.empty(1, dtype=torch.float64, device=dev)
    batches = [H.make_batch(Ua, origin, hv), H.make_batch(Ub, origin, hv)]
    cur = [0]
    fdesc = H.make_rk3_desc(Ua, Ub, origin, hv, (NB, NB, NB), H.HYDRO_BC_OUTFLOW, dU, am, dt, 0.4, fused=True)

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
            H.hydro_fill_ghosts_uniform(ctx, B, NB, NB, NB, H.HYDRO_BC_OUTFLOW)
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
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(1 if fused else 3)]
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        rk3_step(kev[i])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    out = {"t_dev": sum(a.elapsed_time(b) for a, b in ev) / 1e3,
           "kern_s": float(np.mean([a.elapsed_time(b) for st in kev for a, b in st])) / 1e3,
           "status": H.hydro_status(ctx), "rho": bufs[cur[0]][:, 0, 3:-3, 3:-3, 3:-3].clone(), "n": n}

    # the same step replayed as a captured CUDA graph (continuing the run)
    desc = H.make_rk3_desc(bufs[cur[0]], bufs[1 - cur[0]], origin, hv, (NB, NB, NB), H.HYDRO_BC_OUTFLOW, dU, am, dt,
                           0.4, fused=fused)
    graph = H.hydro_rk3_graph_create(ctx, desc)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
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
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    out["t_e2e"] = e0.elapsed_time(e1) / 1e3
    out["bytes_step"] = dev_I.numel() * 8
    ctx.close()
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
    """PPM contact steepening (hydro_mode_t.contact = 1) on the same Sedov
    mesh: the mixed and the FP64 RK3 step as separate launches (the fused
    step does not steepen), each beside the same form without steepening
    from this run (res: mixed_separate, fp64) when that was measured.
    Values are this GPU's (the block runs on rank 0)."""
    out = {"note": "separate launches (ghost fill, hydro_step, hydro_update per stage; dt); the step kernel "
                   "steepens the density and species lines"}
    for name, prec, plain in (("mixed", H.HYDRO_PREC_MIXED, "mixed_separate"), ("fp64", H.HYDRO_PREC_FP64, "fp64")):
        r = run_form(args, H, dev, prec, flush, contact=True)
        ent = {"value": CELLS * args.steps / r["t_dev"], "ms_per_step": 1e3 * r["t_dev"] / args.steps,
               "graph_replay": CELLS * args.steps / r["t_graph"], "kernel_ms": 1e3 * r["kern_s"],
               "device_status": r["status"]}
        if plain in res:
            p = res[plain]
            ent["step_cost_vs_unsteepened"] = r["t_dev"] / p["t_dev"]
            ent["kernel_cost_vs_unsteepened"] = r["kern_s"] / p["kern_s"]
            ent["max_rel_density_diff_vs_unsteepened"] = ((r["rho"] - p["rho"]).abs().max().item() /
                                                          p["rho"].abs().max().item())
        out[name] = ent
    return out


def polytrope_measure(args, H, dev, flush, indicator=None):
    """The rotating n = 1.5 polytrope (Lane-Emden profile, radius 0.5, rigid
    rotation at 0.2 of the Keplerian rate, rotating frame Omega = 0.2, its
    static gravitational field as an input array, ambient density 1e-10,
    outflow).  Throughput of RK3 steps of both forms (graph replay) on
    32,768 sub-grids (256^3); then both forms run --polytrope-steps steps on
    --polytrope-nb^3 sub-grids from the same initial state, and each reports
    the L1 density error against that state, the drift of the total angular
    momentum about z and of the mass.  With an indicator, the mixed form with
    the learned smoothness indicator ("gated") runs beside them.  The old
    hydro module (fluxes at the face centres only) runs in both precisions
    too: the paper's new-versus-old accuracy comparison."""
    import torch
    from paper_2107_10987_gb300 import workloads as W
    from paper_2107_10987_gb300.uniform import UniformRun
    stream = torch.cuda.current_stream()
    omega = 0.2
    forms = (("mixed", H.HYDRO_PREC_MIXED), ("fp64", H.HYDRO_PREC_FP64))
    if indicator is not None:
        forms = forms + (("gated", H.HYDRO_PREC_MIXED), ("fp64_gated", H.HYDRO_PREC_FP64))
    # the old hydro module (fluxes at the face centres only, Sec. III-B), which
    # the paper compares the new one with on a rotating star (Sec. VI)
    forms = forms + (("mixed_old", H.HYDRO_PREC_MIXED), ("fp64_old", H.HYDRO_PREC_FP64))

    def context(name, prec):
        c = H.Context(GAMMA, omega)
        H.hydro_set_mode(c, prec, 0.4, flux_points=1 if name.endswith("_old") else 9)
        if name in ("gated", "fp64_gated"):
            H.hydro_set_indicator(c, indicator[0], indicator[1])
        return c

    out = {"workload": "rotating n=1.5 polytrope, 32,768 sub-grids of 8^3 (256^3 on [-1,1]^3), static gravity "
                       "field input, rotating frame omega=0.2, ambient rho 1e-10, outflow", "omega": omega}

    def timed(run, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for i in range(n):
            flush.zero_()
            ev[i][0].record(stream)
            run.step(use_graph=True)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev])) / 1e3

    nb = 32
    Ui, g, o, h, _ = W.rotating_polytrope(nb, GAMMA)
    cells = Ui.shape[0] * 512
    for name, prec in forms:
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
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["cost_new_over_old_fp64"] = out["fp64"]["ms_per_step"] / out["fp64_old"]["ms_per_step"]
    out["cost_new_over_old_mixed"] = out["mixed"]["ms_per_step"] / out["mixed_old"]["ms_per_step"]
    if indicator is not None:
        out["speedup_gated_vs_mixed"] = out["mixed"]["ms_per_step"] / out["gated"]["ms_per_step"]
        out["speedup_fp64_gated_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp64_gated"]["ms_per_step"]

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
    # precision and launch form of each measured form; the headline is last
    forms = {"fp64": (H.HYDRO_PREC_FP64, False), "fp64_gated": (H.HYDRO_PREC_FP64, False),
             "gated": (H.HYDRO_PREC_MIXED, True), "mixed_separate": (H.HYDRO_PREC_MIXED, False),
             "mixed": (H.HYDRO_PREC_MIXED, True)}
    order = {"all": ["fp64", "fp64_gated", "gated", "mixed_separate", "mixed"],
             "both": ["fp64", "mixed_separate", "mixed"]}.get(args.precision, [args.precision])
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
        if name == order[-1]:
            with ClockSampler(lr) as clk:
                t0 = time.perf_counter()
                res[name] = run_form(args, H, dev, prec, flush, ind, fused)
                res[name]["wall"] = time.perf_counter() - t0
            res[name]["clocks"] = clk.summary()
        else:
            res[name] = run_form(args, H, dev, prec, flush, ind, fused)
        res[name].update(max_over_ranks({k: res[name][k] for k in ("t_dev", "t_e2e", "t_graph")}, dev))

    if rk == 0:
        work = algorithmic_work()
        pk = peaks()
        head = order[-1]
        r = res[head]
        n = r["n"]
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
        traffic_key = "fused" if head_fused else ("fp64" if head.startswith("fp64") else "mixed")
        line = {
            "metric": METRIC, "value": job_rate(CELLS * args.steps, ws, r["t_dev"]), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["t_dev"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == "fp64" else "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": "Sedov blast, uniform octree level of 512 sub-grids of 8^3 (64^3 on [-1,1]^3), "
                                   "outflow, 10 FP64 fields, one step = one full RK3 time step (3 stages)",
                       "sub_grids": n, "cells": CELLS,
                       "precision": "mixed: FP32 reconstruction/fluxes, FP64 dual-energy recovery, accumulation "
                                    "and update" if head != "fp64" else "fp64 (plain)",
                       "launch": ("fused: one persistent launch per RK3 step" if head_fused
                                  else "separate: ten launches per RK3 step"),
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed (256 MB write) between timed steps, outside the timed events"},
            "cell_stage_updates_per_s": 3 * job_rate(CELLS * args.steps, ws, r["t_dev"]),
            "graph_replay": {"value": job_rate(CELLS * args.steps, ws, r["t_graph"]),
                             "ms_per_step": 1e3 * r["t_graph"] / args.steps,
                             "note": "the same RK3 step captured once into a CUDA graph (hydro_rk3_graph_*)"},
            "wall_s_timed_region": r["wall"],
            "kernel_ms": {k_name: 1e3 * r["kern_s"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": work.get("dram_bytes_per_launch_scaled", {}).get(traffic_key),
                         "peak_source": ("FP32: 152 SMs x 128 lanes x 2 flops x 2070 MHz (profiling recipe units)"
                                         if head != "fp64" else "nominal GB300 FP64 from the profiling recipe"),
                         "flops_counted": "algorithmic ops of the method (oracle count), each op one flop",
                         "hbm_frac": (k_bytes / r["kern_s"] / 1e9) / pk["hbm_gbs"] if "hbm_gbs" in pk else None},
            "e2e": {"value": job_rate(CELLS * args.steps, ws, r["t_e2e"]), "unit": UNIT,
                    "h2d_bytes_per_step": r["bytes_step"], "d2h_bytes_per_step": r["bytes_step"]},
            "gpu_launches": (1 if head_fused else 10) * args.steps,
            "clocks": r["clocks"],
            "device_status": r["status"],
        }
        if "mixed_separate" in res and head != "mixed_separate":
            m = res["mixed_separate"]
            am = flops / m["kern_s"] / 1e12
            line["separate_launches"] = {
                "note": "the same mixed RK3 step as ten launches (per stage ghost fill, hydro_step, hydro_update; "
                        "dt), hydro_rk3_step without the fused flag",
                "value": job_rate(CELLS * args.steps, ws, m["t_dev"]), "ms_per_step": 1e3 * m["t_dev"] / args.steps,
                "graph_replay": job_rate(CELLS * args.steps, ws, m["t_graph"]),
                "e2e": job_rate(CELLS * args.steps, ws, m["t_e2e"]),
                "kernel_ms": {"hydro_step_mixed (avg launch)": 1e3 * m["kern_s"]},
                "roofline": {"bound": "alu", "achieved": am, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": am / FP32_PEAK_TFLOPS,
                             "traffic": work.get("dram_bytes_per_launch_scaled", {}).get("mixed")},
                "max_rel_density_diff_vs_fused": (m["rho"] - r["rho"]).abs().max().item() / r["rho"].abs().max().item()}
        if "fp64" in res and head != "fp64":
            f = res["fp64"]
            a64 = flops / f["kern_s"] / 1e12
            line["plain_fp64"] = {
                "value": job_rate(CELLS * args.steps, ws, f["t_dev"]), "ms_per_step": 1e3 * f["t_dev"] / args.steps,
                "kernel_ms": 1e3 * f["kern_s"], "e2e": job_rate(CELLS * args.steps, ws, f["t_e2e"]),
                "roofline": {"bound": "alu", "achieved": a64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a64 / FP64_PEAK_TFLOPS,
                             "traffic": work.get("dram_bytes_per_launch_scaled", {}).get("fp64")}}
            line["speedup_vs_plain_fp64"] = f["t_dev"] / r["t_dev"]
            # both forms ran the same steps from the same state: density difference
            d = (r["rho"] - f["rho"]).abs().max().item() / f["rho"].abs().max().item()
            line["max_rel_density_diff_vs_fp64"] = d
        if "fp64_gated" in res and "fp64" in res:
            fg, f = res["fp64_gated"], res["fp64"]
            line["plain_fp64_with_indicator"] = {
                "value": job_rate(CELLS * args.steps, ws, fg["t_dev"]), "ms_per_step": 1e3 * fg["t_dev"] / args.steps,
                "kernel_ms": 1e3 * fg["kern_s"], "speedup_vs_plain_fp64": f["t_dev"] / fg["t_dev"],
                "max_rel_density_diff_vs_fp64": (fg["rho"] - f["rho"]).abs().max().item() / f["rho"].abs().max().item()}
        if "gated" in res:
            gr = res["gated"]
            line["mixed_with_indicator"] = {
                "value": job_rate(CELLS * args.steps, ws, gr["t_dev"]), "ms_per_step": 1e3 * gr["t_dev"] / args.steps,
                "kernel_ms": 1e3 * gr["kern_s"],
                "speedup_vs_mixed": r["t_dev"] / gr["t_dev"] if head == "mixed" else None,
                "max_rel_density_diff_vs_fp64": ((gr["rho"] - res["fp64"]["rho"]).abs().max().item() /
                                                 res["fp64"]["rho"].abs().max().item()) if "fp64" in res else None,
                "indicator_held_out": ind_eval}
        if args.amr:
            line["amr_batched"] = {"workload": "adaptive octree, ~4,096 leaves of 8^3 at levels 3-6 refined around a "
                                               "blast shell of radius 0.3, leaf order shuffled (seed 1234), outflow",
                                   "mixed": amr_measure(args, H, dev, flush, H.HYDRO_PREC_MIXED, args.steps),
                                   "fp64": amr_measure(args, H, dev, flush, H.HYDRO_PREC_FP64, max(2, args.steps // 5))}
            if indicator is not None:
                line["amr_batched"]["gated"] = amr_measure(args, H, dev, flush, H.HYDRO_PREC_MIXED, args.steps,
                                                           indicator)
                line["amr_batched"]["fp64_gated"] = amr_measure(args, H, dev, flush, H.HYDRO_PREC_FP64,
                                                                max(2, args.steps // 5), indicator)
        if args.polytrope:
            line["rotating_polytrope"] = polytrope_measure(args, H, dev, flush, indicator)
        if args.contact:
            try:
                line["contact_steepening"] = contact_measure(args, H, dev, flush, res)
            except Exception as e:  # an optional block: it never costs the headline line
                line["contact_steepening"] = {"error": f"{type(e).__name__}: {e}"}
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def oracle_sample():
    """The central 4x4x4 sub-grids of the workload (32^3 cells, same h)."""
    from oracle import core, mesh  # noqa: F401
    from paper_2107_10987_gb300 import workloads as W
    Ug, h, lo = W.sedov_box(NB * N, GAMMA)
    c = slice(16, 48)
    sub = Ug[:, c, c, c].copy()
    return sub, h, (lo[0] + 16 * h, lo[1] + 16 * h, lo[2] + 16 * h)


def cpu_baseline(budget_s: float):
    """The oracle as it stands, on all host cores, on a bounded sample."""
    from oracle import core, mesh
    core.build()
    Ug, h, lo = oracle_sample()
    run = mesh.BoxRun(core.OracleParams(gamma=GAMMA), Ug, h, lo, "outflow")
    run.step(0.4)  # warm-up (thread pool, caches)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        run.step(0.4)
        steps += 1
    dt = time.perf_counter() - t0
    cells = Ug[0].size
    out = {"value": cells * steps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{steps} RK3 steps of the central 4x4x4 sub-grids (32^3 cells) of the workload, "
                     f"{dt:.1f} s, OpenMP over sub-grids on all host cores"}
    # the same sample on one core, for a quarter of the budget
    run1 = mesh.BoxRun(core.OracleParams(gamma=GAMMA), Ug, h, lo, "outflow", nthreads=1)
    t0 = time.perf_counter()
    steps1 = 0
    while time.perf_counter() - t0 < budget_s / 4 or steps1 == 0:
        run1.step(0.4)
        steps1 += 1
    dt1 = time.perf_counter() - t0
    out["single_core"] = {"value": cells * steps1 / dt1, "unit": UNIT, "cores": 1,
                          "sample": f"{steps1} RK3 steps of the same sample, {dt1:.1f} s"}
    return out


def reference_arm(args):
    ws, rk, lr = dist_env()
    if rk != 0:
        return
    from oracle import core, mesh
    core.build()
    Ug, h, lo = oracle_sample()
    run = mesh.BoxRun(core.OracleParams(gamma=GAMMA), Ug, h, lo, "outflow")
    for _ in range(args.warmup):
        run.step(0.4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step(0.4)
    dt = time.perf_counter() - t0
    cells = Ug[0].size
    v = cells * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Sedov blast, central 4x4x4 sub-grids (32^3 cells, h = 1/32) of the 512-sub-grid "
                                   "uniform mesh, outflow, one step = one full RK3 time step", "cells": cells},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} RK3 steps of 32^3 cells on all host cores"},
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
