"""Benchmark: cell-updates per second of full SSP-RK3 steps of the two-phase
WENO-IS / MOOD / HLLC solver on the 2D planar-shock / air-bubble workload
(1024 x 1024 cells, Ms = 1.5 water shock, air bubble of radius 0.2).

One "step" is one SSP-RK3 step of the whole grid: CFL reduction, and per stage
the ghost layers, the primitive cache, the x and y face sweeps (projection,
WENO-IS, MOOD, HLLC) and the flux-divergence + RK update, all in this
library's CUDA kernels, with the state resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun): every rank advances its own replica of the workload
(the problems are independent; no data-path collective), value = all cells
updated by all ranks / the slowest rank's time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_00592_gb300 import workloads as wl  # noqa: E402

METRIC = "cell-updates/s per RK3 step"
UNIT = "cell-updates/s"
L2_BYTES = 129 * 2**20

# FP64 operations of one face (add/sub/mul/div/sqrt/min/max each 1), counted
# from the face formulas with nq = ndim + 4 characteristic variables:
#   setup (averages, non-zero L/R entries) 12, projection of 6 cells 48,
#   WENO-IS 100 per variable and side (2 nq x 100), back-projection 16,
#   MOOD admissibility 6, HLLC 114 + 8 (nq - 5) + 11 nq.
def face_flops(ndim: int) -> int:
    nq = ndim + 4
    return 12 + 48 + 200 * nq + 16 + 6 + (114 + 8 * (nq - 5) + 11 * nq)


# A characteristic variable whose stencil is flat to 1e-6 of its magnitude
# takes the linear weights, evaluated as 4 subtractions, 1 multiply and 4 FMAs
# (13 flops) a side instead of WENO-IS's 100.  Flops per face the kernel
# executes, given the fraction of flat face-variables (from ws_census_step;
# the flat test itself is not counted).
def executed_face_flops(ndim: int, flat_fraction: float) -> float:
    nq = ndim + 4
    return face_flops(ndim) - 2 * nq * (100 - 13) * flat_fraction


# algorithmic HBM bytes of one fully fused RK3 cell-update with an FP64 state:
# 3 stages read U^n and U^(s) and write U^(s+1) -> (2 + 3 + 3) nv 8 B
def cell_update_bytes(ndim: int) -> int:
    return 8 * (ndim + 4) * 8


# DRAM bytes moved by one launch of the fused 2D mixed stage on the 1024^2
# shock-bubble at mid-run (ncu, 50.72 MB read + 2.37 MB written; the stage's
# FP32 scratch mostly stays in the 129 MB L2 between launches)
STAGE2D_DRAM_BYTES = 53.09e6


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max_ms(ms: float, device=None) -> float:
    """Slowest rank's timed-region duration (ms); identity on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(cells_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job rate: every rank advances its own replica, so the cells
    updated by all ranks over the slowest rank's time."""
    return world * cells_per_rank * steps / (max_ms * 1e-3)


def dist_setup():
    ws_size = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws_size, rank, local


def sample_case(n: int, rows: int):
    """A bounded sample of the workload for CPU timing: the full-width strip of
    `rows` rows through the bubble's centre (transmissive at the cut rows)."""
    case = wl.shock_bubble_2d(n)
    y0 = n // 2 - rows // 2
    Q = case.Q[:, :, 3 + y0 - 3:3 + y0 + rows + 3, :].copy()
    return case, Q, rows


def cpu_oracle_rate(n: int, rows: int, steps: int):
    import oracle
    case, Q, rows = sample_case(n, rows)
    g = oracle.Grid(2, (n, rows), (case.dx[0], case.dx[1]), case.bc)
    U = oracle.prim_to_cons(2, Q)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        U, _, _ = oracle.step(g, U)
        times.append(time.perf_counter() - t0)
    return n * rows, times, oracle.get_threads()


def workload_config(args, ws_size: int) -> dict:
    """The headline workload, as both arms name it."""
    n = args.n
    return {"workload": f"shock_bubble_2d_{n}x{n}", "grid": [n, n], "run_steps": args.run_steps,
            "timed_steps": f"{args.steps} steps spread evenly over the {args.run_steps}-step run "
                           f"(after {args.warmup} warm-up steps)",
            "cfl": 0.5, "mood": True, "weights": "modified",
            "l2": "L2 flushed (258 MB write) between timed steps",
            "parallelism": f"replicas x{ws_size}"}


def run_reference(args):
    ws_size, rank, _ = dist_setup()
    if rank != 0:
        return
    n, rows = args.n, args.ref_rows
    cells, times, cores = cpu_oracle_rate(n, rows, args.warmup + args.steps)
    t = sum(times[args.warmup:])
    value = cells * args.steps / t
    sample = f"{n}x{rows} strip of the {n}^2 workload through the bubble centre, one oracle RK3 step per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(args, ws_size),
                       "timed_steps": f"{args.steps} oracle steps on a strip of the workload "
                                      f"(after {args.warmup} warm-up steps)",
                       "l2": "CPU run: no GPU cache to flush"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def l1_vs_fp64(ws, case, s_mixed, stream, steps):
    """L1 relative density error of the mixed path against the FP64 path (which
    is bit-identical to the FP64 oracle) after `steps` steps from the same
    initial state, both with the FP64 path's CFL time steps."""
    import torch
    s64 = ws.Solver(2, case.n, case.dx, case.bc, precision="fp64", stream=stream)
    U64 = s64.prim_to_cons(s64.tensor(case.Q))
    U32 = s_mixed.prim_to_cons(s_mixed.tensor(case.Q))
    for _ in range(steps):
        dt = s64.step(U64, want_dt=True)
        s_mixed.step(U32, dt)
    torch.cuda.synchronize()
    sl = wl.interior(2, case.n)
    a = U32[sl][0].double()
    b = U64[sl][0]
    s64.close()
    return {"steps": steps, "value": float((a - b).abs().sum() / b.abs().sum()),
            "reference": "FP64 path (bit-identical to the FP64 oracle)"}


def time_fp64(ws, case, stream, steps):
    """cell-updates/s of the plain FP64 path (bit-identical to the oracle) on the
    same workload, timed the same way (L2 flushed between steps)."""
    import torch
    s64 = ws.Solver(2, case.n, case.dx, case.bc, precision="fp64", stream=stream)
    U = s64.prim_to_cons(s64.tensor(case.Q))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(2):
        s64.step(U)
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s64.step(U)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    s64.close()
    return {"value": case.cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps}


def time_tubes(ws, stream, steps, seed=0):
    """The batched configuration: 4096 independent 1D Riemann tubes of 256..8192
    cells (log-uniform) in one persistent launch per RK stage, mixed precision,
    per-tube CFL steps, autotuned chunking, CUDA-graph replay."""
    import torch
    off, Q = wl.riemann_tubes(ntubes=4096, lmin=256, lmax=8192, seed=seed)
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision="mixed", stream=stream)
    cells = int(sum(off[t + 1] - off[t] - 6 for t in range(len(off) - 1)))
    with torch.cuda.stream(stream):
        U = s.prim_to_cons(s.tensor(Q))
        choice = ws.ws_autotune(s.ctx, U, 2)
        ws.ws_set_graph(s.ctx, True)
        for _ in range(3):
            s.step(U)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(U)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        bad = s.nonphysical()
    s.close()
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "tubes": 4096,
            "cells": cells, "chunk_config": choice, "graph": True, "nonphysical_cells": bad,
            "workload": "4096 Riemann tubes, lengths log-uniform in [256, 8192], per-tube CFL, mixed precision"}


def time_setups(ws, stream, steps):
    """The shock-interface setups of Secs. 6.1 and 6.2 at the paper's grid
    sizes (air shock on an R22 or helium cylinder, 3000 x 1000, reflective
    walls, run to the paper's last time; air shock on a water droplet,
    800 x 800, 2000 steps), mixed precision, MOOD off as in the paper.  The
    timed CFL steps are spread evenly over each run (the work per step follows
    the flow)."""
    import torch
    out = {}
    for name, make, t_end, nmax in (("air_R22_3000x1000", lambda: wl.haas_sturtevant("R22"), 420e-6, 20000),
                                    ("air_He_3000x1000", lambda: wl.haas_sturtevant("He"), 674e-6, 20000),
                                    ("shock_droplet_800x800", lambda: wl.shock_droplet(800), None, 2000)):
        case = make()
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", mood=False, stream=stream)
        with torch.cuda.stream(stream):
            U = s.prim_to_cons(s.tensor(case.Q))
            # run length in steps: to t_end, estimated from the first step (the
            # shock sets the wave speed), within nmax
            dt0 = s.step(U, want_dt=True)
            total = nmax if t_end is None else min(nmax, int(t_end / dt0))
            gap = max(0, total // max(steps, 1) - 1)
            ms, t = 0.0, dt0
            for _ in range(steps):
                for _ in range(gap):
                    s.step(U)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(U)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
            bad = s.nonphysical()
        ms /= steps
        out[name] = {"value": case.cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "timed_steps": f"{steps} spread over {1 + steps * (gap + 1)} steps",
                     "nonphysical_cells": bad}
        s.close()
        del U
    return out


def time_drop3d(ws, stream, steps, peak, n=256, l1_n=96, l1_steps=20):
    """The 3D configuration: the periodic water drop with density noise on n^3,
    mixed precision through the fused 3D stage (two launches per RK stage).
    Also: pressure equilibrium after the timed steps, and the L1 density error
    against the FP64 path (bit-identical to the FP64 oracle) on l1_n^3 after
    l1_steps steps with the FP64 path's CFL time steps."""
    import torch
    case = wl.drop_3d(n, seed=0)
    s = ws.Solver(3, case.n, case.dx, case.bc, precision="mixed", stream=stream)
    with torch.cuda.stream(stream):
        U = s.prim_to_cons(s.tensor(case.Q))
        del case
        for _ in range(3):
            s.step(U)
        # census of the reconstruction's evaluations on a copy of the state the
        # timed steps start from
        Uc = U.clone()
        census = s.census_step(Uc)
        del Uc
        ws.ws_profile(s.ctx, True)
        ms = 0.0
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(U)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        face_ms, face_n = ws.ws_profile_read(s.ctx)["face"]
        ws.ws_profile(s.ctx, False)
        Q = s.cons_to_prim(U)
        sl = wl.interior(3, (n, n, n))
        dp = float((Q[sl][4] / 1e5 - 1.0).abs().max().item())
        del Q
        bad = s.nonphysical()
    s.close()
    del U
    torch.cuda.empty_cache()
    # L1 against the FP64 path on a smaller grid
    small = wl.drop_3d(l1_n, seed=0)
    s64 = ws.Solver(3, small.n, small.dx, small.bc, precision="fp64", stream=stream)
    s32 = ws.Solver(3, small.n, small.dx, small.bc, precision="mixed", stream=stream)
    with torch.cuda.stream(stream):
        U64 = s64.prim_to_cons(s64.tensor(small.Q))
        U32 = s32.prim_to_cons(s32.tensor(small.Q))
        for _ in range(l1_steps):
            dt = s64.step(U64, want_dt=True)
            s32.step(U32, dt)
        torch.cuda.synchronize()
        sl = wl.interior(3, small.n)
        l1 = float(((U32[sl][0] - U64[sl][0]).abs().sum() / U64[sl][0].abs().sum()).item())
    s64.close()
    s32.close()
    cells = n ** 3
    faces_per_stage = 3 * (n + 1) * n * n
    achieved = face_flops(3) * faces_per_stage * 3 * steps / (face_ms * 1e-3) / 1e12
    # executed flops (census), the method's figure beside them: as the 2D line
    flat = census["flat"] / max(census["face_variables"], 1)
    ex = executed_face_flops(3, flat)
    evaluated = census["face_variables"] / (7 * 3)  # faces evaluated per stage (tile edges twice)
    ex_achieved = ex * evaluated * 3 * steps / (face_ms * 1e-3) / 1e12
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "workload": f"drop_3d_{n}^3 (periodic water drop r=0.25 in air, 1% density noise, seed 0), mixed",
            "l2": f"state {cells * 7 * 8 / 1e9:.2f} GB, larger than L2",
            "gpu_launches": int(face_n),
            "roofline": {"bound": "alu", "kernel": "fused 3D RK stage, both passes", "achieved": ex_achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": ex_achieved / peak,
                         "flops_per_face": ex, "faces_per_stage": evaluated,
                         "flops_counted": "executed, as the 2D line (census of the first timed step's state)",
                         "flat_face_variable_fraction": flat,
                         "warp_passes_running_weno_is": census["warp_passes_weno"] / max(census["warp_passes"], 1),
                         "share_of_step": face_ms / ms,
                         "method": {"what": "WENO-IS at every face, as Sec. 3.3 defines the reconstruction",
                                    "flops_per_face": face_flops(3), "faces_per_stage": faces_per_stage,
                                    "achieved": achieved, "frac": achieved / peak}},
            "pressure_equilibrium_max_rel_dev": dp, "nonphysical_cells": bad,
            "l1_density_vs_fp64": {"grid": [l1_n] * 3, "steps": l1_steps, "value": l1}}


def time_learned(ws, case, stream, steps, run_steps, warmup, nograph=False):
    """The learned smooth-face gate on the same run: trained on the GPU by the
    library's kernels, then timed like the plain mixed path, with its L1 density
    difference from the plain mixed path after the timed run.  nograph: the
    contexts get no stream, so a gated step is a sequence of launches instead of
    one graph (profilers cannot look inside graphs with conditional nodes)."""
    import torch
    from paper_1707_00592_gb300 import learned
    P, thr, rep = learned.train_gate(total=2_000_000, epochs=4)
    outs = {}
    if nograph:  # the legacy default stream: no capture, so no graph
        stream = torch.cuda.default_stream()
    for mode in ("plain", "gated", "gated_per_step"):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", stream=stream)
        if mode == "gated":
            ws.ws_set_mlp(s.ctx, P, thr)
        elif mode == "gated_per_step":
            ws.ws_set_mlp(s.ctx, P, thr, ws.GATE_REDO_DRIFT | ws.GATE_REDO_NONPHYS | ws.GATE_PER_STEP)
        torch.cuda.nvtx.range_push(f"learned_{mode}")  # lets a profiler select one mode's launches
        with torch.cuda.stream(stream):
            U = s.prim_to_cons(s.tensor(case.Q))
            for _ in range(warmup):
                s.step(U, 5e-8)
            gap = max(0, (run_steps - warmup - steps) // max(steps, 1))
            flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
            ms = 0.0
            for _ in range(steps):
                for _ in range(gap):
                    s.step(U, 5e-8)
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(U, 5e-8)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
            stats = ws.ws_gate_stats(s.ctx) if mode != "plain" else None
        torch.cuda.nvtx.range_pop()
        outs[mode] = (U[wl.interior(2, case.n)][0].double(), ms / steps, stats)
        s.close()
    b = outs["plain"][0]

    def summary(mode):
        a, ms_, st = outs[mode]
        return {"ms_per_step": ms_, "l1_density_vs_plain_mixed": float((a - b).abs().sum() / b.abs().sum()),
                "gated_face_fraction": st["smooth_faces"] / max(st["faces"], 1.0), "steps_redone": st["redone"]}

    per_step, per_stage = summary("gated_per_step"), summary("gated")
    return {"value": case.cells / (per_step["ms_per_step"] * 1e-3), "unit": UNIT, **per_step,
            "gate": "MLP once per step (RK stage 0), decisions reused in stages 1 and 2",
            "per_stage_mlp": per_stage, "plain_ms_per_step": outs["plain"][1],
            "training": rep, "dt": "fixed 5e-8 for all runs (same trajectory)"}


def run_ours(args):
    import torch
    import paper_1707_00592_gb300 as ws

    ws_size, rank, local = dist_setup()
    if ws_size > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    n = args.n
    case = wl.shock_bubble_2d(n)
    with torch.cuda.stream(stream):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision=args.precision, stream=stream)
        Q = s.tensor(case.Q)
        U0 = s.prim_to_cons(Q)
        U = U0.clone()
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            s.step(U)
        stream.synchronize()
        # the K timed steps are spread over the whole run (the per-step work
        # depends on the flow state), the run advancing untimed between them
        gap = max(0, (args.run_steps - args.warmup - args.steps) // max(args.steps, 1))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if ws_size > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        # census of the reconstruction's evaluations at each timed step's state,
        # on a copy, outside the timed events and the kernel profile
        census = {k: 0 for k in ws.CENSUS_KEYS} if args.precision == "mixed" else None
        mood_counts = np.zeros((3, 3), dtype=np.int64)  # direction x order (5th, 3rd, 1st)
        Uc = torch.empty_like(U) if census is not None else None
        ws.ws_profile(s.ctx, True)
        with ClockSampler(dev) as clk:
            for k in range(args.steps):
                if gap:
                    ws.ws_profile(s.ctx, False)
                    for _ in range(gap):
                        s.step(U)
                    ws.ws_profile(s.ctx, True, reset=False)
                if census is not None:
                    ws.ws_profile(s.ctx, False)
                    Uc.copy_(U)
                    c = s.census_step(Uc)
                    for key in ws.CENSUS_KEYS:
                        census[key] += c[key]
                    mood_counts += s.mood()[0]  # the census step replays the timed step bit for bit
                    ws.ws_profile(s.ctx, True, reset=False)
                flush.zero_()  # evict the state from L2 between timed steps
                ev[k][0].record(stream)
                s.step(U)
                ev[k][1].record(stream)
            stream.synchronize()
        del Uc
        torch.cuda.synchronize()
        prof = ws.ws_profile_read(s.ctx)
        ws.ws_profile(s.ctx, False)
        ms = sum(a.elapsed_time(b) for a, b in ev)
        ms = reduce_max_ms(ms, device="cuda")
        cells = case.cells
        value = aggregate_rate(cells, args.steps, ws_size, ms)
        launches = int(sum(v[1] for v in prof.values()))

        # end to end through the public C ABI with host buffers: H2D of the
        # state, one RK3 step, D2H of the state, per step
        Uh = U0.cpu().pin_memory()
        ws.ws_run_host(s.ctx, Uh, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ws.ws_run_host(s.ctx, Uh, 1)
        e2e_t = (time.perf_counter() - t0) / args.steps
        state_bytes = s.size * 8

        l1 = None
        fp64_cmp = None
        if args.precision == "mixed" and args.l1_steps > 0:
            l1 = l1_vs_fp64(ws, case, s, stream, args.l1_steps)
        if args.precision == "mixed" and args.fp64_steps > 0:
            fp64_cmp = time_fp64(ws, case, stream, args.fp64_steps)
        tubes = time_tubes(ws, stream, args.tube_steps) if args.tube_steps > 0 else None
        setups = time_setups(ws, stream, args.setup_steps) if args.setup_steps > 0 and args.precision == "mixed" else None
        drop = None
        if args.drop_steps > 0 and args.precision == "mixed":
            p32 = args.fp32_peak if args.fp32_peak is not None else ws.ws_peak_probe("fp32")
            drop = time_drop3d(ws, stream, args.drop_steps, p32, n=args.drop_n)
        gate = (time_learned(ws, case, stream, args.steps, args.run_steps, args.warmup, args.learned_nograph)
                if args.learned and args.precision == "mixed" else None)

    clocks = clk.summary()
    if rank != 0:
        if ws_size > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, which = load_peaks()
    face_ms, face_n = prof["face"]
    per_launch_s = face_ms * 1e-3 / max(face_n, 1)
    # the FP64 path launches one face sweep per direction; the mixed path one
    # fused stage kernel covering both directions' faces
    faces_per_launch = (n + 1) * n * (1 if args.precision == "fp64" else 2)
    flops = face_flops(2) * faces_per_launch
    achieved = flops / per_launch_s / 1e12
    if args.precision == "fp64":
        peak = args.fp64_peak if args.fp64_peak is not None else ws.ws_peak_probe("fp64")
        kname, psrc = "face sweep (FP64)", "FP64 FMA chain probe on this GPU (2 flops per DFMA)"
    else:
        peak = args.fp32_peak if args.fp32_peak is not None else ws.ws_peak_probe("fp32")
        kname, psrc = ("fused RK stage (FP32 mixed: tile load, x and y faces, update)",
                       "FP32 FMA chain probe on this GPU (2 flops per FFMA)")
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": STAGE2D_DRAM_BYTES if args.precision == "mixed" and n == 1024 else None,
                "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one fused-stage launch "
                                  "(1024^2, step ~300, stage 1), bytes per launch",
                "peak_source": psrc,
                "flops_per_face": face_flops(2), "faces_per_launch": faces_per_launch,
                "face_ms_per_launch": per_launch_s * 1e3,
                "share_of_step": face_ms / ms,
                "hbm_bytes_per_cell_update": cell_update_bytes(2),
                "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": which}
    if census is not None and census["face_variables"]:
        # The headline figure counts the flops the kernel executes: WENO-IS only
        # where the stencil is not flat (census of the timed steps' states), the
        # linear weights elsewhere, over every face evaluation (tile edges twice).
        # The figure of the method (WENO-IS at every face) is kept beside it.
        flat = census["flat"] / census["face_variables"]
        ex = executed_face_flops(2, flat)
        evaluated = census["face_variables"] / (6 * 3 * args.steps)
        ex_achieved = ex * evaluated / per_launch_s / 1e12
        roofline["method"] = {"what": "WENO-IS at every face, as Sec. 3.3 defines the reconstruction",
                              "flops_per_face": face_flops(2), "faces_per_launch": faces_per_launch,
                              "achieved": achieved, "frac": achieved / peak}
        roofline.update({
            "achieved": ex_achieved, "frac": ex_achieved / peak, "flops_per_face": ex,
            "faces_per_launch": evaluated,
            "flops_counted": "executed: WENO-IS (100 flops a side) for face-variables with a non-flat stencil, "
                             "the linear weights (13 flops a side) for flat ones, over every face evaluation "
                             "(faces on tile edges twice); the flat test itself is not counted",
            "flat_face_variable_fraction": flat,
            "warp_passes_running_weno_is": census["warp_passes_weno"] / max(census["warp_passes"], 1),
            "census": f"ws_census_step on a copy of the state before each of the {args.steps} timed steps"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_size, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {**workload_config(args, ws_size), "precision": args.precision},
            "gpu_launches": launches,
            "kernel_ms": {k: v[0] for k, v in prof.items() if v[1]},
            "roofline": roofline,
            "e2e": {"value": cells / e2e_t, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes}}
    if clocks:
        line["clocks"] = clocks
    if census is not None:
        line["mood"] = {"what": "face sides reconstructed at each order by the MOOD cascade (Sec. 3.4), summed "
                                "over the three RK stages of every timed step (from the census replay of each)",
                        **{ax: dict(zip(("5th", "3rd", "1st"), (int(v) for v in mood_counts[d])))
                           for d, ax in enumerate(("x", "y"))}}
    if l1 is not None:
        line["l1_density_vs_fp64"] = l1
    if fp64_cmp is not None:
        line["fp64_plain"] = fp64_cmp
    if tubes is not None:
        line["batched_tubes"] = tubes
    if drop is not None:
        line["drop_3d"] = drop
    if setups is not None:
        line["shock_interface_setups"] = setups
    if gate is not None:
        line["learned_gate"] = gate
    if ws_size == 1 and not args.no_cpu_baseline:
        cells_c, times, cores = cpu_oracle_rate(n, args.cpu_rows, args.cpu_steps)
        line["cpu_baseline"] = {"kind": "oracle", "value": cells_c * len(times) / sum(times), "unit": UNIT,
                                "cores": cores,
                                "sample": f"{args.cpu_steps} oracle RK3 steps on the {n}x{args.cpu_rows} strip "
                                          f"of the {n}^2 workload through the bubble centre"}
    print(json.dumps(line), flush=True)
    if ws_size > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--cpu-rows", type=int, default=128)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--ref-rows", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-peak", type=float, default=None)
    ap.add_argument("--fp32-peak", type=float, default=None)
    ap.add_argument("--l1-steps", type=int, default=200)
    ap.add_argument("--run-steps", type=int, default=2000)
    ap.add_argument("--tube-steps", type=int, default=10)
    ap.add_argument("--drop-steps", type=int, default=10)
    ap.add_argument("--learned-nograph", action="store_true")
    ap.add_argument("--drop-n", type=int, default=256)
    ap.add_argument("--setup-steps", type=int, default=10)
    ap.add_argument("--learned", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=5)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
