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

# Flops of the method (one per add, subtract, multiply, divide, square root,
# min, max or comparison; none for an operand that is an exact zero, or +-1 in
# a product), as the op-counting build of the FP64 oracle counts them on
# generic data (oracle/flop_count.cpp; tests/test_flop_count.py checks every
# term below against it).  nq = ndim + 4 characteristic variables per face.
WENO_FLOPS = 99  # one WENO-IS reconstruction, one variable, one side (Sec. 3.3)


def hllc_flops(nq: int) -> int:
    """HLLC flux and face velocity of one face (Sec. 3.2.1)."""
    return 172 + 20 * (nq - 5)


def face_flops(ndim: int) -> int:
    """One face: averages and the non-zero entries of L and R 13, projection of
    six cells 48, WENO-IS of every variable and side, back-projection of both
    sides 16, MOOD admissibility of both sides 12, HLLC."""
    nq = ndim + 4
    return 13 + 48 + 2 * nq * WENO_FLOPS + 16 + 12 + hllc_flops(nq)


def prim_flops(ndim: int) -> int:
    """Per cell and RK stage: primitive recovery (Eq. eos) and sound speed."""
    return 10 + 3 * ndim


def divergence_flops(ndim: int) -> int:
    """Per cell and RK stage: flux divergence of every field over the ndim
    directions with the Gamma/Pi source terms (Sec. 3.1)."""
    nv = ndim + 4
    return 2 * nv * ndim + (ndim - 1) * nv + 8 * ndim


def stage_flops(ndim: int, n) -> int:
    """The method's flops of one RK stage on a grid of n cells per direction:
    every distinct face once, every cell's primitives and divergence once (the
    RK update and the CFL reduction, about 100 flops per cell and step, are
    not counted)."""
    cells = int(np.prod([n[d] for d in range(ndim)]))
    faces = sum((n[d] + 1) * cells // n[d] for d in range(ndim))
    return faces * face_flops(ndim) + cells * (prim_flops(ndim) + divergence_flops(ndim))


# A characteristic variable whose stencil is flat to 1e-6 of its magnitude
# takes the linear weights, which the mixed kernel evaluates as 4 differences,
# 1 product and 4 fused multiply-adds (13 flops) a side instead of WENO-IS.
# Flops per face the kernel executes, given the fraction of flat
# face-variables (from ws_census_step; the flat test itself is not counted).
LINEAR_FLOPS = 13


def executed_face_flops(ndim: int, flat_fraction: float) -> float:
    nq = ndim + 4
    return face_flops(ndim) - 2 * nq * (WENO_FLOPS - LINEAR_FLOPS) * flat_fraction


# FP32 peak of an ALU-bound kernel from the unit counts and the clock: 152 SMs
# x 128 FP32 lanes x 2 flops per fused multiply-add x 2.07 GHz (maximum SM
# clock).  A paired FP32 instruction does two lanes' work in two pipe cycles,
# so pairing does not raise it.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# algorithmic HBM bytes of one fully fused RK3 cell-update with an FP64 state:
# 3 stages read U^n and U^(s) and write U^(s+1) -> (2 + 3 + 3) nv 8 B
def cell_update_bytes(ndim: int) -> int:
    return 8 * (ndim + 4) * 8


# DRAM bytes moved by one launch of the fused 2D mixed stage on the 1024^2
# shock-bubble, in the default tail-filled configuration (ncu, one resident
# step at step 10 of a 60-step run): stage 0 reads the carried FP32 image
# (25.49 MB read, 0.03 MB written), stage 1 the image and K0 (50.86 + 0.46 MB),
# stage 2 also the FP64 state it updates (101.59 + 24.63 MB; the rest of its
# writes are still in L2 at the end); the mean over the three launches (the
# 32 x 15-only configuration moves 67.5 MB)
STAGE2D_DRAM_BYTES = (25.513728 + 51.326464 + 126.210816) / 3 * 1e6
STAGE2D_DRAM_SOURCE = ("dram__bytes_read.sum + dram__bytes_write.sum per fused-stage launch, mean of the three "
                       "stages of one resident step (1024^2, step 10 of 60; ncu)")


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


def inadmissible_tubes(off, U):
    """{tube: number of interior cells with rho <= 0, Gamma <= 0 or p + P_inf
    <= 0 (or not finite)} of a host copy of the tubes' conservative state."""
    rho, mu, E, G, P = U
    with np.errstate(all="ignore"):
        pe = E - 0.5 * mu * mu / rho - P  # Gamma p
        ok = (rho > 0) & (G > 0) & ((G + 1.0) * pe / G + P > 0) & np.isfinite(pe)
    out = {}
    for t in range(len(off) - 1):
        k = int(np.count_nonzero(~ok[off[t] + 3:off[t + 1] - 3]))
        if k:
            out[t] = k
    return out


def time_tubes(ws, stream, steps, seed=0, run_steps=1000, sample=64):
    """The batched configuration: 4096 independent 1D Riemann tubes of 256..8192
    cells (log-uniform) in one persistent launch per RK stage, mixed precision,
    per-tube CFL steps, autotuned chunking, CUDA-graph replay; run_steps steps
    with the timed steps spread evenly over the run.  Then the L1 density
    difference of a seeded sample of tubes against the FP64 path (bit-identical
    to the FP64 oracle) run on that sample alone for the same number of
    per-tube CFL steps (the tubes are independent, so a tube's mixed-precision
    trajectory does not depend on the batch around it)."""
    import torch
    off, Q = wl.riemann_tubes(ntubes=4096, lmin=256, lmax=8192, seed=seed)
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision="mixed", stream=stream)
    cells = int(sum(off[t + 1] - off[t] - 6 for t in range(len(off) - 1)))
    warm = 3
    gap = max(0, (run_steps - warm - steps) // max(steps, 1))
    with torch.cuda.stream(stream):
        U = s.prim_to_cons(s.tensor(Q))
        choice = ws.ws_autotune(s.ctx, U, 2)
        ws.ws_set_graph(s.ctx, True)
        for _ in range(warm):
            s.step(U)
        done = warm
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        ms = 0.0
        for _ in range(steps):
            for _ in range(gap):
                s.step(U)
            done += gap
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(U)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            done += 1
        while done < run_steps:
            s.step(U)
            done += 1
        bad = s.nonphysical()
        Um = U.cpu().numpy()
    s.close()
    del U, flush
    bad_tubes = inadmissible_tubes(off, Um)

    def fp64_alone(pick):
        """The FP64 path on the picked tubes alone, run_steps per-tube CFL steps."""
        lens = np.array([off[t + 1] - off[t] for t in pick])
        soff = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        Qs = np.concatenate([Q[:, off[t]:off[t + 1]] for t in pick], axis=1)
        s64 = ws.Solver(1, (1,), (1.0,), tube_offsets=soff, precision="fp64", stream=stream)
        with torch.cuda.stream(stream):
            U64 = s64.prim_to_cons(s64.tensor(Qs))
            ws.ws_set_graph(s64.ctx, True)
            for _ in range(run_steps):
                s64.step(U64)
            bad64 = s64.nonphysical()
            U64 = U64.cpu().numpy()
        s64.close()
        return U64, soff, lens, bad64

    # the tubes the mixed run left with an inadmissible cell, run again alone
    # on the FP64 path (bit-identical to the oracle): does the scheme itself
    # fail on them?
    same = None
    if bad_tubes:
        _, _, _, bad_same = fp64_alone(sorted(bad_tubes))
        same = {"tubes": len(bad_tubes), "mixed_nonphysical_cells": int(sum(bad_tubes.values())),
                "fp64_nonphysical_cells": bad_same}
    # the seeded sample, alone, in FP64
    rng = np.random.default_rng(seed + 1)
    pick = np.sort(rng.choice(len(off) - 1, size=sample, replace=False))
    U64, soff, lens, bad64 = fp64_alone(pick)
    num = den = 0.0
    for k, t in enumerate(pick):
        a = Um[0, off[t] + 3:off[t + 1] - 3]
        b = U64[0, soff[k] + 3:soff[k + 1] - 3]
        num += float(np.abs(a - b).sum())
        den += float(np.abs(b).sum())
    # the method's flops of a step: every tube's faces (one more than its
    # cells) and cells, three stages; over the step's event time (the graph
    # of the three stage launches)
    ntubes = len(off) - 1
    flops = 3 * ((cells + ntubes) * face_flops(1) + cells * (prim_flops(1) + divergence_flops(1)))
    achieved = flops / (ms / steps * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "persistent tube stage (mixed), three launches per step", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "flops_per_step": flops,
                "flops_source": f"the method's flops (op-counting build of the FP64 oracle): {face_flops(1)} per "
                                f"face, {prim_flops(1) + divergence_flops(1)} per cell and stage",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz"}
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "tubes": 4096,
            "cells": cells, "chunk_config": choice, "graph": True, "roofline": roofline, "nonphysical_cells": bad,
            "nonphysical_tubes": len(bad_tubes), "nonphysical_tubes_fp64_alone": same,
            "run_steps": run_steps, "timed_steps": f"{steps} spread evenly over the {run_steps}-step run",
            "workload": "4096 Riemann tubes, lengths log-uniform in [256, 8192], per-tube CFL, mixed precision",
            "l1_density_vs_fp64": {"value": num / den, "tubes": int(sample), "cells": int(lens.sum() - 6 * sample),
                                   "steps": run_steps, "fp64_nonphysical_cells": bad64,
                                   "what": "sum over a seeded sample of tubes of |rho_mixed - rho_fp64| / sum "
                                           "|rho_fp64| after run_steps per-tube CFL steps of each path"}}


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
        ws.ws_set_resident(s.ctx, True)
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


def time_drop3d(ws, stream, steps, probe, n=256, run_steps=500, l1_n=128, l1_steps=500):
    """The 3D configuration: the periodic water drop with density noise on n^3,
    mixed precision through the fused 3D stage (two launches per RK stage), run
    for run_steps CFL steps with the timed steps spread evenly over the run.
    After the run: pressure equilibrium (Sec. 5.1: p stays uniform across the
    advected interface) and the inadmissible cells.  The L1 density drift
    against the FP64 path (bit-identical to the FP64 oracle) is taken on l1_n^3
    after l1_steps steps with the FP64 path's CFL time steps (the FP64 path
    updates 2e7 cells/s in 3D, so 256^3 for 500 steps would take 7 minutes)."""
    import torch
    case = wl.drop_3d(n, seed=0)
    s = ws.Solver(3, case.n, case.dx, case.bc, precision="mixed", stream=stream)
    warm = 3
    gap = max(0, (run_steps - warm - steps) // max(steps, 1))
    with torch.cuda.stream(stream):
        U = s.prim_to_cons(s.tensor(case.Q))
        del case
        ws.ws_autotune(s.ctx, U, 2)
        stage_cfg = ws.ws_get_stage_config(s.ctx)
        ws.ws_set_resident(s.ctx, True)  # consecutive steps carry the FP32 image
        for _ in range(warm):
            s.step(U)
        done = warm
        census = {k: 0 for k in ws.CENSUS_KEYS}
        Uc = torch.empty_like(U)
        # census replays in a context of their own, so that the timed context's
        # steps follow one another undisturbed
        sc = ws.Solver(3, (n, n, n), (1.0 / n,) * 3, (("periodic", "periodic"),) * 3, precision="mixed",
                       stream=stream)
        ws.ws_set_stage_config(sc.ctx, stage_cfg["index"])
        ms = 0.0
        ws.ws_profile(s.ctx, True)
        for k in range(steps):
            ws.ws_profile(s.ctx, False)
            for _ in range(gap):
                s.step(U)
            done += gap
            # census of the reconstruction's evaluations on a copy of the state
            # the timed step starts from
            Uc.copy_(U)
            c = sc.census_step(Uc)
            for key in ws.CENSUS_KEYS:
                census[key] += c[key]
            ws.ws_profile(s.ctx, True, reset=False)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(U)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            done += 1
        face_ms, face_n = ws.ws_profile_read(s.ctx)["face"]
        ws.ws_profile(s.ctx, False)
        del Uc
        sc.close()
        while done < run_steps:
            s.step(U)
            done += 1
        Q = s.cons_to_prim(U)
        sl = wl.interior(3, (n, n, n))
        dp = float((Q[sl][4] / 1e5 - 1.0).abs().max().item())
        del Q
        bad = s.nonphysical()
    s.close()
    del U
    torch.cuda.empty_cache()
    # L1 against the FP64 path
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
        Q64 = s64.cons_to_prim(U64)
        dp64 = float((Q64[sl][4] / 1e5 - 1.0).abs().max().item())
    s64.close()
    s32.close()
    del U64, U32, Q64
    torch.cuda.empty_cache()
    cells = n ** 3
    flops = 3 * stage_flops(3, (n, n, n)) * steps  # the method's flops of the timed steps
    achieved = flops / (face_ms * 1e-3) / 1e12
    flat = census["flat"] / max(census["face_variables"], 1)
    ex = executed_face_flops(3, flat)
    evaluated = census["face_variables"] / (7 * 3 * steps)  # faces evaluated per stage (tile edges twice)
    ex_achieved = (ex * evaluated + cells * (prim_flops(3) + divergence_flops(3))) * 3 * steps / (face_ms * 1e-3) / 1e12
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "run_steps": run_steps, "timed_steps": f"{steps} spread evenly over the {run_steps}-step run "
                                                  f"(after {warm} warm-up steps)",
            "workload": f"drop_3d_{n}^3 (periodic water drop r=0.25 in air, 1% density noise, seed 0), mixed",
            "l2": f"state {cells * 7 * 8 / 1e9:.2f} GB, larger than L2",
            "stage_config": stage_cfg,
            "gpu_launches": int(face_n),
            "roofline": {"bound": "alu", "kernel": "fused 3D RK stage, both passes", "achieved": achieved,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                         "flops_per_step": 3 * stage_flops(3, (n, n, n)),
                         "flops_source": f"the method's flops (op-counting build of the FP64 oracle): "
                                         f"{face_flops(3)} per face, {prim_flops(3) + divergence_flops(3)} per "
                                         "cell and stage",
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz",
                         "peak_probe_measured": probe, "frac_of_probe": achieved / probe,
                         "share_of_step": face_ms / ms,
                         "executed": {"achieved": ex_achieved, "frac": ex_achieved / FP32_PEAK_TFLOPS,
                                      "flops_per_face": ex, "faces_per_stage": evaluated,
                                      "flat_face_variable_fraction": flat,
                                      "warp_passes_running_weno_is":
                                          census["warp_passes_weno"] / max(census["warp_passes"], 1),
                                      "census": "ws_census_step on a copy of the state before each timed step"}},
            "pressure_equilibrium_max_rel_dev": {"after_steps": run_steps, "value": dp,
                                                 "what": "max |p/p0 - 1| over the cells (p0 = 1e5 Pa uniform)"},
            "nonphysical_cells": bad,
            "l1_density_vs_fp64": {"grid": [l1_n] * 3, "steps": l1_steps, "value": l1,
                                   "fp64_pressure_equilibrium_max_rel_dev": dp64,
                                   "reference": "FP64 path (bit-identical to the FP64 oracle), its CFL steps"}}


def time_learned(ws, stream, steps, n=2048, run_steps=4000, warmup=3, dt=4e-8, train_faces=10_000_000,
                 nograph=False):
    """The learned smooth-face gate on the shock-bubble at n^2 for run_steps
    steps: trained on the GPU by the library's kernels on about train_faces
    faces from plain runs of the 1D gas-water tube, the 1024^2 shock-bubble and
    the 3D drop, then timed like the plain mixed path (timed steps spread
    evenly over the run, L2 flushed between them) against the plain mixed path
    on the same fixed time steps; after the run, the L1 density difference
    between the gated and the plain states and the steps the gate redid
    plainly.  nograph: the contexts get no stream, so a gated step is a
    sequence of launches instead of one graph (profilers cannot look inside
    graphs with conditional nodes)."""
    import torch
    from paper_1707_00592_gb300 import learned
    t0 = time.perf_counter()
    P, thr, rep = learned.train_gate(total=train_faces, epochs=4)
    rep["train_s"] = time.perf_counter() - t0
    case = wl.shock_bubble_2d(n)
    outs = {}
    if nograph:  # the legacy default stream: no capture, so no graph
        stream = torch.cuda.default_stream()
    gap = max(0, (run_steps - warmup - steps) // max(steps, 1))
    for mode in ("plain", "gated", "gated_per_step"):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", stream=stream)
        if mode == "plain":
            ws.ws_set_resident(s.ctx, True)
        if mode == "gated":
            ws.ws_set_mlp(s.ctx, P, thr)
        elif mode == "gated_per_step":
            ws.ws_set_mlp(s.ctx, P, thr, ws.GATE_REDO_DRIFT | ws.GATE_REDO_NONPHYS | ws.GATE_PER_STEP)
        torch.cuda.nvtx.range_push(f"learned_{mode}")  # lets a profiler select one mode's launches
        with torch.cuda.stream(stream):
            U = s.prim_to_cons(s.tensor(case.Q))
            done = 0
            for _ in range(warmup):
                s.step(U, dt)
            done += warmup
            flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
            ms = 0.0
            for _ in range(steps):
                for _ in range(gap):
                    s.step(U, dt)
                done += gap
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(U, dt)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                done += 1
            while done < run_steps:
                s.step(U, dt)
                done += 1
            stats = ws.ws_gate_stats(s.ctx) if mode != "plain" else None
            bad = s.nonphysical()
        torch.cuda.nvtx.range_pop()
        outs[mode] = (U[wl.interior(2, case.n)][0].double().cpu(), ms / steps, stats, bad)
        s.close()
        del U, flush
        torch.cuda.empty_cache()
    b = outs["plain"][0]

    def summary(mode):
        a, ms_, st, bad = outs[mode]
        return {"ms_per_step": ms_, "l1_density_vs_plain_mixed": float((a - b).abs().sum() / b.abs().sum()),
                "gated_face_fraction": st["smooth_faces"] / max(st["faces"], 1.0), "steps_redone": st["redone"],
                "steps_gated": st["steps"], "nonphysical_cells": bad}

    per_step, per_stage = summary("gated_per_step"), summary("gated")
    plain_ms = outs["plain"][1]
    return {"value": case.cells / (per_step["ms_per_step"] * 1e-3), "unit": UNIT, **per_step,
            "workload": f"shock_bubble_2d_{n}x{n}, {run_steps} steps of fixed dt {dt:g} "
                        f"({steps} timed, spread evenly over the run)",
            "gate": "MLP once per step (RK stage 0), decisions reused in stages 1 and 2",
            "per_stage_mlp": per_stage, "plain_ms_per_step": plain_ms,
            "speedup_vs_plain": plain_ms / per_step["ms_per_step"],
            "training": rep, "dt": f"fixed {dt:g} for all runs (same trajectory)"}


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
        stage_cfg = None
        if args.precision == "mixed" and args.autotune:
            # the fused stage's tile shape and launch mode, chosen by timing
            # each candidate on a scratch copy of the initial state
            ws.ws_autotune(s.ctx, U0, args.autotune)
            stage_cfg = ws.ws_get_stage_config(s.ctx)
        if args.precision == "mixed" and args.resident:
            # consecutive steps of the run carry the FP32 image of the state
            # from one step's last stage to the next step's first (identical
            # results; the first step of the run converts the FP64 state)
            ws.ws_set_resident(s.ctx, True)
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
        # the census runs in a context of its own (same configuration), so
        # that the timed context's steps follow one another undisturbed
        sc = None
        if census is not None:
            sc = ws.Solver(2, case.n, case.dx, case.bc, precision=args.precision, stream=stream)
            if stage_cfg is not None:
                ws.ws_set_stage_config(sc.ctx, stage_cfg["index"])
        ws.ws_profile(s.ctx, True)
        with ClockSampler(dev) as clk:
            for k in range(args.steps):
                if gap:
                    ws.ws_profile(s.ctx, False)
                    for _ in range(gap):
                        s.step(U)
                    ws.ws_profile(s.ctx, True, reset=False)
                if census is not None:
                    Uc.copy_(U)
                    c = sc.census_step(Uc)
                    for key in ws.CENSUS_KEYS:
                        census[key] += c[key]
                    mood_counts += sc.mood()[0]  # the census step replays the timed step bit for bit
                flush.zero_()  # evict the state from L2 between timed steps
                ev[k][0].record(stream)
                s.step(U)
                ev[k][1].record(stream)
            stream.synchronize()
        del Uc
        if sc is not None:
            sc.close()
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
        # the host link: one state each way between pinned host memory and
        # the device, timed with events (the bound the end-to-end step sits on)
        link = {}
        Ud = torch.empty_like(U0)
        for name, dst, src in (("h2d_gbs", Ud, Uh), ("d2h_gbs", Uh, Ud)):
            dst.copy_(src, non_blocking=True)
            best = 1e30
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dst.copy_(src, non_blocking=True)
                b.record(stream)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            link[name] = state_bytes / (best * 1e-3) / 1e9
        del Ud

        l1 = None
        fp64_cmp = None
        if args.precision == "mixed" and args.l1_steps > 0:
            l1 = l1_vs_fp64(ws, case, s, stream, args.l1_steps)
        if args.precision == "mixed" and args.fp64_steps > 0:
            fp64_cmp = time_fp64(ws, case, stream, args.fp64_steps)
        tubes = (time_tubes(ws, stream, args.tube_steps, run_steps=args.tube_run_steps)
                 if args.tube_steps > 0 else None)
        setups = time_setups(ws, stream, args.setup_steps) if args.setup_steps > 0 and args.precision == "mixed" else None
        drop = None
        if args.drop_steps > 0 and args.precision == "mixed":
            p32 = args.fp32_peak if args.fp32_peak is not None else ws.ws_peak_probe("fp32")
            drop = time_drop3d(ws, stream, args.drop_steps, p32, n=args.drop_n, run_steps=args.drop_run_steps,
                               l1_n=args.drop_l1_n, l1_steps=args.drop_l1_steps)
        gate = (time_learned(ws, stream, args.steps, n=args.learned_n, run_steps=args.learned_run_steps,
                             train_faces=args.learned_train_faces, nograph=args.learned_nograph)
                if args.learned and args.precision == "mixed" else None)

    clocks = clk.summary()
    if rank != 0:
        if ws_size > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, which = load_peaks()
    face_ms, face_n = prof["face"]
    per_launch_s = face_ms * 1e-3 / max(face_n, 1)
    if args.precision == "fp64":
        # one face sweep per direction: the faces of one direction
        flops = face_flops(2) * (n + 1) * n
        peak, kname = FP64_PEAK_TFLOPS, "face sweep (FP64, one direction per launch)"
        psrc = "152 SMs x 2 FP64 lanes x 2 flops per DFMA x 2.07 GHz (unit counts, maximum SM clock)"
        probe = args.fp64_peak if args.fp64_peak is not None else ws.ws_peak_probe("fp64")
    else:
        # one fused launch is one RK stage: every face of both directions,
        # every cell's primitives and flux divergence
        flops = stage_flops(2, (n, n))
        peak, kname = FP32_PEAK_TFLOPS, "fused RK stage (FP32 mixed: tile load, x and y faces, update)"
        psrc = "152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (unit counts, maximum SM clock)"
        probe = args.fp32_peak if args.fp32_peak is not None else ws.ws_peak_probe("fp32")
    achieved = flops / per_launch_s / 1e12
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": STAGE2D_DRAM_BYTES if args.precision == "mixed" and n == 1024 else None,
                "traffic_source": STAGE2D_DRAM_SOURCE,
                "flops_per_launch": flops,
                "flops_source": f"the method's flops, from the op-counting build of the FP64 oracle: "
                                f"{face_flops(2)} per face ({2 * (n + 1) * n} faces), "
                                f"{prim_flops(2) + divergence_flops(2)} per cell ({n * n} cells) and stage",
                "peak_source": psrc, "peak_probe_measured": probe,
                "peak_probe_source": "dependent FMA chains on this GPU (ws_peak_probe), 2 flops per FMA",
                "frac_of_probe": achieved / probe,
                "ms_per_launch": per_launch_s * 1e3,
                "share_of_step": face_ms / ms,
                "hbm_bytes_per_cell_update": cell_update_bytes(2),
                "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": which}
    if census is not None and census["face_variables"]:
        # what the kernel executes: WENO-IS only where the stencil is not flat
        # (census of the timed steps' states), the linear weights elsewhere,
        # over every face evaluation (tile edges twice)
        flat = census["flat"] / census["face_variables"]
        ex = executed_face_flops(2, flat)
        evaluated = census["face_variables"] / (6 * 3 * args.steps)
        ex_achieved = (ex * evaluated + (n * n) * (prim_flops(2) + divergence_flops(2))) / per_launch_s / 1e12
        roofline["executed"] = {
            "achieved": ex_achieved, "frac": ex_achieved / peak, "flops_per_face": ex,
            "faces_per_launch": evaluated,
            "what": f"executed: WENO-IS ({WENO_FLOPS} flops a side) for face-variables with a non-flat stencil, "
                    f"the linear weights ({LINEAR_FLOPS} flops a side) for flat ones, over every face evaluation "
                    "(faces on tile edges twice); the flat test itself is not counted",
            "flat_face_variable_fraction": flat,
            "warp_passes_running_weno_is": census["warp_passes_weno"] / max(census["warp_passes"], 1),
            "census": f"ws_census_step on a copy of the state before each of the {args.steps} timed steps"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_size, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {**workload_config(args, ws_size), "precision": args.precision,
                       "stage_config": stage_cfg,
                       "resident": bool(args.resident and args.precision == "mixed")},
            "gpu_launches": launches,
            "kernel_ms": {k: v[0] for k, v in prof.items() if v[1]},
            "roofline": roofline,
            "e2e": {"value": cells / e2e_t, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "ms_per_step": e2e_t * 1e3,
                    "link": {**link, "copies_ms": 1e3 * state_bytes * (1 / link["h2d_gbs"] + 1 / link["d2h_gbs"]) / 1e9,
                             "what": "pinned host <-> device copy of one state, best of 5, CUDA events; the "
                                     "end-to-end step overlaps its banded copies with stages 0 and 2"}}}
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
    ap.add_argument("--l1-steps", type=int, default=2000)
    ap.add_argument("--run-steps", type=int, default=2000)
    ap.add_argument("--tube-steps", type=int, default=10)
    ap.add_argument("--drop-steps", type=int, default=10)
    ap.add_argument("--learned-nograph", action="store_true")
    ap.add_argument("--drop-n", type=int, default=256)
    ap.add_argument("--drop-run-steps", type=int, default=500)
    ap.add_argument("--drop-l1-n", type=int, default=128)
    ap.add_argument("--drop-l1-steps", type=int, default=500)
    ap.add_argument("--setup-steps", type=int, default=10)
    ap.add_argument("--autotune", type=int, default=10, help="steps per candidate of ws_autotune (0: default)")
    ap.add_argument("--resident", type=int, default=1, help="carry the FP32 image between steps (ws_set_resident)")
    ap.add_argument("--learned", type=int, default=1)
    ap.add_argument("--learned-n", type=int, default=2048)
    ap.add_argument("--learned-run-steps", type=int, default=4000)
    ap.add_argument("--learned-train-faces", type=int, default=10_000_000)
    ap.add_argument("--tube-run-steps", type=int, default=1000)
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
