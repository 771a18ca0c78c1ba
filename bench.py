#!/usr/bin/env python
"""Throughput of the PIC + Thomas-BMT step on GB300.

One step = the fused gather / Boris / spin / advance / Esirkepov kernel
(pic_push_deposit; in 3D3V by default in the binned layout, where it stores
every particle into its new tile's slot range), the Yee update
(pic_field_update), the tile sort every --sort-every steps (3D3V binned: a
re-bin every 64 steps; --compact for the compact layout sorted every 2) and,
every --diag-every steps, the FP64 Eq. (4) moments of every species
(accumulated inside the fused kernel).  Workloads:

  config2 (default)  3D3V laser-wakefield precision study: 512 x 256 x 256
                     cells (dx = lambda/20, dy = dz = lambda/8), 2 ppc
                     electrons at 0.003 n_c, LP laser a0 = 3
  config3            2D3V pre-polarised hydrogen: 4096 x 1024 cells
                     (dx = lambda/32), 8 + 8 ppc electrons and protons, CP a0 = 60
  config1            2D3V 256 x 128, 4 ppc, LP a0 = 4 (small; L2 resident)
  config5            gradient of the beam loss (energy-weighted polarization
                     above 50 MeV) by the adjoint: 1024 x 512, 8 ppc, 64-knot
                     density ramp, a0 = 5, --adj-steps steps with a checkpoint
                     every --checkpoint steps; adjoint time against a forward run
  config4            parameter scan: 256 independent 2D3V runs of uneven
                     sizes (128x64 .. 1024x512), densities, a0, ppc and
                     lengths (300-1500 steps), run to completion as one batch
                     (pic_batch_*, autotuned tiles and sort cadence) and, for
                     comparison, one after another through the single-run calls

Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Several GPUs run independent replicas (one per rank, launched by torchrun):
the step has no exchange between runs, so there is no collective on the
data path; ranks only meet at the barriers around the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "particle-steps/s (push+spin+deposit) and % HBM roofline, FP32 vs FP64 at stated error"
UNIT = "particle-steps/s"
# Algorithmic bytes of the fused kernel, the minimum the method moves: per
# particle read cell, offsets, u(3), s(3), w and write cell, offsets, u, s --
# 2D3V 40 + 36 = 76 B, 3D3V (one more offset) 44 + 40 = 84 B; per cell the E,
# B window (24 B) and the current added to J (12 B).  The cell word (read and
# written, 8 B) keeps its width in FP64; every other byte doubles.
BYTES_PER_PARTICLE = {2: 76, 3: 84}
FIXED_WIDTH_BYTES = 8
BYTES_PER_CELL = 36
# Bytes the binned 3D3V layout adds per particle (it writes every particle to
# the other buffer, so the weight and the id move with it: read id 4 B, write
# w and id 8 B).  Reported beside the roofline, not counted as algorithmic;
# the id (8 B) keeps its width in FP64, the weight (4 B) doubles.
LAYOUT_BYTES_BINNED = (8, 4)
# CPU samples of the workload (the oracle is slow): the CPU-baseline leg and
# the precision study run CPU_SAMPLE_STEPS steps of CPU_SAMPLE (10-30 s of
# oracle work); the reference arm runs every one of its --steps on REF_SAMPLE
# (a fraction of a second of oracle work per step)
CPU_SAMPLE = {2: {"ny": 32}, 3: {"nz": 4}}
REF_SAMPLE = {2: {"ny": 32}, 3: {"ny": 32, "nz": 4}}
CPU_SAMPLE_STEPS = 6
# tile-sort cadence of the compact layout: 2D3V every 64 steps (config 3 in
# its interaction phase: 36.3, 37.4, 38.0 G particle-steps/s sorted every 16,
# 32, 64 steps), 3D3V every 2 (the binned layout, its default, re-bins every 64)
DEFAULT_SORT_EVERY = {2: 64, 3: 2}
# 3D3V runs the binned layout by default (headroom %, least spare slots per
# tile range), re-binned every DEFAULT_REBIN_EVERY steps
DEFAULT_BINS = (25, 16)
DEFAULT_REBIN_EVERY = 64
# the fused kernel of each dimension and the sources its DRAM traffic depends
# on (the kernel, its headers, and the sort, whose in-tile order it reads in)
KERNEL = {2: ("k_step_fused", ("k_particles.cu", "pic_device.cuh", "pic_ptx.cuh", "k_sort.cu")),
          3: ("k_step_fused3", ("k_particles3.cu", "pic_device3.cuh", "pic_step3.cuh", "pic_device.cuh", "pic_ptx.cuh",
                                "k_sort.cu"))}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["config2", "config3", "config1", "config4", "config5", "precision",
                                           "window"],
                    default="config2")
    ap.add_argument("--prec-steps", type=int, default=2000, help="precision: steps of the FP32 and FP64 runs")
    ap.add_argument("--prec-cut-steps", type=int, default=200, help="precision: steps of the cut against the oracle")
    ap.add_argument("--prec-static", action="store_true",
                    help="precision: the box stays put (default: it co-moves with the pulse, as --workload window)")
    ap.add_argument("--adj-steps", type=int, default=1000, help="config5: run length of the adjoint")
    ap.add_argument("--checkpoint", type=int, default=50, help="config5: checkpoint interval")
    ap.add_argument("--scan-runs", type=int, default=256, help="config4: runs of the scan")
    ap.add_argument("--sort-every", type=int, default=0, help="0: 64 in 2D3V, 2 in 3D3V (64 binned)")
    ap.add_argument("--diag-every", type=int, default=10)
    ap.add_argument("--tile", type=int, nargs="+", default=None)
    ap.add_argument("--bins", type=int, nargs=2, default=None, metavar=("PCT", "EXTRA"),
                    help="3D3V binned layout: headroom percent and least spare slots per tile range "
                         "(default 25 16)")
    ap.add_argument("--compact", action="store_true", help="3D3V: the compact layout with periodic tile sorts")
    ap.add_argument("--ny", type=int, default=0, help="smaller ny for profiling captures")
    ap.add_argument("--nz", type=int, default=0, help="smaller nz (3D3V) for profiling captures")
    ap.add_argument("--precision", type=int, choices=[32, 64], default=32)
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=10, help="timed steps of the FP64 line (0: skip)")
    ap.add_argument("--window-cells", type=int, default=16,
                    help="window: cells a move of the co-moving window (a multiple of the tile width)")
    ap.add_argument("--window-steps", type=int, default=200,
                    help="config2: timed steps of the co-moving window leg (0: skip)")
    ap.add_argument("--window-at", type=float, default=0.75,
                    help="window: the box starts to move when the envelope peak reaches this fraction of nx")
    ap.add_argument("--start-step", type=int, default=-1,
                    help="untimed steps before the warm-up ends (-1: the laser-plasma interaction phase, "
                         "40 steps past the pulse peak's arrival at x = 0)")
    return ap.parse_args(argv)


def interaction_start(wl, dt):
    """First step of the laser-plasma interaction phase: 40 steps after the
    envelope peak reaches x = 0 (the plasma starts two cells later), when the
    front half of the pulse is already in the plasma."""
    if wl.pol == "none" or wl.a0 <= 0:
        return 0
    return int(math.ceil(wl.t_peak_periods * 2 * math.pi / dt)) + 40


def window_start(wl, dt, at):
    """Step at which the laser envelope's peak reaches x = at * nx; a window
    that starts there at the speed of light keeps the peak at that point."""
    dx = wl.dx_lambda * 2 * math.pi
    return int(math.ceil((wl.t_peak_periods * 2 * math.pi + at * wl.nx * dx) / dt))


def fused_bytes(dim, n_particles, cells, precision, binned):
    """(algorithmic bytes, layout bytes) of one fused-kernel launch."""
    wb = precision // 32
    alg = (FIXED_WIDTH_BYTES + (BYTES_PER_PARTICLE[dim] - FIXED_WIDTH_BYTES) * wb) * n_particles + \
        BYTES_PER_CELL * wb * cells
    lay = (LAYOUT_BYTES_BINNED[0] + LAYOUT_BYTES_BINNED[1] * wb) * n_particles if binned else 0
    return alg, lay


def workload(name, ny=0, nz=0):
    if name == "config4":  # one run of the scan stands for it where a single workload is needed
        return W.batch_scan(1)[0][0]
    if name == "config5":
        return W.CONFIG5
    if name == "window":
        name = "config2"
    wl = {"config1": W.CONFIG1, "config2": W.CONFIG2, "config3": W.CONFIG3}[name]
    if ny:
        wl = W.scaled(wl, ny=ny)
    if nz and wl.dim == 3:
        wl = W.scaled(wl, nz=nz)
    return wl


def n_cells(wl):
    return wl.nx * wl.ny * (wl.nz if wl.dim == 3 else 1)


# ---------------------------------------------------------------------------
# ranks: replicas only
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def combine(elapsed_s, units, world, device=None):
    """Whole-job numbers from every rank: the slowest rank's time and the sum
    of the units all ranks processed."""
    if world == 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_cost(wl, steps):
    """Work estimate of one scan run: cells x steps (field update) plus
    particles x steps (the particle step)."""
    cells = wl.nx * wl.ny * (wl.nz if wl.dim == 3 else 1)
    x0, x1 = (0, wl.nx) if wl.bc_x == "periodic" else (2, wl.nx - 2)
    particles = sum(sp.ppc for sp in wl.species) * (x1 - x0) * wl.ny * (wl.nz if wl.dim == 3 else 1)
    return (cells + particles) * steps


def balance_runs(runs, world):
    """Indices of the runs each rank takes: largest first, each to the rank
    with the least work so far (greedy longest-processing-time split)."""
    order = sorted(range(len(runs)), key=lambda r: -run_cost(*runs[r]))
    load = [0] * world
    share = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda i: (load[i], i))
        share[k].append(r)
        load[k] += run_cost(*runs[r])
    return [sorted(s) for s in share]


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        mx = [num(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash(dim):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL[dim][1]:
        with open(os.path.join(ROOT, "paper_2002_02211_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_record(dim, wl, binned=False):
    """dram bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source for this workload
    (and layout)."""
    p = os.path.join(ROOT, "profiles", KERNEL[dim][0] + ("_binned" if binned else "") + ".traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_hash(dim) or rec.get("workload", wl.name) != wl.name:
        return None
    return rec


# ---------------------------------------------------------------------------
# the oracle leg (CPU baseline and --impl reference)
# ---------------------------------------------------------------------------
def sample_workload(wl, table=None):
    cut = (table or CPU_SAMPLE)[wl.dim]
    return W.scaled(wl, **cut), ", ".join(f"{k}={v}" for k, v in cut.items())


def cpu_sample(wl, table=None, threads="single thread"):
    import oracle
    sample, cut = sample_workload(wl, table)
    parts = W.generate_particles(sample)
    sim = oracle.OracleSim(sample, parts)
    n = sum(len(p["x"]) for p in sim.p)
    shape = "x".join(str(v) for v in ((sample.nx, sample.ny, sample.nz) if wl.dim == 3 else (sample.nx, sample.ny)))
    desc = f"{wl.name} with {cut} ({shape} cells, {n} particles), FP64 C oracle, {threads}"
    return sim, n, desc


def run_oracle_steps(sim, steps):
    t0 = time.perf_counter()
    sim.step(steps)
    return time.perf_counter() - t0


def cpu_baseline(wl):
    """The oracle on a sample of the workload: its OpenMP build on every host
    core (the push and the Yee stages in parallel, the deposit serial; the
    same bits as the plain build) and, beside it, the plain build on one core."""
    import oracle
    with oracle.parallel() as nthreads:
        psim, n, pdesc = cpu_sample(wl, threads=f"OpenMP build, {oracle.threads()} threads")
        pdt = run_oracle_steps(psim, CPU_SAMPLE_STEPS)
    sim, n1, desc = cpu_sample(wl)
    dt = run_oracle_steps(sim, CPU_SAMPLE_STEPS)
    return {"value": n * CPU_SAMPLE_STEPS / pdt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{CPU_SAMPLE_STEPS} steps of {pdesc}", "seconds": round(pdt, 2),
            "single_thread": {"value": n1 * CPU_SAMPLE_STEPS / dt, "cores": 1, "seconds": round(dt, 2),
                              "sample": f"{CPU_SAMPLE_STEPS} steps of {desc}"}}, sim


def precision_study(pic, wl, oracle_sim, bins=None):
    """The CPU-baseline sample run on the GPU in FP32 and FP64: largest error
    of every particle against the FP64 oracle after the same steps, and the
    error of the Eq. (4) polarization of each species."""
    sample, cut = sample_workload(wl)
    parts = W.generate_particles(sample)
    pos = ("x", "y", "z") if wl.dim == 3 else ("x", "y")
    out = {}
    for prec in (32, 64):
        with pic.Simulation(pic.config_from_workload(sample, precision=prec, bins=bins)) as sim:
            for s, d in enumerate(parts):
                sim.set_particles(s, d)
            if sample.neutralizing_background:
                sim.capture_background()
            sim.step(CPU_SAMPLE_STEPS)
            du = ds = dx = dp = 0.0
            for s in range(len(parts)):
                g = sim.get_particles_f64(s)
                o = oracle_sim.p[s]
                live = g["ix"] >= 0
                ids = g["id"][live]
                ok = o["alive"][ids] > 0
                ids = ids[ok]
                sel = np.flatnonzero(live)[ok]
                un = np.maximum(np.sqrt(sum(o[k][ids] ** 2 for k in ("ux", "uy", "uz"))), 1e-3)
                du = max(du, float((np.sqrt(sum((g[k][sel] - o[k][ids]) ** 2 for k in ("ux", "uy", "uz"))) / un).max()))
                ds = max(ds, float(np.sqrt(sum((g[k][sel] - o[k][ids]) ** 2 for k in ("sx", "sy", "sz"))).max()))
                for a in pos:
                    dx = max(dx, float(np.abs(g["i" + a][sel] + g["o" + a][sel] - o[a][ids]).max()))
                gm = sim.polarization(s)
                om = oracle_sim.moments(s)
                dp = max(dp, float(np.abs(gm["P"] - om[:3]).max()))
            out[f"fp{prec}"] = {"u_rel_max": du, "s_abs_max": ds, "x_cells_max": dx, "P_abs_max": dp}
    out["sample"] = f"{CPU_SAMPLE_STEPS} steps of {wl.name} with {cut}, every particle"
    return out


def main_reference(args):
    rank, world, _ = dist_env()
    wl = workload(args.workload, args.ny, args.nz)
    if rank != 0:
        return
    import oracle
    with oracle.parallel() as nthreads:   # every host core; the plain build's bits
        sim, n, desc = cpu_sample(wl, REF_SAMPLE, threads=f"OpenMP build, {nthreads} threads")
        run_oracle_steps(sim, args.warmup)
        dt = run_oracle_steps(sim, args.steps)
    v = n * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{args.steps} steps of {desc}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main_ours(args):
    import torch

    import paper_2002_02211_gb300 as pic

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    wl = workload(args.workload, args.ny, args.nz)
    dim = wl.dim
    bins = None
    if dim == 3 and not args.compact:
        bins = tuple(args.bins) if args.bins else DEFAULT_BINS
    if args.sort_every <= 0:
        args.sort_every = DEFAULT_REBIN_EVERY if bins else DEFAULT_SORT_EVERY[dim]
    parts = W.generate_particles(wl)
    n_particles = sum(len(p["ix"]) for p in parts)
    cells = n_cells(wl)

    stream = torch.cuda.Stream(device=dev)
    cfg = pic.config_from_workload(wl, sort_every=args.sort_every, tile=args.tile,
                                   precision=args.precision, bins=bins)
    sim = pic.Simulation(cfg, stream=stream)
    for s, d in enumerate(parts):
        sim.set_particles(s, d)
    if wl.neutralizing_background:
        sim.capture_background()
    sim.sync()

    state = {"since_sort": 0, "k": 0, "sorts": 0}
    ev_pairs = []

    def one_step(record):
        if state["since_sort"] >= args.sort_every:
            sim.sort()
            state["since_sort"] = 0
            state["sorts"] += 1
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        sim.push_deposit()
        if record:
            e1.record(stream)
            ev_pairs.append((e0, e1))
        sim.field_update()
        state["since_sort"] += 1
        state["k"] += 1

    # a8: the Eq. (4) moments of every species are accumulated inside the
    # fused kernel every diag_every steps (no extra pass, no host sync)
    sim.set_diagnostics(args.diag_every)
    # untimed: the run is advanced to the laser-plasma interaction phase (the
    # last `warmup` of these steps are the warm-up proper)
    dt = sim.grid()[0]
    start_step = args.start_step if args.start_step >= 0 else interaction_start(wl, dt)
    start_step = max(start_step, args.warmup)
    for _ in range(start_step):
        one_step(False)
    sim.sync()

    clocks = ClockSampler(local)
    launches0 = sim.launch_count()
    sorts0 = state["sorts"]
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        one_step(True)
    end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    launches = sim.launch_count() - launches0
    sorts_in = state["sorts"] - sorts0
    sim.sync()
    diag_step, diag = sim.get_diagnostics()
    elapsed_raw = start.elapsed_time(end) * 1e-3

    # the tile sort (3D3V binned: the re-bin) runs every sort_every steps; when
    # the timed steps hold fewer sorts than their share, the missing share of a
    # measured sort is added to the time (never subtracted)
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sa.record(stream)
    sim.sort()
    sb.record(stream)
    torch.cuda.synchronize(dev)
    sort_s = sa.elapsed_time(sb) * 1e-3
    missing = max(0.0, args.steps / args.sort_every - sorts_in)
    elapsed = elapsed_raw + missing * sort_s

    fused_ms = np.array([a.elapsed_time(b) for a, b in ev_pairs])
    t_fused = float(fused_ms.mean()) * 1e-3
    # the fused kernel over the run, in tenths (the laser enters and heats the plasma)
    fused_trend = [round(float(c.mean()), 3) for c in np.array_split(fused_ms, min(10, len(fused_ms)))]
    tmax, units = combine(elapsed, n_particles * args.steps, world, dev)
    value = units / tmax

    peak, peak_kind = measured_hbm_peak()
    wb = args.precision // 32
    bytes_fused, bytes_layout = fused_bytes(dim, n_particles, cells, args.precision, bool(bins))
    achieved = bytes_fused / t_fused / 1e9
    tr = traffic_record(dim, wl, bool(bins)) if args.precision == 32 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": KERNEL[dim][0], "kernel_ms": t_fused * 1e3, "kernel_ms_by_tenth": fused_trend,
                "algorithmic_bytes": bytes_fused,
                "bytes_per_particle": BYTES_PER_PARTICLE[dim], "bytes_per_cell": BYTES_PER_CELL,
                "layout_bytes": bytes_layout,
                "layout_bytes_what": "binned layout: id read, w and id written per particle (not algorithmic)"
                                     if bins else None,
                "peak_source": f"{peak_kind} hbm_gbs"}
    timing = {"start_step": start_step, "timed_steps": [start_step, start_step + args.steps],
              "sorts_timed": sorts_in, "sort_ms": sort_s * 1e3,
              "sort_share_added_ms": missing * sort_s * 1e3, "elapsed_raw_ms": elapsed_raw * 1e3}

    # end to end through the C ABI with host buffers: upload the particle state
    # from pinned memory, one step, read back the Eq. (4) moments
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        pinned = []
        ptrs = []
        for d in parts:
            pp = {}
            keys = ("ix", "iy", "ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w", "id")
            keys += ("iz", "oz") if dim == 3 else ()
            for k in keys:
                t = torch.from_numpy(np.ascontiguousarray(d[k])).pin_memory()
                pinned.append(t)
                pp[k] = t.data_ptr()
            ptrs.append((len(d["ix"]), pp))
        h2d = sum(len(d["ix"]) * 4 * (14 if dim == 3 else 12) for d in parts)
        d2h = len(parts) * 7 * 8
        # the step's result: its Eq. (4) moments, summed in the fused kernel
        # (in-step diagnostics every step) and read back
        sim.set_diagnostics(1)
        barrier(world)
        torch.cuda.synchronize(dev)
        phase = []  # per step: events before the upload, after it, after the step
        moments = None
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            for s, (n, pp) in enumerate(ptrs):
                sim.set_particles_raw(s, n, pp)
            ev[1].record(stream)
            sim.push_deposit()
            sim.field_update()
            ev[2].record(stream)
            moments = sim.get_diagnostics()
            phase.append(ev)
        torch.cuda.synchronize(dev)
        te = time.perf_counter() - t0
        sim.set_diagnostics(args.diag_every)
        assert moments is not None and moments[1][0]["count"] > 0
        upload_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in phase]))
        step_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in phase]))
        # the tile sort inside the upload, timed alone on the uploaded state
        # (pic_sort re-sorts the same particles), so the host link's share
        # of the upload is the rest
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sa.record(stream)
        sim.sort()
        sb.record(stream)
        torch.cuda.synchronize(dev)
        sort_alone = sa.elapsed_time(sb)
        te, eu = combine(te, n_particles * args.e2e_steps, world, dev)
        e2e = {"value": eu / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": args.e2e_steps, "ms_per_step": te * 1e3 / args.e2e_steps,
               "breakdown_ms": {"upload": upload_ms, "of_which_sort": sort_alone,
                                "of_which_h2d_and_pack": upload_ms - sort_alone,
                                "h2d_GBps": h2d / ((upload_ms - sort_alone) * 1e-3) / 1e9
                                if upload_ms > sort_alone else None,
                                "step": step_ms},
               "what": "per step: pic_set_particles of every species from pinned host memory "
                       "(read in place by the upload kernel, then the tile sort), pic_push_deposit "
                       "with the Eq. (4) sums of every species in the fused kernel, pic_field_update, "
                       "pic_get_diagnostics (D2H of the moments); breakdown from CUDA events around "
                       "the upload and the step, the sort timed alone after the last upload"}

    sim.close()

    # FP64 instantiation of the same step on the same workload
    fp64 = None
    if args.precision == 32 and args.fp64_steps > 0:
        cfg64 = pic.config_from_workload(wl, sort_every=args.sort_every, tile=args.tile, precision=64, bins=bins)
        with pic.Simulation(cfg64, stream=stream) as s64:
            for s, d in enumerate(parts):
                s64.set_particles(s, d)
            if wl.neutralizing_background:
                s64.capture_background()
            s64.set_diagnostics(args.diag_every)
            s64.step(start_step)   # the same point of the run as the FP32 line
            s64.sync()
            barrier(world)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64.step(args.fp64_steps)
            b.record(stream)
            torch.cuda.synchronize(dev)
            t64, u64 = combine(a.elapsed_time(b) * 1e-3, n_particles * args.fp64_steps, world, dev)
            s64.sync()
        fp64 = {"value": u64 / t64, "unit": UNIT, "ms_per_step": t64 * 1e3 / args.fp64_steps,
                "steps": args.fp64_steps, "dtype": "f64",
                "timed_steps": [start_step, start_step + args.fp64_steps],
                "bound": "alu: the FP64 pipe, 75% of its peak busy at 4% of DRAM bandwidth "
                         "(profiles/k_step_fused3-fp64_3d3v-512x256x32.md)"}

    # config 2 with the co-moving window on (Sec. 2), timed from the step it starts
    win = None
    if dim == 3 and bins and args.window_steps > 0 and not (args.ny or args.nz):
        win = window_leg(pic, wl, args, stream, dev, world, args.window_steps, bins, args.sort_every)
        win.pop("particles", None)

    cpu = None
    study = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, orc_sample = cpu_baseline(wl)
        study = precision_study(pic, wl, orc_sample, bins)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == 32 else "f64",
                "data": "synthetic",
                "config": {"workload": wl.name,
                           "cells": [wl.nx, wl.ny] + ([wl.nz] if dim == 3 else []),
                           "particles": n_particles,
                           "species": [s.name for s in wl.species], "sort_every": args.sort_every,
                           "diag_every": args.diag_every, "tile": args.tile or "default",
                           "layout": ("binned (headroom %d%%, at least %d spare slots per tile)" % tuple(bins))
                                     if bins else "compact",
                           "l2": "inputs larger than L2 (particle state %.2f GB)"
                                 % (n_particles * (8 + (dim + 7) * 4 * wb) / 1e9),
                           "start_step": start_step,
                           "parallelism": f"replicas x{world}"},
                "timing": timing, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches, "fp64": fp64, "precision_study": study, "window": win,
                "diagnostics": {"step": diag_step,
                                "P": {sp.name: [round(v, 6) for v in d["P"]] for sp, d in zip(wl.species, diag)},
                                "ekin_mean_mev": {sp.name: d["ekin_mean"] for sp, d in zip(wl.species, diag)}}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# config4: the batched parameter scan against looped single runs
# ---------------------------------------------------------------------------
def main_scan(args):
    import torch

    import paper_2002_02211_gb300 as pic

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    # replicas: every rank runs its share of the scan, split by estimated work
    every_run = W.batch_scan(args.scan_runs)
    runs = [every_run[r] for r in balance_runs(every_run, world)[rank]]
    parts = [W.generate_particles(wl) for wl, _ in runs]
    stream = torch.cuda.Stream(device=dev)
    cfgs = [pic.config_from_workload(wl) for wl, _ in runs]
    work = sum(len(p[0]["ix"]) * n for p, (_, n) in zip(parts, runs))

    def load(sim, r):
        for s, d in enumerate(parts[r]):
            sim.set_particles(s, d)
        sim.capture_background()

    # batched: upload, autotune (its probe steps are real steps of the runs),
    # then every run to completion
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with pic.Batch(cfgs, [n for _, n in runs], stream=stream) as b:
        for r in range(len(runs)):
            load(b.run(r), r)
        stream.synchronize()
        t_up = time.perf_counter() - t0
        t0 = time.perf_counter()
        chosen = b.tune(4, tiles=((16, 8), (32, 8)), sorts=(16, 32, 64))
        done0 = b.steps_done()
        launches0 = b.launch_count()
        stream.synchronize()
        t_tune = time.perf_counter() - t0
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(10 ** 9)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        t_run = e0.elapsed_time(e1) * 1e-3
        launches = b.launch_count() - launches0
        t1 = time.perf_counter()
        pol = [b.run(r).polarization(0)["P"].tolist() for r in range(len(runs))]
        t_read = time.perf_counter() - t1
        tuned_work = sum(len(p[0]["ix"]) * d for p, d in zip(parts, done0))
    timed_work = work - tuned_work
    t_run, timed_work_all = combine(t_run, timed_work, world, dev)
    e2e_time, work_all = combine(t_up + t_tune + t_run + t_read, work, world, dev)

    # looped: the same runs one after another, each through pic_step
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r, (wl, n) in enumerate(runs):
        cfg = pic.config_from_workload(wl, sort_every=chosen[2], tile=chosen[:2])
        with pic.Simulation(cfg, stream=stream) as sim:
            load(sim, r)
            sim.step(n)
            sim.sync()
    t_loop = time.perf_counter() - t0
    t_loop, _ = combine(t_loop, 0, world, dev)

    if rank == 0:
        value = timed_work_all / t_run
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": max(n for _, n in runs),
                "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"batched scan of {args.scan_runs} 2D3V runs (seed 4)",
                           "runs_per_rank": len(runs), "particle_steps": work_all,
                           "tuned": {"tile": list(chosen[:2]), "sort_every": chosen[2]},
                           "l2": "inputs larger than L2",
                           "parallelism": f"replicas x{world} (runs split by cells x steps + particles x steps)"},
                "batched_s": t_run, "looped_single_runs": {"value": work_all / t_loop, "seconds": t_loop,
                                                           "what": "each run alone: pic_create, upload, pic_step"},
                "speedup_vs_looped": (work_all / t_loop) and value / (work_all / t_loop),
                "e2e": {"value": work_all / e2e_time, "unit": UNIT,
                        "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                        "what": "upload of every run's particles, autotune, all steps, Eq. (4) read-back"},
                "clocks": clk, "gpu_launches": launches,
                "P_first_runs": pol[:4]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# config5: the adjoint against forward runs
# ---------------------------------------------------------------------------
def main_adjoint(args):
    import torch

    import paper_2002_02211_gb300 as pic
    from paper_2002_02211_gb300.autograd import adjoint_forward_step

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    wl = W.CONFIG5
    parts = W.generate_particles(wl)
    parts[0]["w"] = W.ramp_weights(wl, parts, W.ramp_knots()).astype(np.float32)
    n = len(parts[0]["ix"])
    loss = dict(species=0, axis=1, e_cut_mev=50.0, e_width_mev=5.0)
    stream = torch.cuda.Stream(device=dev)
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    for prec in (32, 64):
        def fresh():
            sim = pic.Simulation(pic.config_from_workload(wl, precision=prec), stream=stream)
            sim.set_particles(0, parts[0])
            sim.capture_background()
            sim.sync()
            return sim

        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with fresh() as sim:            # production forward: fused kernel, tile sorts
            ev[0].record(stream)
            sim.step(args.adj_steps)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            t_fwd = ev[0].elapsed_time(ev[1]) * 1e-3
        with fresh() as sim:            # the adjoint's own forward steps (no sorts)
            ev[0].record(stream)
            for _ in range(args.adj_steps):
                adjoint_forward_step(sim)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            t_split = ev[0].elapsed_time(ev[1]) * 1e-3
        with fresh() as sim:
            barrier(world)
            t0 = time.perf_counter()
            value, dla0 = sim.adjoint(args.adj_steps, args.checkpoint, **loss)
            t_adj = time.perf_counter() - t0
            g = sim.adjoint_particle_grads(0)
        out[f"fp{prec}"] = {"forward_s": t_fwd, "forward_adjoint_path_s": t_split, "adjoint_s": t_adj,
                            "adjoint_over_forward": t_adj / t_fwd,
                            "adjoint_over_adjoint_path_forward": t_adj / t_split,
                            "loss": value, "dloss_da0": dla0,
                            "dloss_dw_abs_sum": float(np.abs(g["w"]).sum())}
        if prec == 64:
            # accuracy: the FP64 adjoint's dL/da0 against central differences
            # of the same forward path, on a 150-step horizon (the run's
            # sensitivity grows with the horizon: at 1000 steps the exact
            # derivative of the discrete run and any finite difference part)
            def loss_at(a0, steps):
                cfg = pic.config_from_workload(W.scaled(wl, a0=a0), precision=64)
                with pic.Simulation(cfg, stream=stream) as sim:
                    sim.set_particles(0, parts[0])
                    sim.capture_background()
                    for _ in range(steps):   # the adjoint's own forward steps
                        adjoint_forward_step(sim)
                    return sim.loss(**loss)

            acc = {"steps": 150}
            with fresh() as sim:
                acc["adjoint"] = sim.adjoint(150, args.checkpoint, **loss)[1]
            for h in (1e-4, 1e-8):
                acc[f"fd_h{h:g}"] = (loss_at(wl.a0 + h, 150) - loss_at(wl.a0 - h, 150)) / (2 * h)
            acc["rel_err_vs_fd_h1e-8"] = abs(acc["adjoint"] - acc["fd_h1e-08"]) / abs(acc["fd_h1e-08"])
            acc["long_horizon_fd_h1e-4"] = (loss_at(wl.a0 + 1e-4, args.adj_steps) -
                                            loss_at(wl.a0 - 1e-4, args.adj_steps)) / 2e-4
            out["fp64"]["accuracy"] = acc
    clk = clocks.stop()
    if rank == 0:
        r32 = out["fp32"]
        line = {"metric": METRIC, "value": n * args.adj_steps / r32["adjoint_s"], "unit": UNIT + " (adjoint)",
                "n_gpus": world, "steps": args.adj_steps, "warmup": 0, "ms_per_step": 1e3 * r32["adjoint_s"] / args.adj_steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "particles": n, "checkpoint_every": args.checkpoint,
                           "loss": loss, "parallelism": f"replicas x{world}"},
                "adjoint": out, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# config1: the small L2-resident run as the latency case, pic_step replayed
# from CUDA graphs against pic_step launching every kernel
# ---------------------------------------------------------------------------
def main_latency(args):
    import torch

    import paper_2002_02211_gb300 as pic

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    wl = workload(args.workload, args.ny, args.nz)
    parts = W.generate_particles(wl)
    n_particles = sum(len(p["ix"]) for p in parts)
    sort_every = args.sort_every if args.sort_every > 0 else DEFAULT_SORT_EVERY[wl.dim]
    stream = torch.cuda.Stream(device=dev)
    out = {}
    clk = None
    for mode, graphs in (("graphs", 32), ("launched", 0)):
        with pic.Simulation(pic.config_from_workload(wl, sort_every=sort_every, tile=args.tile), stream=stream) as sim:
            for s, d in enumerate(parts):
                sim.set_particles(s, d)
            if wl.neutralizing_background:
                sim.capture_background()
            sim.set_graphs(graphs)
            sim.set_diagnostics(args.diag_every)
            # warm-up: a whole sort cycle, so every graph the timed steps use is captured
            sim.step(max(args.warmup, 2 * sort_every))
            sim.sync()
            clocks = ClockSampler(local)
            l0 = sim.launch_count()
            g0 = sim.graph_stats()
            barrier(world)
            torch.cuda.synchronize(dev)
            clocks.start()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record(stream)
            sim.step(args.steps)
            b.record(stream)
            t_host = time.perf_counter() - t0
            torch.cuda.synchronize(dev)
            c = clocks.stop()
            if mode == "graphs":
                clk = c
            t, u = combine(a.elapsed_time(b) * 1e-3, n_particles * args.steps, world, dev)
            g1 = sim.graph_stats()
            out[mode] = {"value": u / t, "ms_per_step": 1e3 * t / args.steps,
                         "host_issue_ms_per_step": 1e3 * t_host / args.steps,
                         "kernels_per_step": (sim.launch_count() - l0) / args.steps,
                         "graph_launches_per_step": (g1[1] - g0[1] + g1[0] - g0[0]) / args.steps}
            sim.sync()
    if rank == 0:
        g = out["graphs"]
        line = {"metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": g["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "cells": [wl.nx, wl.ny], "particles": n_particles,
                           "sort_every": sort_every, "diag_every": args.diag_every,
                           "l2": "L2-resident (about 13 MB): the latency and graph case, not a roofline case",
                           "parallelism": f"replicas x{world}"},
                "pic_step": out, "graph_speedup": g["value"] / out["launched"]["value"],
                "clocks": clk, "gpu_launches": int(round(g["kernels_per_step"] * args.steps))}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# precision: the 3D3V laser-wakefield workload run in FP32 and in FP64 on the
# GPU from the same seeded state (Eq. 4 polarization and kinetic-energy
# moments compared every 10 steps), and a cut of it with the pulse in the
# plasma run beside the FP64 oracle
# ---------------------------------------------------------------------------
def _moments_run(pic, wl, parts, precision, steps, every, stream, bins, window=None):
    """Eq. (4) moments of species 0 every `every` steps of one run;
    window = (cells a move, fraction of nx where the envelope peak starts it)
    runs it co-moving."""
    import torch
    cfg = pic.config_from_workload(wl, sort_every=DEFAULT_REBIN_EVERY, precision=precision, bins=bins,
                                   window_cells=window[0] if window else 0)
    rows = []
    with pic.Simulation(cfg, stream=stream) as sim:
        for s, d in enumerate(parts):
            sim.set_particles(s, d)
        if wl.neutralizing_background:
            sim.capture_background()
        sim.set_diagnostics(every)
        if window:
            stage_window(sim, wl, parts, window[0], window_start(wl, sim.grid()[0], window[1]), steps)
        t0 = time.perf_counter()
        done = 0
        while done < steps:
            n = min(every, steps - done)
            sim.step(n)
            done += n
            st, d = sim.get_diagnostics()
            if st == done:
                m = d[0]
                rows.append((done, np.array(m["P"]), m["ekin_mean"], m["ekin_var"], m["count"]))
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
    return rows, seconds


def _cut_against_oracle(pic, oracle, steps, stream):
    """FP32 and FP64 GPU runs of a 512 x 32 x 8 cut of the workload (binned
    layout, default tiles) beside the FP64 oracle, from the step where the
    envelope peak is 30 steps from x = 0 (the laser at full amplitude from the
    first step, the plasma driven within a few steps)."""
    wl = W.scaled(W.CONFIG2, name="3d3v-512x32x8-cut-ppc2-lp-a0_3", ny=32, nz=8)
    parts = W.generate_particles(wl)
    sims = {}
    for prec in (32, 64):
        sim = pic.Simulation(pic.config_from_workload(wl, sort_every=DEFAULT_REBIN_EVERY, precision=prec,
                                                      bins=DEFAULT_BINS), stream=stream)
        for s, d in enumerate(parts):
            sim.set_particles(s, d)
        sims[prec] = sim
    dt = sims[32].grid()[0]
    start = int(round(wl.t_peak_periods * 2 * math.pi / dt)) - 30
    with oracle.parallel() as nthreads:
        orc = oracle.OracleSim(wl, parts, step=start)
        for sim in sims.values():
            sim.set_step(start)
            sim.capture_background()
        t0 = time.perf_counter()
        for sim in sims.values():
            sim.step(steps)
        orc.step(steps)
        t_orc = time.perf_counter() - t0
    om = orc.moments(0)
    p = orc.p[0]
    alive = p["alive"].astype(bool)
    un = np.maximum(np.sqrt(p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2), 1e-3)
    out = {"workload": wl.name, "steps": [start, start + steps], "particles": int(len(p["x"])),
           "oracle_threads": nthreads, "oracle_seconds": round(t_orc, 1),
           "hot_fraction_|u|>0.5": float(((un > 0.5) & alive).mean()),
           "oracle_P": om[:3].tolist(), "oracle_ekin_mean_mev": om[5]}
    for prec, sim in sims.items():
        g = sim.polarization(0)
        gp = sim.get_particles_f64(0)
        live = gp["ix"] >= 0
        ids = gp["id"][live]
        both = alive[ids]
        ids = ids[both]
        sel = np.flatnonzero(live)[both]
        du = np.sqrt(sum((gp[k][sel] - p[k][ids]) ** 2 for k in ("ux", "uy", "uz"))) / un[ids]
        ds = np.sqrt(sum((gp[k][sel] - p[k][ids]) ** 2 for k in ("sx", "sy", "sz")))
        dx = max(float(np.abs(gp["i" + a][sel] + gp["o" + a][sel] - p[a][ids]).max()) for a in ("x", "y", "z"))
        out[f"fp{prec}"] = {
            "P_abs_err": float(np.abs(np.array(g["P"]) - om[:3]).max()),
            "ekin_mean_rel_err": abs(g["ekin_mean"] - om[5]) / abs(om[5]),
            "ekin_var_rel_err": abs(g["ekin_var"] - om[6]) / abs(om[6]),
            "count_diff": int(g["count"] - om[4]),
            "u_rel_max": float(du.max()), "u_rel_median": float(np.median(du)),
            "s_abs_max": float(ds.max()), "x_cells_max": dx,
            "particles_over_1e-5_u": int((du > 1e-5).sum())}
        sim.close()
    return out


def main_precision(args):
    import torch

    import oracle
    import paper_2002_02211_gb300 as pic

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank != 0:
        return
    stream = torch.cuda.Stream(device=dev)
    wl = W.CONFIG2
    parts = W.generate_particles(wl)
    every = 10
    runs = {}
    window = None if args.prec_static else (args.window_cells, args.window_at)
    for prec in (32, 64):
        runs[prec] = _moments_run(pic, wl, parts, prec, args.prec_steps, every, stream, DEFAULT_BINS, window)
    r32, r64 = runs[32][0], runs[64][0]
    by_step = {}
    for (s32, p32, m32, v32, c32), (s64, p64, m64, v64, c64) in zip(r32, r64):
        assert s32 == s64
        by_step[s32] = {"dP": float(np.abs(p32 - p64).max()), "dmean": abs(m32 - m64) / abs(m64),
                        "dvar": abs(v32 - v64) / abs(v64) if v64 else 0.0, "dcount": c32 - c64,
                        "P64": p64.tolist(), "mean64": m64}
    steps = sorted(by_step)
    series = [[st, by_step[st]["dP"], by_step[st]["dmean"], by_step[st]["dvar"]] for st in steps[::10]]
    end = by_step[steps[-1]]
    cut = _cut_against_oracle(pic, oracle, args.prec_cut_steps, stream)
    line = {"metric": "precision study: FP32 against FP64 on the GPU, and the GPU against the FP64 oracle",
            "workload": wl.name, "steps": args.prec_steps, "diag_every": every,
            "co_moving_window": None if window is None else
            {"cells_per_move": window[0], "speed_c": 1.0,
             "start_step": window_start(wl, wl.cfl / math.sqrt(sum((1 / (d * 2 * math.pi)) ** 2 for d in
                                                                  (wl.dx_lambda, wl.dy_lambda, wl.dz_lambda))),
                                        window[1])},
            "fp32_seconds": round(runs[32][1], 2), "fp64_seconds": round(runs[64][1], 2),
            "fp32_vs_fp64": {"max_over_run": {"P_abs": max(by_step[s]["dP"] for s in steps),
                                              "ekin_mean_rel": max(by_step[s]["dmean"] for s in steps),
                                              "ekin_var_rel": max(by_step[s]["dvar"] for s in steps)},
                             "end_of_run": {"step": steps[-1], "P_abs": end["dP"], "ekin_mean_rel": end["dmean"],
                                            "ekin_var_rel": end["dvar"], "count_diff": end["dcount"],
                                            "P_fp64": end["P64"], "ekin_mean_mev_fp64": end["mean64"]},
                             "every_100_steps": {"columns": ["step", "P_abs", "ekin_mean_rel", "ekin_var_rel"],
                                                 "rows": series}},
            "cut_against_oracle": cut}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# window: config 2 with the co-moving window on the stepping path
# ---------------------------------------------------------------------------
def stage_window(sim, wl, parts, ncells, w0, end_step):
    """Turns the co-moving window on from step w0 (speed c, ncells cells a
    move) and stages the plasma of every move before step end_step: four
    seeded draws of the uncovered columns staged in turn, ids continuing
    after the initial particles'.  Returns the plasmas staged."""
    dt, dx = sim.grid()[:2]
    n_moves = max(0, int(math.ceil((end_step - w0) * dt / dx / ncells))) + 2
    draws = [W.injection_particles(wl, ncells, seed=900 + k) for k in range(min(4, n_moves))]
    next_id = [len(p["ix"]) for p in parts]
    for k in range(n_moves):
        slab = []
        for s, d in enumerate(draws[k % len(draws)]):
            e = dict(d)
            e["id"] = (d["id"] + next_id[s]).astype(np.int32)
            next_id[s] += len(d["ix"])
            slab.append(e)
        sim.stage_injection(slab)
    sim.set_window(ncells, w0, 1.0)
    return n_moves


def window_leg(pic, wl, args, stream, dev, world, steps, bins, sort_every):
    """Config 2 run the way Sec. 2 runs it: once the envelope peak reaches
    --window-at of the box, the box follows it at the speed of light, pic_step
    moving it --window-cells cells at a time (in the binned layout by
    relabelling whole tile columns) and taking in the plasma staged for each
    move.  Timed from the step the window starts, every step a pic_step(1)
    call bracketed by CUDA events, so the cost of a move is the difference
    between the steps that make one and the steps that do not."""
    import torch

    ncells = args.window_cells
    parts = W.generate_particles(wl)
    n_particles = sum(len(p["ix"]) for p in parts)
    cfg = pic.config_from_workload(wl, sort_every=sort_every, tile=args.tile, bins=bins, window_cells=ncells)
    sim = pic.Simulation(cfg, stream=stream)
    for s, d in enumerate(parts):
        sim.set_particles(s, d)
    sim.capture_background()
    sim.set_diagnostics(args.diag_every)
    dt = sim.grid()[0]
    w0 = max(window_start(wl, dt, args.window_at), args.warmup)
    n_moves = stage_window(sim, wl, parts, ncells, w0, w0 + steps)
    # untimed: the run up to the step the window starts (its last `warmup`
    # steps are the warm-up)
    sim.step(w0)
    sim.sync()

    clocks = ClockSampler(int(dev.index or 0))
    launches0 = sim.launch_count()
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs, moved = [], []
    start.record(stream)
    for _ in range(steps):
        w = sim.window()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(1)
        b.record(stream)
        evs.append((a, b))
        moved.append(sim.window() > w)
    end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    launches = sim.launch_count() - launches0
    sim.sync()
    diag_step, diag = sim.get_diagnostics()
    elapsed = start.elapsed_time(end) * 1e-3
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    moved = np.array(moved)
    out = {"left": sim.staged_injections(), "shift": sim.window(), "binned": sim.binned(0) if bins else False}
    sim.close()
    tmax, units = combine(elapsed, n_particles * steps, world, dev)
    plain = float(step_ms[~moved].mean()) if (~moved).any() else None
    with_move = float(step_ms[moved].mean()) if moved.any() else None
    return {"value": units / tmax, "unit": UNIT, "ms_per_step": tmax * 1e3 / steps, "steps": steps,
            "timed_steps": [w0, w0 + steps], "particles": n_particles,
            "window": {"cells_per_move": ncells, "speed_c": 1.0, "start_step": w0,
                       "peak_at_cell": round(args.window_at * wl.nx), "moves_timed": int(moved.sum()),
                       "cells_moved_total": out["shift"], "step_ms_without_move": plain,
                       "step_ms_with_move": with_move,
                       "move_ms": (with_move - plain) if plain is not None and with_move is not None else None,
                       "plasma_staged": n_moves, "plasma_left": out["left"], "binned_at_end": out["binned"]},
            "clocks": clk, "gpu_launches": launches,
            "diagnostics": {"step": diag_step,
                            "P": {sp.name: [round(v, 6) for v in d["P"]] for sp, d in zip(wl.species, diag)}},
            "note": "value counts the particles at the start; a move removes and injects equal plasma volumes"}


def main_window(args):
    """Config 2 co-moving (window_leg) as its own JSON line."""
    import torch

    import paper_2002_02211_gb300 as pic

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    wl = workload("config2", args.ny, args.nz)
    bins = None if args.compact else (tuple(args.bins) if args.bins else DEFAULT_BINS)
    sort_every = args.sort_every if args.sort_every > 0 else (DEFAULT_REBIN_EVERY if bins else DEFAULT_SORT_EVERY[3])
    stream = torch.cuda.Stream(device=dev)
    leg = window_leg(pic, wl, args, stream, dev, world, args.steps, bins, sort_every)
    if rank == 0:
        line = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name + "-comoving", "cells": [wl.nx, wl.ny, wl.nz],
                           "particles": leg["particles"], "sort_every": sort_every,
                           "layout": ("binned (headroom %d%%, at least %d spare slots per tile)" % tuple(bins))
                                     if bins else "compact",
                           "l2": "inputs larger than L2", "start_step": leg["window"]["start_step"],
                           "parallelism": f"replicas x{world}"},
                "window": leg["window"], "timing": {"timed_steps": leg["timed_steps"]},
                "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": leg["clocks"],
                "gpu_launches": leg["gpu_launches"], "diagnostics": leg["diagnostics"], "note": leg["note"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        main_reference(args)
    elif args.workload == "window":
        main_window(args)
    elif args.workload == "config1":
        main_latency(args)
    elif args.workload == "precision":
        main_precision(args)
    elif args.workload == "config4":
        main_scan(args)
    elif args.workload == "config5":
        main_adjoint(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
