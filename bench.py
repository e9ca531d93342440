#!/usr/bin/env python
"""Benchmark of the GB300 WCSPH particle loop.

A step is one pass of the whole per-timestep hot path over the workload: drift + cell
keys, radix sort, reorder + EOS shadow, cell table, density pass (neighbour scan and list,
continuity or summation density, EOS), momentum pass with the corrector kick and the FP64
reductions (one captured CUDA graph). Default workload: the 3D dam break of the scale
configuration (2,000,000 fluid + 906,828 wall particles, Wendland C2, FP32 pair loops with
an FP64 integrator, neighbour rebuild every step), the largest configuration that runs on
one GPU. Inputs are resident in HBM; L2 is flushed (a 512 MB write) between timed steps
when the state fits in L2 (the small workloads), and not when the state alone is larger
than L2 (the 3D dam break, the batch).

Prints one JSON line. ``--impl reference`` times the CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "neighbour-pair interactions/s and particle-steps/s, FP32 vs FP64 at stated error"
UNIT = "neighbour-pair interactions/s"
# steps of the timed adjoint (gradient of the final kinetic energy) per workload
ADJOINT_STEPS = {"taylor_green_3d": 50, "dam_break_3d": 20}
FP32_LANES_PER_SM = 128   # FP32 CUDA-core lanes per Blackwell SM (4 sub-partitions x 32)
STATE_BYTES_PER_PARTICLE = 124  # one copy of the FP64 state (x, u, rho, m, rates, tag)


def sm_max_mhz(clocks: dict):
    """The SM clock ceiling: nvidia-smi's clocks.max.sm sampled during the run, else the
    figure MEASURED_PEAKS.json records for this pool; (MHz, source)."""
    if clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"]), "clocks.max.sm sampled during the run"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, ValueError, KeyError, TypeError):
        return None, "unknown"


def workload(name: str, wall_bc: str = "density", integrator: str = "kdk"):
    """The workload, or for the batched configuration the list of its instances; with
    wall_bc "adami" the solid-wall pressure condition replaces the continuity walls, with
    integrator "pec" the midpoint predict-evaluate-correct form replaces kick-drift-kick."""
    import workloads as W
    table = {
        "dam_break_2d": lambda: W.dam_break_2d(),
        "taylor_green_2d": lambda: W.taylor_green_2d(),
        # Sec. 4.1's run: EDAC, 100^2, h = 1.2 dx, Re = 100, to t = 2 s
        "taylor_green_2d_edac": lambda: W.taylor_green_2d_edac(),
        "taylor_green_3d": lambda: W.taylor_green_3d(),
        "dam_break_3d": lambda: W.dam_break_3d(),
        # the same tank at twice the spacing (~0.48 M particles): the size for ncu captures
        "dam_break_3d_dx01": lambda: W.dam_break_3d(dx=0.01),
        "batch_tg2d": lambda: W.batch_tg2d(),
        "falling_cube_3d": lambda: W.falling_cube_3d(),
    }
    wl = table[name]()
    if wall_bc == "adami":
        wl = [w.with_wall_bc(1) for w in wl] if isinstance(wl, list) else wl.with_wall_bc(1)
    if integrator == "pec":
        wl = [w.with_integrator(1) for w in wl] if isinstance(wl, list) else wl.with_integrator(1)
    return wl


class BatchView:
    """The attributes of a batch that the reporting reads from a single workload."""

    def __init__(self, wls):
        w0 = wls[0]
        self.instances = wls
        self.name = f"batch_tg2d_{len(wls)}"
        self.dim, self.kernel, self.precision = w0.dim, w0.kernel, w0.precision
        self.density, self.alpha, self.xsph_eps, self.nu = w0.density, w0.alpha, w0.xsph_eps, w0.nu
        self.h, self.dt = w0.h, w0.dt
        self.n_total = sum(w.n_total for w in wls)
        self.n_fluid = sum(w.n_fluid for w in wls)


class Runner:
    """One problem (Simulation) or a batch of them (BatchSimulation) behind the same calls."""

    def __init__(self, G, wl):
        self.G = G
        self.batch = isinstance(wl, list)
        if self.batch:
            self.sim = G.BatchSimulation(wl)
            self.sch = [G.scheme_of(w) for w in wl]
            self.dts = [w.dt for w in wl]
        else:
            self.sim = G.Simulation.from_workload(wl)
            self.sch = G.scheme_of(wl)
            self.dt = wl.dt
        self.stream = self.sim.stream
        self.n = self.sim.n

    def step(self, k):
        if self.batch:
            self.sim.step_batch(self.sch, self.dts, k)
        else:
            self.sim.step(self.sch, self.dt, k)

    def step_async(self, k):
        if self.batch:
            self.sim.step_batch_async(self.sch, self.dts, k)
        else:
            self.sim.step_async(self.sch, self.dt, k)

    def counts(self):
        """Interacting pairs, candidates and wall-destination pairs of the last step."""
        if self.batch:
            d = self.sim.batch_diagnostics()
            return float(d[:, 8].sum()), float(d[:, 9].sum()), float(d[:, 12].sum())
        d = self.sim.diagnostics()
        return float(d[8]), float(d[9]), float(d[12])

    def autotune(self):
        return self.sim.autotune(None if self.batch else self.sch)

    def kernels_per_step(self):
        return self.sim.kernels_per_step(self.sch[0] if self.batch else self.sch)

    def __getattr__(self, name):  # set_step_mode, tuning, set_timing, phase_times, ...
        return getattr(self.sim, name)


def describe(wl) -> dict:
    if isinstance(wl, BatchView):
        ns = [w.n_total for w in wl.instances]
        return {
            "workload": f"{wl.name}: {len(ns)} independent 2D Taylor-Green instances of "
                        f"{min(ns):,}-{max(ns):,} particles ({wl.n_total:,} in all), quintic "
                        f"h=dx, Re in [50, 1000], FP32 pair loops / FP64 integrator, one "
                        f"batched step for all instances, neighbour rebuild every step"
                        + (", midpoint predict-evaluate-correct integrator (two neighbour "
                           "builds and evaluations per step)"
                           if getattr(wl.instances[0], "integrator", 0) else ""),
            "particles": wl.n_total,
            "fluid_particles": wl.n_fluid,
            "l2": "no flush: the working set (~500 MB) exceeds L2",
            "parallelism": "replicas (one independent batch per GPU)",
        }
    kern = {0: "quintic spline", 1: "Wendland C2", 2: "cubic spline"}[wl.kernel]
    prec = "FP32 pair loops / FP64 integrator" if wl.precision == 1 else "FP64"
    return {
        "workload": f"{wl.name}: {wl.n_fluid:,} fluid + {wl.n_total - wl.n_fluid:,} wall particles, "
                    f"{wl.dim}D, {kern} h={wl.h:g}, {prec}, alpha={wl.alpha:g}, xsph={wl.xsph_eps:g}, "
                    f"nu={wl.nu:g}, dt={wl.dt:.6g}, neighbour rebuild every step"
                    + (", solid-wall pressure of Adami et al." if getattr(wl, "wall_bc", 0) else "")
                    + (", midpoint predict-evaluate-correct integrator (two neighbour builds "
                       "and evaluations per step)" if getattr(wl, "integrator", 0) else "")
                    + (", EDAC pressure equation (density held at rho0)"
                       if getattr(wl, "density", 0) == 2 else ""),
        "particles": wl.n_total,
        "fluid_particles": wl.n_fluid,
        "l2": ("flushed between timed steps (512 MB write)"
               if STATE_BYTES_PER_PARTICLE * wl.n_total <= (129 << 20) else
               f"no flush: the FP64 state alone ({STATE_BYTES_PER_PARTICLE * wl.n_total / 1e6:.0f} "
               f"MB) exceeds L2"),
        "parallelism": "replicas (one independent problem per GPU)",
        **({"pairs_counted": "end-of-step evaluation only (the midpoint evaluation of each "
                             "step is not counted)"} if getattr(wl, "integrator", 0) else {}),
        **({"paper_context": "Sec. 4.4 reports the pair-loop kernel of its GPU backend on "
                             "this problem (a free-falling cube of water) at about 180 GFLOP/s "
                             "FP32 and 80 GFLOP/s FP64 on a Tesla T4: other hardware, for "
                             "context; roofline.achieved is the same kind of figure here"}
           if wl.name.startswith("falling_cube") else {}),
    }


# --------------------------------------------------------------------- flops
def kernel_flops(wl) -> tuple[int, int]:
    """Flops of f(q) = w'(q)/q and of w(q) as the kernels evaluate them."""
    return {0: (12, 14), 1: (5, 6), 2: (6, 8)}[wl.kernel]


def pass_flops(wl) -> dict:
    """Algorithmic FP32 operations (add, sub, mul, div, sqrt = 1; a Neumaier compensated
    add = 4) per unit of each pair pass, counted from the operations the passes perform:
    density pass: per candidate (separation + squared distance), per listed pair
    (continuity rate or summation term); momentum pass: per fluid-destination pair
    (pressure, viscosity or AV, XSPH on fluid sources), per wall-destination pair 0."""
    d = wl.dim
    kf, kw = kernel_flops(wl)
    sep = 3 * d - 1                                   # differences, squares, sum
    cand = sep                                        # + compare
    if wl.density == 1:                               # summation: m W, compensated add
        listed = sep + 2 + kw + 2 + 4
    else:                                             # continuity: m Gk (v_ij . r_ij)
        listed = sep + 2 + kf + 1 + (3 * d - 1) + 2 + 4
    mom = sep + 2 + kf + 1 + d + 1 + 2 + 2            # q, Gk, v_ij, Pr_i+Pr_j, rhobar, cg
    if wl.alpha:
        mom += 0.5 * ((2 * d - 1) + 3 + 3)            # AV on approaching pairs (about half)
    if wl.nu:
        mom += 7 + d * 2                              # laminar coefficient and cv v_ij
    mom += d * (2 + 4)                                # cg dx (+cv v), compensated add
    xsph = (kw + 1 + 3 + d * (1 + 4)) if wl.xsph_eps else 0
    return {"candidate": cand, "listed_pair": listed, "fluid_dest_pair": mom,
            "xsph_fluid_source_pair": xsph}


def stream_bytes(wl, ncells: int) -> dict:
    """Algorithmic DRAM bytes of one step's streaming kernels (in-step form; 8-byte FP64
    state words, d = dimension). keys (drift + cell key + histograms): a fluid particle
    reads x, u, a, xsph and the tag and writes x and the key, a wall reads x and the tag
    and writes the key; each radix pass reads and writes a (key, index) pair; the reorder
    reads the permutation, the key and the state it gathers (tag, x, u, rho, m, and a for
    fluid), writes x, u, rho, m, tag and the shadow P, Q (2 x 16 B FP32, 2 x 32 B FP64),
    and reads and writes one 4-byte offset per cell."""
    d = wl.dim
    n, nf = wl.n_total, wl.n_fluid
    shadow = 32 if wl.precision == 1 else 64
    bits = max(0, (max(ncells, 1) - 1).bit_length())
    passes = max(1, (bits + 7) // 8)
    keys = nf * (4 * d * 8 + 4 + d * 8 + 4) + (n - nf) * (d * 8 + 4 + 4)
    reorder = (n * (4 + 4 + 4 + 2 * d * 8 + 16) + nf * d * 8
               + n * (2 * d * 8 + 16 + 4 + shadow) + ncells * 8)
    return {"keys": keys, "sort": passes * n * 16, "reorder": reorder, "passes": passes}


# ------------------------------------------------------------ ncu traffic
PAIR_KERNEL_SOURCES = ("sph_device.cuh", "sph_launch.h", "step_impl.cuh", "reduce_impl.cuh",
                       "pairs_impl.cuh", "pair_units.h", "pairs.cu") + tuple(
                           f"pairs_{p}_t{t}.cu" for p in ("f32", "f64") for t in (1, 2, 4, 8))


def source_hash() -> str:
    """Hash of the pair kernels' sources; ncu figures taken from other kernels are not
    reported."""
    import hashlib
    d = os.path.join(ROOT, "paper_1909_04504_gb300", "csrc")
    h = hashlib.sha256()
    for f in PAIR_KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def measured_traffic(workload_name: str, kernel: str, lanes: int):
    """DRAM bytes (read + write) per launch of `kernel` at `lanes` lanes per destination
    from the committed ncu summary, or None when the kernels changed since the capture or
    no capture used that shape."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != source_hash():
        return None
    return t.get(workload_name, {}).get(kernel, {}).get(str(lanes))


# --------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index: str):
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_index, f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ whole-job totals
def job_totals(dist, total_ms: float, units: float, device="cpu"):
    """The whole job's view of one timed region: the slowest rank's time and the units all
    ranks processed (each rank runs its own replica: weak scaling, no data-path collective)."""
    if dist is None:
        return total_ms, units
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------ GPU arm
def gpu_arm(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_1909_04504_gb300 as G

    dev = torch.cuda.current_device()
    raw = workload(args.workload, args.wall_bc, args.integrator)
    wl = BatchView(raw) if isinstance(raw, list) else raw
    sim = Runner(G, raw)
    sch = sim.sch
    stream = sim.stream
    sim.step(args.warmup)
    if args.step_mode == "auto":
        sim.autotune()  # tile shape and step form (graph of phases / persistent launch)
    else:
        sim.set_step_mode(G.STEP_PERSISTENT if args.step_mode == "persistent" else G.STEP_GRAPH)
    if args.lanes:
        sim.set_groups(args.lanes)  # both passes (after the autotuner, which it overrides)
    sim_lanes, sim_mode, density_lanes = sim.tuning()
    mode = "persistent" if sim_mode == G.STEP_PERSISTENT else "graph"
    sim.step(3)
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or 0) or (129 << 20)
    # inputs larger than L2 need no flush between steps: the state alone exceeds it
    flush_each = (not sim.batch) and STATE_BYTES_PER_PARTICLE * sim.n <= l2_bytes
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    counts = [0.0, 0.0, 0.0]  # interacting pairs, candidates, wall-destination pairs
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        uuid = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    # ---- timed region: K steps, L2 flushed before each, CUDA events on the step stream
    for k in range(args.steps):
        if flush_each:
            with torch.cuda.stream(stream):
                flush.zero_()
        e0[k].record(stream)
        sim.step_async(1)
        e1[k].record(stream)
        dg = sim.counts()  # waits for the step (outside the events)
        for q in range(3):
            counts[q] += dg[q]
    sim.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    # ---- kernel durations: the same steps with events recorded between the phases inside
    # the step (graph event nodes / phase-end stamps of the persistent kernel)
    sim.set_timing(True)
    phases = {k: 0.0 for k in G.Simulation.PHASES}
    pcounts = [0.0, 0.0, 0.0]
    psteps_n = min(args.steps, 200)
    for k in range(psteps_n):
        if flush_each:
            with torch.cuda.stream(stream):
                flush.zero_()
        sim.step_async(1)
        ph = sim.phase_times()  # waits for the step
        for key in phases:
            phases[key] += ph[key]
        dg = sim.counts()
        for q in range(3):
            pcounts[q] += dg[q]
    sim.set_timing(False)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    total_ms = sum(step_ms)
    pairs, cand, wall_pairs = counts
    n = sim.n
    total_ms, job_pairs = job_totals(dist, total_ms, pairs, device=dev)
    _, job_cand = job_totals(dist, total_ms, cand, device=dev)
    _, job_psteps = job_totals(dist, total_ms, float(n) * args.steps, device=dev)
    value = job_pairs / (total_ms / 1e3)
    psteps = job_psteps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (the longer pair pass), algorithmic flops over
    # its live duration (CUDA events recorded on the launching stream inside the graph)
    fl = pass_flops(wl)
    p_pairs, p_cand, p_wall = pcounts
    listed = p_pairs  # interacting pairs (summation also lists wall-wall pairs: not counted)
    fluid_pairs = p_pairs - p_wall
    fluid_src_frac = wl.n_fluid / wl.n_total        # XSPH sources: fluid share (estimate)
    flops = {"density": (fl["candidate"] * p_cand + fl["listed_pair"] * listed) / psteps_n,
             "momentum": (fl["fluid_dest_pair"] * fluid_pairs
                          + fl["xsph_fluid_source_pair"] * fluid_pairs * fluid_src_frac) / psteps_n}
    mhz, mhz_source = sm_max_mhz(clocks)
    peak = sms * FP32_LANES_PER_SM * 2 * (mhz or 0.0) * 1e6 / 1e12
    if wl.precision == 0:
        peak = peak / 64.0  # FP64 CUDA-core rate of this part: 1/64 of FP32
    per_pass = {}
    for k in ("density", "momentum"):
        ms = phases[k] / psteps_n
        ach = flops[k] / (ms / 1e3) / 1e12
        per_pass[k] = {"avg_launch_ms": round(ms, 5), "flops_per_launch": flops[k],
                       "achieved_tflops": round(ach, 4),
                       "frac": round(ach / peak, 5) if peak > 0 else None}
    dom = max(per_pass, key=lambda k: per_pass[k]["avg_launch_ms"])
    names = {"density": "k_density (neighbour scan + list, continuity/summation, EOS)",
             "momentum": "k_momentum (pressure, AV/viscosity, XSPH, corrector kick, reductions)"}
    roofline = {"bound": "alu", "achieved": per_pass[dom]["achieved_tflops"],
                "peak": round(peak, 3), "unit": "TFLOP/s", "frac": per_pass[dom]["frac"],
                "traffic": measured_traffic(args.workload, "k_" + dom,
                                            sim_lanes if dom == "momentum" else density_lanes),
                "kernel": names[dom],
                "flops_per_launch": flops[dom], "avg_launch_ms": per_pass[dom]["avg_launch_ms"],
                "peak_source": f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flop x "
                               f"{mhz} MHz ({mhz_source})"
                               + (" / 64 (FP64)" if wl.precision == 0 else ""),
                "passes": per_pass}
    phase_avg = {k: round(v / psteps_n, 5) for k, v in phases.items()}
    # the streaming kernels against the measured HBM copy bandwidth
    _, _, ncells = sim.grid()
    sb = stream_bytes(wl, int(ncells))
    hbm = measured_hbm_gbs()
    streaming = {}
    for k in ("keys", "sort", "reorder"):
        ms = phases[k] / psteps_n
        gbs = sb[k] / (ms / 1e3) / 1e9
        streaming[k] = {"bytes_per_step": sb[k], "avg_ms": round(ms, 5), "achieved_gbs": round(gbs, 1),
                        "frac": round(gbs / hbm, 4) if hbm else None}
    roofline["streaming"] = {"peak_gbs": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                             "sort_passes": sb["passes"], "kernels": streaming,
                             "note": "phase times include ~2-3 us of event-node gaps each"}

    # ---- end to end through the C ABI with host buffers: every step loads the state from
    # pinned host memory, steps, and reads the stepped state and the diagnostics back. Two
    # contexts of the same problem take the steps in turn, each on its own stream with the
    # asynchronous load and save, so that one's copies overlap the other's step (the copy
    # engines, not the step, bound a step that moves the whole FP64 state both ways)
    nbytes = sim.state_bytes()
    pinned = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()
    results = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
    sim.save_state_into(pinned)
    e2e_steps = min(args.steps, 100)
    sim.set_timing(False)
    sim2 = Runner(G, raw)  # created after the autotuner: the same tile shape and step form
    if args.step_mode != "auto":
        sim2.set_step_mode(G.STEP_PERSISTENT if args.step_mode == "persistent" else G.STEP_GRAPH)
    if args.lanes:
        sim2.set_groups(args.lanes)
    ctxs = (sim, sim2)
    for s_ in ctxs:
        s_.load_state(pinned)
        s_.step(1)  # captures the step without timing events
    tt = time.perf_counter()
    e2e_pairs = 0.0
    pending = [False, False]
    for k in range(e2e_steps):
        s_ = ctxs[k & 1]
        if pending[k & 1]:
            s_.synchronize()
            e2e_pairs += s_.counts()[0]
        s_.load_state_async(pinned)
        s_.step_async(1)
        s_.save_state_into_async(results[k & 1])
        pending[k & 1] = True
    for b in (0, 1):
        if pending[b]:
            ctxs[b].synchronize()
            e2e_pairs += ctxs[b].counts()[0]
    e2e_s = time.perf_counter() - tt
    sim2.close()
    e2e_ms, e2e_job_pairs = job_totals(dist, e2e_s * 1e3, e2e_pairs, device=dev)
    e2e = {"value": e2e_job_pairs / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes + 8 * G.DIAG_COUNT,
           "steps": e2e_steps,
           "contexts": 2,
           "path": "sph_load_state_async(pinned host state) + sph_step_async + "
                   "sph_save_state_async(pinned host buffer: the stepped state) + sph_synchronize "
                   "+ sph_diagnostics per step, two contexts of the problem in turn (one's copies "
                   "overlap the other's step), host clock"}

    # ---- FP64 mode of the same workload (the metric compares FP32 with FP64)
    fp64 = None
    if wl.precision == 1 and args.fp64_steps > 0 and not sim.batch:
        sim64 = G.Simulation.from_workload(wl.with_precision(0))
        sim64.step(sch, wl.dt, args.warmup)
        if args.step_mode == "auto":
            sim64.autotune(sch)
        else:
            sim64.set_step_mode(G.STEP_PERSISTENT if args.step_mode == "persistent" else G.STEP_GRAPH)
        f0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps)]
        f1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps)]
        p64 = 0.0
        for k in range(args.fp64_steps):
            with torch.cuda.stream(sim64.stream):
                flush.zero_()
            f0[k].record(sim64.stream)
            sim64.step_async(sch, wl.dt, 1)
            f1[k].record(sim64.stream)
            sim64.synchronize()
            p64 += sim64.diagnostics()[8]
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in zip(f0, f1))
        ms64, p64 = job_totals(dist, ms64, p64, device=dev)
        v64 = p64 / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps,
                "fp32_speedup": round(value / v64, 3)}
        sim64.close()

    # ---- the batch against its alternatives: the same instances with FP64 pair loops, and
    # as separate problems (one context and stream each, every step launched before any wait)
    batch_vs = None
    if sim.batch and args.fp64_steps > 0:
        rounds = max(3, min(args.fp64_steps, 50))
        insts = wl.instances
        b64 = G.BatchSimulation(insts, precision=0)
        b64.step_batch(sim.sch, sim.dts, args.warmup)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(b64.stream)
        b64.step_batch_async(sim.sch, sim.dts, rounds)
        g1.record(b64.stream)
        b64.synchronize()
        torch.cuda.synchronize()
        ms64 = g0.elapsed_time(g1) / rounds
        p64 = float(b64.batch_diagnostics()[:, 8].sum())
        b64.close()
        singles = [G.Simulation.from_workload(w) for w in insts]
        for one, sc, w in zip(singles, sim.sch, insts):
            one.step(sc, w.dt, args.warmup)
        torch.cuda.synchronize()
        tt = time.perf_counter()
        for _ in range(rounds):
            for one, sc, w in zip(singles, sim.sch, insts):
                one.step_async(sc, w.dt, 1)
        for one in singles:
            one.synchronize()
        ms_sep = (time.perf_counter() - tt) * 1e3 / rounds
        p_sep = sum(float(one.diagnostics()[8]) for one in singles)
        for one in singles:
            one.close()
        # the same batch in the persistent form: one cooperative launch per step, replayed
        # from a captured graph
        bp = G.BatchSimulation(insts)
        bp.step_batch(sim.sch, sim.dts, args.warmup)
        bp.set_groups(sim_lanes)
        bp.set_step_mode(G.STEP_PERSISTENT)
        bp.step_batch(sim.sch, sim.dts, 3)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(bp.stream)
        bp.step_batch_async(sim.sch, sim.dts, rounds)
        q1.record(bp.stream)
        bp.synchronize()
        torch.cuda.synchronize()
        ms_p = q0.elapsed_time(q1) / rounds
        p_p = float(bp.batch_diagnostics()[:, 8].sum())
        bp.close()
        ms_p, p_p = job_totals(dist, ms_p, p_p, device=dev)
        ms64, p64 = job_totals(dist, ms64, p64, device=dev)
        ms_sep, p_sep = job_totals(dist, ms_sep, p_sep, device=dev)
        batch_vs = {
            "fp64_batch": {"value": p64 / (ms64 / 1e3), "unit": UNIT, "steps": rounds,
                           "ms_per_step": ms64, "fp32_speedup": round(value / (p64 / (ms64 / 1e3)), 3)},
            "separate_problems": {"value": p_sep / (ms_sep / 1e3), "unit": UNIT, "steps": rounds,
                                  "ms_per_step": ms_sep,
                                  "batched_speedup": round(value / (p_sep / (ms_sep / 1e3)), 3),
                                  "path": "one Simulation per instance (default tile shape, "
                                          "graph mode), sph_step_async on each, host clock"},
            "persistent_form": {"value": p_p / (ms_p / 1e3), "unit": UNIT, "steps": rounds,
                                "ms_per_step": ms_p, "lanes": sim_lanes,
                                "vs_graph_of_phases": round((p_p / (ms_p / 1e3)) / value, 3),
                                "path": "one cooperative launch per step replayed from a "
                                        "captured CUDA graph, CUDA events on the stream"}}

    # ---- hand-written adjoint: K steps forward, then the same K steps with the reverse sweep
    adjoint = None
    k_adj = args.adjoint_steps if args.adjoint_steps >= 0 else ADJOINT_STEPS.get(args.workload, 0)
    if args.integrator != "kdk":
        k_adj = 0  # the adjoint covers the kick-drift-kick integrator
    if k_adj > 0 and not sim.batch and sch.density == G.CONTINUITY:
        sim.set_timing(False)
        sim.load_state(pinned)
        sim.sim.backward(sch, wl.dt, k_adj)  # warm: workspace and graphs
        sim.load_state(pinned)
        sim.synchronize()
        tt = time.perf_counter()
        sim.step(k_adj)
        sim.synchronize()
        fwd_s = time.perf_counter() - tt
        sim.load_state(pinned)
        sim.synchronize()
        tt = time.perf_counter()
        _, g_nu, _ = sim.sim.backward(sch, wl.dt, k_adj)
        adj_s = time.perf_counter() - tt
        fwd_ms, _ = job_totals(dist, fwd_s * 1e3, 0.0, device=dev)
        adj_ms, _ = job_totals(dist, adj_s * 1e3, 0.0, device=dev)
        adjoint = {"steps": k_adj, "ckpt_every": math.ceil(math.sqrt(k_adj)),
                   "forward_ms": round(fwd_ms, 3), "forward_and_adjoint_ms": round(adj_ms, 3),
                   "ratio": round(adj_ms / fwd_ms, 3), "dKE_dnu": g_nu,
                   "path": "sph_backward (checkpoint every ckpt_every steps, recompute, taped "
                           "neighbour lists, reverse sweep) vs sph_step, host clock around the "
                           "synchronous calls"}

    # ---- the Taylor-Green runs of Sec. 4.1: max |u| over the whole run against the exact
    # U exp(b t), b = -8 pi^2 / Re
    decay = None
    if not sim.batch and getattr(wl, "density", 0) == 2:
        with G.Simulation.from_workload(wl) as run:  # from t = 0
            run.step(sch, wl.dt, wl.steps)
            h = run.history()
        t = h[:, 0]
        b = -8.0 * math.pi ** 2 * wl.nu  # Re = U L / nu with U = L = 1
        rel = np.abs(h[:, 3] / np.exp(b * t) - 1.0)
        fitted = math.log(h[-1, 3] / h[0, 3]) / (t[-1] - t[0])
        decay = {"steps": int(h.shape[0]), "t_end": float(t[-1]),
                 "max_u_end": float(h[-1, 3]), "exact_end": math.exp(b * t[-1]),
                 "max_rel_error_vs_exact": float(rel.max()),
                 "fitted_rate": fitted, "exact_rate": b,
                 "path": "sph_step over the paper's whole run from t = 0 (a new context), "
                         "max |u| of each step's record against U exp(-8 pi^2 t / Re)"}

    state0 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sim.batch:
        state0 = one_step_states(wl, sch)
    # the captured step's kernels, plus, for a single problem with a fixed step size, the
    # one-thread kernel of each sph_step_async call that sets the step size on the stream
    per_call = 0 if isinstance(raw, list) or wl.dt <= 0 else 1
    launches = (sim.kernels_per_step() + per_call) * args.steps
    sim.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if wl.precision == 1 else "f64", "data": "synthetic",
        "config": dict(describe(wl), step_mode=mode, momentum_lanes=sim_lanes,
                       density_lanes=density_lanes,
                       l2=("flushed between timed steps (512 MB write)" if flush_each else
                           f"no flush: inputs larger than L2 ({l2_bytes >> 20} MiB)")),
        "particle_steps_per_s": psteps, "candidates_per_s": job_cand / (total_ms / 1e3),
        "pairs_per_step": pairs / args.steps, "phase_ms": phase_avg,
        "roofline": roofline, "e2e": e2e, "fp64_mode": fp64, "adjoint": adjoint, "decay": decay,
        "batch_vs": batch_vs,
        "gpu_launches": launches, "clocks": clocks, "wall_s": round(t_wall, 3),
    }
    return line, state0, wl


def one_step_states(wl, sch):
    """GPU state after one step in FP32 and FP64 mode (for the error beside the metric)."""
    import paper_1909_04504_gb300 as G
    out = {}
    for prec in (1, 0):
        with G.Simulation.from_workload(wl.with_precision(prec)) as s:
            s.step(sch, wl.dt, 1)
            out[prec] = s.state()
    return out


# ---------------------------------------------------------------- oracle legs
def oracle_batch_sample(wls, target_s: float):
    """The oracle on the instances of a batch in order, 2 steps each, until target_s."""
    import oracle as O
    O.build()
    pairs, el, used = 0.0, 0.0, 0
    for w in wls:
        t0 = time.perf_counter()
        _, h = O.run(w, O.state_of(w), w.dt, 2)
        el += time.perf_counter() - t0
        pairs += float(h[:, 8].sum())
        used += 1
        if el > target_s:
            break
    sample = (f"2 steps (+1 initial evaluation) of each of the first {used} of {len(wls)} "
              f"instances, {el:.1f} s")
    return pairs / el, el, sample, O.threads()


def one_step_increment(wl, prop, new, old):
    """new - old; on a periodic position axis the minimum image (a wrapped particle moved
    the short way)."""
    import numpy as np
    d = np.asarray(new, np.float64) - np.asarray(old, np.float64)
    ax = {"x": 0, "y": 1, "z": 2}.get(prop)
    if ax is not None and wl.periodic[ax]:
        L = wl.hi[ax] - wl.lo[ax]
        d = d - L * np.round(d / L)
    return d


def cpu_baseline(wl, target_s: float, states=None) -> dict:
    """The oracle as it stands, timed on the host cores on a bounded sample of the workload."""
    import numpy as np

    import oracle as O
    if isinstance(wl, BatchView):
        v, _, sample, cores = oracle_batch_sample(wl.instances, target_s)
        return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    O.build()
    s = O.state_of(wl)
    t0 = time.perf_counter()
    _, h = O.run(wl, s, wl.dt, 1)
    t1 = time.perf_counter() - t0  # one step + the initial evaluation
    steps = max(1, min(2000, int(target_s / max(t1 / 2.0, 1e-6)) - 1))
    t0 = time.perf_counter()
    st, h = O.run(wl, s, wl.dt, steps)
    dt = time.perf_counter() - t0
    pairs = float(h[:, 8].sum())  # the initial evaluation is timed and counted too
    out = {"value": pairs / dt, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
           "sample": f"{steps} steps of {wl.name} from its initial state "
                     f"({steps + 1} right-hand-side evaluations), {dt:.1f} s"}
    if states is not None:
        ref, _ = O.run(wl, s, wl.dt, 1)
        err = {}
        props = ("x", "y", "z", "u", "v", "w", "rho") if wl.dim == 3 else ("x", "y", "u", "v", "rho")
        for prec, g in states.items():
            per = {}
            for k in props:
                if prec == 1:  # relative L2 of the one-step increment (minimum image)
                    a = one_step_increment(wl, k, g[k], s[k])
                    b = one_step_increment(wl, k, ref[k], s[k])
                    per[k] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
                else:  # normwise on the field
                    a, b = g[k], ref[k]
                    per[k] = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
            key = "fp32_increment_rel_l2" if prec == 1 else "fp64_normwise"
            err[key] = max(per.values())
            err[key + "_per_field"] = per
        out["one_step_error_vs_oracle"] = err
    return out


def reference_arm(args):
    """Times the oracle on the host cores in the base contract's reference slot."""
    import oracle as O
    wl = workload(args.workload, args.wall_bc, args.integrator)
    if isinstance(wl, list):
        v, el, sample, cores = oracle_batch_sample(wl, args.ref_seconds)
        return {
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(BatchView(wl)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
    O.build()
    s = O.state_of(wl)
    t0 = time.perf_counter()
    st, _ = O.run(wl, s, wl.dt, max(1, args.warmup))
    warm_s = time.perf_counter() - t0
    per_step = warm_s / (max(1, args.warmup) + 1)
    steps = args.steps
    cap = max(1, int(args.ref_seconds / max(per_step, 1e-6)))
    sample_steps = min(steps, cap)
    t0 = time.perf_counter()
    st, h = O.run(wl, st, wl.dt, sample_steps)
    el = time.perf_counter() - t0
    pairs = float(h[:, 8].sum())
    value = pairs / el
    sample = (f"{sample_steps} oracle steps of {wl.name} (+1 initial evaluation) after "
              f"{args.warmup} warm-up steps, {el:.1f} s")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / sample_steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": describe(wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------- variable smoothing length search
VH_WORKLOADS = ("gaussian_blob_3d", "gaussian_blob_2d")
VH_METRIC = "neighbour pairs/s of the variable-h octree search (build + query)"
VH_UNIT = "neighbour pairs/s"
VH_N = 1_000_000
VH_LEAF = 32  # of leaves of 8, 16, 32, 64: fastest in 2D, within 4 % of 64 in 3D


def vh_set(name: str):
    import workloads as W
    return W.gaussian_blob(VH_N, dim=3 if name.endswith("3d") else 2, precision=W.PREC_FP32)


def vh_flops(dim: int, cand: float, pairs: float) -> float:
    """Algorithmic FP32 flops of the query: per pair examined the squared distance (d
    subtractions, d products, d - 1 sums) and the radius (k max(h_i, h_j), squared); per
    neighbour the density term (h_ij: 2, reciprocal, square root, q, 1 / h_ij^d: d - 1,
    the Wendland polynomial: 7, sigma w m: 3, the compensated add: 4). Node tests are not
    counted (a lower bound)."""
    test = 3 * dim + 1
    dens = 2 + 1 + 1 + 1 + (dim - 1) + 7 + 3 + 4
    return test * cand + dens * pairs


def vh_describe(s, leaf: int = VH_LEAF) -> dict:
    import numpy as np
    return {"workload": f"{s.name}: {s.n:,} particles, {s.dim}D, normal positions truncated at "
                        f"r = 3, h = 1.2 (m / rho)^(1/{s.dim}) from the number density "
                        f"({float(np.min(s.h)):.4g} .. {float(np.max(s.h)):.4g}), Wendland C2, "
                        f"FP32 predicate and density, octree leaves of <= {leaf}",
            "particles": s.n, "parallelism": "replicas (one independent problem per GPU)"}


def vh_arm(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_1909_04504_gb300 as G

    dev = torch.cuda.current_device()
    s = vh_set(args.workload)
    v = G.VariableHSearch(s.dim, s.kernel, s.precision, s.n, leaf_size=args.leaf_size)
    z = s.z if s.dim == 3 else None
    v.set(s.x, s.y, z, s.h, s.m)
    for _ in range(args.warmup):
        v.search()
    st = v.stats()
    stream = torch.cuda.ExternalStream(v.stream_handle)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        uuid = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
    sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    v.set_timing(True)
    v.search()
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    # ---- timed region: K searches, L2 flushed before each (the inputs fit in L2); the
    # device time of each search from the events recorded around its two phases
    build, query = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        v.search()
        ph = v.phase_times()
        build.append(ph["build"])
        query.append(ph["query"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    v.set_timing(False)
    total_ms = sum(build) + sum(query)
    pairs = float(st["pairs"]) * args.steps
    total_ms, job_pairs = job_totals(dist, total_ms, pairs, device=dev)
    value = job_pairs / (total_ms / 1e3)
    # ---- end to end through the public API: the inputs from host memory, the search, the
    # density back to the host, per step (host clock)
    e2e_steps = max(3, min(args.steps, 20))
    rho = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        v.set(s.x, s.y, z, s.h, s.m)
        v.search()
        rho = v.density()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": st["pairs"] * e2e_steps / e2e_s, "unit": VH_UNIT,
           "h2d_bytes_per_step": 8 * s.n * (5 if s.dim == 3 else 4),
           "d2h_bytes_per_step": 8 * s.n, "steps": e2e_steps,
           "path": "sph_vh_set (host arrays) + sph_vh_search + sph_vh_density per step, host clock"}
    mhz, mhz_src = sm_max_mhz(clocks)
    q_ms = statistics.mean(query)
    flops = vh_flops(s.dim, st["candidates"], st["pairs"])
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12 if mhz else None
    achieved = flops / (q_ms / 1e3) / 1e12
    B = 10 if s.dim == 3 else 15
    launches = 2 + 1 + 4 + 1 + B + (B + 1) + 1
    line = {
        "metric": VH_METRIC, "value": value, "unit": VH_UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": dict(vh_describe(s, args.leaf_size), l2="flushed between timed searches (512 MB write)"),
        "phase_ms": {"build": statistics.mean(build), "query": q_ms},
        "search": {k: st[k] for k in ("nodes", "leaves", "depth", "candidates", "pairs", "max_count")},
        "pairs_per_particle": st["pairs"] / s.n,
        "candidates_per_pair": st["candidates"] / max(st["pairs"], 1),
        "roofline": {"bound": "alu", "achieved": round(achieved, 4),
                     "peak": round(peak, 3) if peak else None, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 5) if peak else None, "traffic": None,
                     "kernel": "k_vh_query (octree walk, predicate, list, density)",
                     "flops_per_launch": flops, "avg_launch_ms": round(q_ms, 5),
                     "peak_source": f"derived: {sms} SMs (device) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz} MHz ({mhz_src})"},
        "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks,
        "wall_s": round(t_wall, 3),
        "density_range": [float(np.min(rho)), float(np.max(rho))] if rho is not None else None,
    }
    v.close()
    return line, s


def vh_cpu_sample(s, target_s: float, seed: int = 5):
    """The oracle's selected-rows form on a bounded sample of the particles (every pair of
    a sampled particle examined): (pairs/s, seconds, rows, cores)."""
    import numpy as np

    import oracle as O
    O.build()
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = rng.choice(s.n, 64, replace=False)
    t0 = time.perf_counter()
    O.vh_rows(s.dim, s.kernel, s.precision, s.x, s.y, s.z, s.h, s.m, rows)
    probe = max(time.perf_counter() - t0, 1e-3)
    k = int(min(s.n, max(64, 64 * target_s / probe)))
    rows = rng.choice(s.n, k, replace=False)
    t0 = time.perf_counter()
    off, _, _ = O.vh_rows(s.dim, s.kernel, s.precision, s.x, s.y, s.z, s.h, s.m, rows)
    el = time.perf_counter() - t0
    return float(off[-1]) / el, el, k, O.threads()


def vh_cpu_baseline(s, target_s: float) -> dict:
    v, el, k, cores = vh_cpu_sample(s, target_s)
    return {"value": v, "unit": VH_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} sampled particles of {s.name}, each tested against all {s.n:,} "
                      f"(the oracle's all-pairs relation and density), {el:.1f} s"}


def vh_reference_arm(args):
    s = vh_set(args.workload)
    v, el, k, cores = vh_cpu_sample(s, args.ref_seconds)
    return {
        "impl": "reference", "metric": VH_METRIC, "value": v, "unit": VH_UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": vh_describe(s, args.leaf_size),
        "cpu_baseline": {"value": v, "unit": VH_UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{k} sampled particles, each against all {s.n:,}, {el:.1f} s"},
        "e2e": {"value": v, "unit": VH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dam_break_3d",
                    choices=["dam_break_2d", "taylor_green_2d", "taylor_green_2d_edac",
                             "taylor_green_3d", "dam_break_3d", "dam_break_3d_dx01", "batch_tg2d",
                             "falling_cube_3d"] + list(VH_WORKLOADS))
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="reference arm: seconds of oracle time in the timed sample")
    ap.add_argument("--step-mode", default="auto", choices=["auto", "graph", "persistent"],
                    help="auto: the autotuner picks the tile shape and the step form")
    ap.add_argument("--wall-bc", default="density", choices=["density", "adami"],
                    help="wall condition: continuity walls (the configurations') or the "
                         "solid-wall pressure of Adami et al.")
    ap.add_argument("--integrator", default="kdk", choices=["kdk", "pec"],
                    help="kick-drift-kick (the paper's form) or the two-evaluation midpoint "
                         "predict-evaluate-correct form")
    ap.add_argument("--adjoint-steps", type=int, default=-1,
                    help="K of the timed adjoint (-1: 50 for taylor_green_3d, 20 for "
                         "dam_break_3d, none otherwise; 0: off)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="lanes per destination of both pair passes (0: the autotuner's or "
                         "the default shape)")
    ap.add_argument("--leaf-size", type=int, default=VH_LEAF,
                    help="variable-h search: particles per octree leaf before a split")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        arm = vh_reference_arm if args.workload in VH_WORKLOADS else reference_arm
        print(json.dumps(arm(args)), flush=True)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    if args.workload in VH_WORKLOADS:
        line, vs = vh_arm(args, rank, world, dist)
        cpu = (lambda: vh_cpu_baseline(vs, args.cpu_seconds))
    else:
        line, states, wl = gpu_arm(args, rank, world, dist)
        cpu = (lambda: cpu_baseline(wl, args.cpu_seconds, states))
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu()
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
