#!/usr/bin/env python3
"""Benchmark of the GB300 PIC step with in-situ cost measurement and dynamic
load balancing (the method of arXiv 2104.11385).

Headline workload: the 3D laser-foil at scale, 512 x 512 x 1024 cells in 8192
boxes of 32^3, a hydrogen foil 16 cells thick at 30 n_c with 64 electrons + 64
protons per foil cell (536,870,912 particles), a0 = 20 laser, FP64, load
balancing every 20 steps.  One step = one full PIC cycle (per-tile sort, TMA
tile staging, gather, Boris push, Esirkepov deposit with clock64 box costs, Yee
update, boundaries) plus the load-balancing routine at its interval (dynamic,
knapsack, device-clock costs, threshold 10 %).  Beside it: the 256^3 foil, the
4096 log-normal boxes, the serving recipe (1000 2D3V requests) and the FP64 CPU
oracle on the host cores.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica of the workload (weak
scaling, no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import re
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal
# FP64 peak from unit counts and clocks, for context beside the measured one:
# SMs x 2 DFMA lanes/clk/SM x 2 flop x 2.07 GHz (the SM count read from the device)
FP64_LANES_PER_SM_CLK = 2
SM_MAX_GHZ = 2.07
# algorithmic FP64 flops per particle update, in-cell path (3D linear: gather 126,
# local positions and half-node shifts 6, Boris push 70, Esirkepov deposit 73, positions 3)
FLOPS_PER_PARTICLE = {(3, 1): 275.0, (3, 2): 763.0, (3, 3): 1591.0, (2, 1): 168.0, (2, 2): 348.0,
                      (2, 3): 546.0}
BYTES_PER_PARTICLE = 104.0  # read x,y,z,ux,uy,uz,w (56) + write x..uz (48)
BYTES_PER_CELL = 120.0      # read E,B,J (72) + write E,B (48)

# DRAM traffic of the FP64 particle kernel <3,1> from one ncu capture on the
# foil recipe at half extents (128^3 cells, 8,388,608 particles; 256 threads,
# 2 CTAs/SM): dram__bytes_read.sum + dram__bytes_write.sum = 501.01 + 409.76 MB
# (the capture's summary sits with the ncu profiles).  Traffic grows with the
# particle count, so a full launch is scaled by particles.  The figure is
# reported only while the kernel's code (comments aside) hashes to what was
# captured.
TRAFFIC_CAPTURE = {"bytes_per_particle": (501.010432e6 + 409.757440e6) / 8388608, "dim": 3, "order": 1,
                   "sources": ("paper_2104_11385_gb300/csrc/pic_particle_kernel.cuh",
                               "paper_2104_11385_gb300/csrc/pic_particles_f64_3d.cu",
                               "paper_2104_11385_gb300/csrc/pic_dd.cuh",
                               "paper_2104_11385_gb300/csrc/pic_internal.h",
                               "paper_2104_11385_gb300/csrc/pic_sync.cuh"),
                   "sha256": "82cc630c91293752a1621f91ff9feac441b0448dc4fe5d75df8e4a03b78108c0"}


def _kernel_sources_sha(paths):
    """SHA-256 of the kernel's code: comments, blank lines and trailing blanks
    dropped, so that a comment edit does not count as a kernel change."""
    h = hashlib.sha256()
    here = os.path.dirname(os.path.abspath(__file__))
    for rel in paths:
        with open(os.path.join(here, rel)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()


def _traffic_per_launch(wl, nparts):
    c = TRAFFIC_CAPTURE
    if (wl["dim"], wl["order"]) != (c["dim"], c["order"]):
        return None
    try:
        if _kernel_sources_sha(c["sources"]) != c["sha256"]:
            return None
    except OSError:
        return None
    return c["bytes_per_particle"] * nparts


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        return float(json.load(open(MEASURED))["hbm_gbs"])
    except Exception:
        return HBM_FALLBACK_GBS


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="foil_at_scale",
                    choices=["foil256", "uniform32", "lognormal4096", "laser_ion_2d", "foil_at_scale"])
    ap.add_argument("--secondary", default="foil256", choices=["foil256", "none"],
                    help="a second, compact line of arms on the 256^3 foil")
    ap.add_argument("--scale", type=int, default=1, help="divide the workload extents (small cases for profiling)")
    ap.add_argument("--sched", default="queue", choices=["lists", "queue"])
    ap.add_argument("--split", type=int, default=0, help="work units per worker (0: library default)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--precision", type=int, default=1, choices=[1, 2, 3],
                    help="particle push arithmetic of the main arm: 1 FP64, 2 float-float, 3 FP32")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0, help="cells per tile edge with --threads (0: library default)")
    ap.add_argument("--ppt", type=int, default=0, help="particles per thread with --threads (0: library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-server", action="store_true")
    ap.add_argument("--no-cost-arms", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--repeats", type=int, default=5,
                    help="K-step windows timed on the balanced arm for the spread (median, best) beside the value")
    ap.add_argument("--static-steps", type=int, default=5,
                    help="timed steps of the no-balancing arm (about 8x slower per step than the balanced one)")
    ap.add_argument("--server-requests", type=int, default=1000)
    ap.add_argument("--server-steps-max", type=int, default=2000,
                    help="request lengths U[100, max] steps (the serving recipe's range is 100..2000)")
    ap.add_argument("--server-half", action="store_true",
                    help="also serve the mix with Poisson arrivals at 0.5x the saturated rate")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--timeline", type=int, default=0,
                    help="instead of the bench line: N steps of the workload under each load-balancing mode "
                         "(none / static / dynamic), with E and the time per step every interval")
    ap.add_argument("--timeline-modes", default="none,static,dynamic,dynamic_sfc",
                    help="comma-separated modes of --timeline: none, static, dynamic (knapsack, device-clock "
                         "costs), dynamic_sfc, dynamic_heuristic (knapsack, particle/cell-count costs), "
                         "dynamic_kernel_time")
    return ap.parse_args()


def _jsonable(o):
    """numpy scalars and arrays in the JSON line"""
    if hasattr(o, "tolist"):
        return o.tolist()
    return str(o)


def max_over_ranks(value, world):
    """Maximum of a per-rank float over all ranks (the slowest rank sets the
    job's time); plain value when running alone."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name, scale, seed_offset=0):
    from paper_2104_11385_gb300 import workloads as W
    if name == "foil256":
        return W.foil256(seed=2 + seed_offset, scale=scale)
    if name == "uniform32":
        return W.uniform32(seed=1 + seed_offset)
    if name == "laser_ion_2d":
        return W.laser_ion_2d(seed=6 + seed_offset, scale=scale)
    if name == "foil_at_scale":
        return W.foil_at_scale(seed=5 + seed_offset, scale=scale)
    n = max(2, 16 // scale)  # scale > 1: fewer boxes of the same recipe
    return W.lognormal(seed=3 + seed_offset, nbox=(n, n, n))


def lb_interval(wl):
    return int(wl.get("lb_interval", 10))


def workload_desc(wl):
    nparts = sum(len(s["x"]) for s in wl["species"])
    return {
        "workload": wl["name"], "cells": list(wl["ncell"]), "box": list(wl["box"]),
        "boxes": int(math.prod(wl["ncell"][a] // wl["box"][a] for a in range(3))),
        "particles": nparts, "species": len(wl["species"]), "shape_order": wl["order"],
        "lb": "dynamic knapsack, device-clock costs, interval %d, theta 0.10" % lb_interval(wl),
        "l2": "inputs larger than L2 (particle state %.1f GB)" % (nparts * 64 / 1e9),
    }


def fp64_peak():
    """The FP64 FMA throughput of this GPU, measured by libpic's probe (a DFMA
    loop timed with CUDA events), and the unit-count figure beside it."""
    import torch
    from paper_2104_11385_gb300.sim import probe_fp64_fma
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    measured = probe_fp64_fma(20000)
    nominal = nsm * FP64_LANES_PER_SM_CLK * 2 * SM_MAX_GHZ * 1e9 / 1e12
    return measured, nominal, nsm


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def run_ours(args, rank, world, wl=None, full=True):
    """All arms of one workload.  full=False runs the compact set (balanced,
    float-float, FP32, static order) used for the secondary workload."""
    import numpy as np
    import torch
    import paper_2104_11385_gb300 as pic

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if wl is None:
        wl = make_workload(args.workload, args.scale, seed_offset=rank)
    nparts = sum(len(s["x"]) for s in wl["species"])
    ncells = int(math.prod(wl["ncell"]))
    stream = torch.cuda.Stream()
    interval = lb_interval(wl)
    sched = pic.SCHED_QUEUE if args.sched == "queue" else pic.SCHED_LISTS
    lbkw = dict(mode=pic.LB_DYNAMIC, interval=interval, theta=0.10, policy=pic.POLICY_KNAPSACK,
                cost=pic.COST_DEVICE_CLOCK, split=args.split, sched=sched)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(sim, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), world)

    def rate(ms, k):
        return nparts * k * world / (ms / 1e3)

    def release(sim):
        sim.close()
        torch.cuda.empty_cache()

    def profiled(sim, k):
        sim.set_profiling(True)
        sim.step(k)
        st = sim.stats()
        sim.set_profiling(False)
        return st

    def per_step(st, key):
        return st[key] / max(st["steps"], 1)

    # ---- balanced (the paper's dynamic load balancing, on the SMs)
    sim = pic.from_workload(wl, stream=stream.cuda_stream)
    sim.step(1)                                      # measure per-box clock costs once
    sim.rebalance(**dict(lbkw, theta=0.0))           # initial cost-driven mapping
    sim.set_lb_params(**lbkw)
    sim.set_launch(precision=args.precision)
    if args.threads or args.ctas_per_sm:
        sim.set_launch(threads=args.threads, ctas_per_sm=args.ctas_per_sm, tile=args.tile, ppt=args.ppt)
        tuned = sim.get_launch()
    else:
        tuned = sim.autotune(steps_per_candidate=2)  # threads, CTAs/SM, units per worker
    sim.step(args.warmup)
    nlog0 = len(sim.lb_log())
    with ClockSampler(dev) as cs:
        ms_bal = timed(sim, args.steps)
    clocks = cs.summary()
    lb_timed = sim.lb_log()[nlog0:]  # the load-balancing calls made inside the timed steps
    # spread of the step time: the same K-step window again (the line's value is
    # the first window, timed as the contract says; these are beside it)
    reps = [ms_bal / args.steps] + [timed(sim, args.steps) / args.steps for _ in range(max(0, args.repeats - 1))]
    # kernel-level timing: the same number of steps again, with CUDA events on
    # the library's stream around each launch
    st = profiled(sim, args.steps)
    kernels_per_step = st["launches"] / max(st["steps"], 1)
    release(sim)
    tkw = {k: tuned[k] for k in ("threads", "ctas_per_sm", "split", "tile", "ppt")}

    # ---- reduced-precision variants (float-float push; FP32 push)
    variants = {}
    if not args.no_mixed and args.precision == 1:
        for prec in (2, 3):
            sim = pic.from_workload(wl, stream=stream.cuda_stream)
            sim.set_launch(precision=prec)
            sim.step(1)
            sim.rebalance(**dict(lbkw, theta=0.0))
            sim.set_lb_params(**lbkw)
            vtuned = sim.autotune(steps_per_candidate=2)
            sim.step(args.warmup)
            ms_v = timed(sim, args.steps)
            vst = profiled(sim, args.steps)
            release(sim)
            kms = per_step(vst, "ms_particle")
            variants[prec] = {"value": rate(ms_v, args.steps), "unit": "particle-updates/s",
                              "ms_per_step": ms_v / args.steps, "particle_kernel_ms": kms, "launch": vtuned,
                              "phase_ms_per_step": {"particle": kms, "fields": per_step(vst, "ms_fields"),
                                                    "sort": per_step(vst, "ms_sort")},
                              "hbm_frac": BYTES_PER_PARTICLE * nparts / (kms / 1e3) / 1e9 / hbm_peak_gbs()}
        variants[2]["arithmetic"] = ("float-float (FP32 pairs, ~48-bit significand) gather, Boris and deposit "
                                     "weights; FP64 storage, positions and current sums; parity 1e-10 vs the "
                                     "FP64 oracle (tests/test_gpu_parity.py)")
        variants[3]["arithmetic"] = ("FP32 gather, Boris and deposit weights; FP64 storage, positions and "
                                     "current sums; parity 3e-5 (500 FP32 roundoffs) vs the FP64 oracle "
                                     "(tests/test_gpu_parity.py)")

    # ---- static box order (no load balancing: the fixed starting mapping)
    sim = pic.from_workload(wl, stream=stream.cuda_stream)
    sim.set_launch(threads=tuned["threads"], ctas_per_sm=tuned["ctas_per_sm"], tile=tuned["tile"], ppt=tuned["ppt"],
                   precision=args.precision)
    sim.step(1 + min(args.warmup, 2))
    ks = max(1, args.static_steps)
    ms_static = timed(sim, ks)
    release(sim)
    static = {"value": rate(ms_static, ks), "ms_per_step": ms_static / ks, "timed_steps": ks,
              "speedup_balanced_over_static": (ms_static / ks) / (ms_bal / args.steps),
              "what": "mode NONE: one unit per box, fixed equal-count Morton mapping, per-worker lists"}

    srt = sorted(reps)
    spread = {"windows": len(reps), "steps_per_window": args.steps, "median_ms_per_step": srt[len(srt) // 2],
              "best_ms_per_step": srt[0], "worst_ms_per_step": srt[-1],
              "median_value": rate(srt[len(srt) // 2] * args.steps, args.steps)}
    out = {"value": rate(ms_bal, args.steps), "ms_per_step": ms_bal / args.steps, "step_time_spread": spread,
           "clocks": clocks,
           "gpu_launches": int(round(kernels_per_step * args.steps)), "static_order": static,
           "mixed_precision": variants.get(2), "fp32": variants.get(3),
           "config": dict(workload_desc(wl), sched=args.sched, launch=tuned), "launch": tuned}
    ms_part = per_step(st, "ms_particle")
    out["phase_ms_per_step"] = {"particle": ms_part, "fields": per_step(st, "ms_fields"),
                                "sort": per_step(st, "ms_sort")}
    out["cell_updates_per_s"] = ncells * args.steps * world / (ms_bal / 1e3)
    out["fdtd_cell_updates_per_s"] = ncells / (per_step(st, "ms_fields") / 1e3)
    out["lb"] = {"calls_in_timed_steps": len(lb_timed), "adopted": sum(1 for r in lb_timed if r["adopted"]),
                 "last": lb_timed[-1] if lb_timed else None}
    out["_nparts"] = nparts
    if not full:
        return out

    # ---- the other schedule kind, for the side-by-side line
    other = "lists" if args.sched == "queue" else "queue"
    sim = pic.from_workload(wl, stream=stream.cuda_stream)
    okw = dict(lbkw, sched=pic.SCHED_LISTS if other == "lists" else pic.SCHED_QUEUE)
    sim.set_launch(**tkw, precision=args.precision)
    sim.step(1)
    sim.rebalance(**dict(okw, theta=0.0))
    sim.set_lb_params(**okw)
    sim.step(args.warmup)
    ms_other = timed(sim, args.steps)
    release(sim)
    out["other_schedule"] = {"sched": other, "value": rate(ms_other, args.steps),
                             "ms_per_step": ms_other / args.steps}

    # ---- cutting against ordering: the balanced arm's work units (heavy boxes
    # cut by the measured costs, the autotuned split) mapped once and never
    # again, pulled from the queue either in box-index order (no cost input in
    # the order) or longest-first (the knapsack's cost order)
    order_arms = {}
    for name, policy in (("static_units_box_order", pic.POLICY_BOX_ORDER),
                         ("static_units_lpt_order", pic.POLICY_KNAPSACK)):
        sim = pic.from_workload(wl, stream=stream.cuda_stream)
        sim.set_launch(**tkw, precision=args.precision)
        sim.step(1)
        r = sim.rebalance(**dict(lbkw, policy=policy, theta=0.0, sched=pic.SCHED_QUEUE,
                                 split=tuned["split"]))
        sim.step(args.warmup)
        ms_o = timed(sim, args.steps)
        release(sim)
        order_arms[name] = {"value": rate(ms_o, args.steps), "ms_per_step": ms_o / args.steps,
                            "units": r["n_units"], "adopted": r["adopted"]}
    nb = order_arms["static_units_box_order"]["ms_per_step"]
    nl = order_arms["static_units_lpt_order"]["ms_per_step"]
    order_arms["speedup_cutting"] = static["ms_per_step"] / nb
    order_arms["speedup_lpt_order_over_box_order"] = nb / nl
    order_arms["speedup_dynamic_over_static_lpt"] = nl / out["ms_per_step"]
    order_arms["what"] = ("static_order -> static_units_box_order: cutting heavy boxes alone; -> "
                          "static_units_lpt_order: the same units in cost order; -> balanced: remapping every "
                          "interval with fresh device-clock costs")
    out["cutting_vs_ordering"] = order_arms

    # ---- the paper's cost strategies side by side (same schedule, same tuning)
    cost_arms = {"device_clock": out["value"]}
    if not args.no_cost_arms:
        # the heuristic needs no device capture: with capture off the same
        # mappings run without the clock64 / %globaltimer work, which is the
        # capture's overhead (the paper measured about 2x for CUPTI)
        for name, cst, cap in (("heuristic", pic.COST_HEURISTIC, True), ("kernel_time", pic.COST_KERNEL_TIME, True),
                               ("heuristic_no_capture", pic.COST_HEURISTIC, False)):
            ckw = dict(lbkw, cost=cst)
            sim = pic.from_workload(wl, stream=stream.cuda_stream)
            if not cap:
                sim.set_cost_capture(clock=False, kernel_time=False)
            sim.step(1)
            sim.rebalance(**dict(ckw, theta=0.0))
            sim.set_lb_params(**ckw)
            sim.set_launch(**tkw, precision=args.precision)
            sim.step(args.warmup)
            cost_arms[name] = rate(timed(sim, args.steps), args.steps)
            release(sim)
        cost_arms["capture_overhead"] = cost_arms["heuristic_no_capture"] / cost_arms["heuristic"] - 1.0
    out["cost_strategies"] = cost_arms

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        pinned = []
        for s in wl["species"]:
            pinned.append({k: torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory()
                           for k in ("x", "y", "z", "ux", "uy", "uz", "w", "id")})
        out_e = torch.empty(ncells, dtype=torch.float64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for p in pinned for v in p.values())
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = pic.Simulation(wl["dim"], wl["ncell"], wl["box"], wl["dx"], dt=wl["dt"],
                             shape_order=wl["order"], absorb_cells=wl["absorb"], stream=stream.cuda_stream)
        for s, p in zip(wl["species"], pinned):
            sim.add_species(s["q"], s["m"], p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"], p["w"], ids=p["id"])
        L = wl["laser"]
        sim.add_laser(L["a0"], L["w0"], L["tau"], L["t_peak"], L["omega"], L["xc"], L["yc"], L["k_ant"])
        sim.set_launch(**tkw, precision=args.precision)
        # the first mapping from the particle counts (the heuristic cost, known
        # before any step), the next from the first step's in-situ clock costs
        sim.rebalance(**dict(lbkw, cost=pic.COST_HEURISTIC, theta=0.0))
        sim.step(1)
        sim.rebalance(**dict(lbkw, theta=0.0))
        sim.set_lb_params(**lbkw)
        d2h = 0
        for _ in range(args.steps):
            sim.step(1)
            # each step's result: the in-situ per-box costs and counts, read back
            costs, npb = sim.box_costs(pic.COST_DEVICE_CLOCK)
            d2h += costs.nbytes + npb.nbytes
        sim.read_field(pic.EX, out=out_e)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d2h += out_e.numel() * 8
        sim.close()
        del pinned
        secs = max_over_ranks(t1 - t0, world)
        out["e2e"] = {"value": nparts * (args.steps + 1) * world / secs, "unit": "particle-updates/s",
                      "h2d_bytes_per_step": int(h2d / (args.steps + 1)),
                      "d2h_bytes_per_step": int(d2h / (args.steps + 1)),
                      "what": "pic_init + pic_add_species from pinned host arrays (the run's input, amortised over "
                              "its steps) + rebalance on heuristic costs + 1 step + rebalance on its clock costs "
                              "+ K steps, each followed by reading its per-box costs and counts back, + Ex back "
                              "at the end"}

    # ---- roofline of the dominant kernel (the particle kernel)
    flops = FLOPS_PER_PARTICLE[(wl["dim"], wl["order"])] * nparts
    achieved_tf = flops / (ms_part / 1e3) / 1e12
    hbm = hbm_peak_gbs()
    peak_src = "measured" if os.path.exists(MEASURED) else "fallback"
    hbm_achieved = BYTES_PER_PARTICLE * nparts / (ms_part / 1e3) / 1e9
    hbm_obj = {"achieved_gbs": hbm_achieved, "peak_gbs": hbm, "frac": hbm_achieved / hbm,
               "peak_source": peak_src, "bytes_per_particle": BYTES_PER_PARTICLE,
               "frac_of_nominal": hbm_achieved / HBM_NOMINAL_GBS}
    kname = "pic_particle_kernel<%d,%d> (gather+Boris+Esirkepov+cost)" % (wl["dim"], wl["order"])
    if args.precision == 1:
        # the FP64 kernel is bound by the FP64 pipe: algorithmic flops against
        # the FP64 FMA throughput measured here
        measured, nominal, nsm = fp64_peak()
        out["roofline"] = {"bound": "alu", "achieved": achieved_tf, "peak": measured, "unit": "TFLOP/s",
                           "frac": achieved_tf / measured, "traffic": _traffic_per_launch(wl, nparts),
                           "kernel": kname,
                           "peak_note": ("FP64 pipe, measured: pic_probe_fp64_fma (DFMA chains on every SM, "
                                         "CUDA events) %.3f TFLOP/s; from unit counts %d SMs x %d DFMA lanes/clk "
                                         "x 2 flop x %.2f GHz = %.3f TFLOP/s"
                                         % (measured, nsm, FP64_LANES_PER_SM_CLK, SM_MAX_GHZ, nominal)),
                           "frac_of_unit_count_peak": achieved_tf / nominal,
                           "algorithmic_flop_per_particle": FLOPS_PER_PARTICLE[(wl["dim"], wl["order"])],
                           "hbm": hbm_obj}
    else:
        # float-float and FP32 leave the FP64 pipe nearly idle: report the particle
        # bytes against HBM (the traffic capture is of the FP64 kernel, so none here)
        out["roofline"] = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                           "frac": hbm_achieved / hbm, "traffic": None, "kernel": kname,
                           "peak_note": "%s HBM copy bandwidth" % peak_src}
    return out


def run_c3(args, steps=10):
    """Batched uneven boxes: 4096 boxes of 16^3 cells (256^3), box particle
    counts round(exp(N(ln 2000, 2^2))) (~60M particles), quadratic shape, one
    persistent autotuned launch per step; static box order against
    device-clock, kernel-time and heuristic costs, and how well each cost
    tracks the particle count."""
    import numpy as np
    import torch
    from scipy.stats import spearmanr
    import paper_2104_11385_gb300 as pic
    from paper_2104_11385_gb300 import workloads as W
    wl = W.lognormal(seed=3)
    nparts = sum(len(s["x"]) for s in wl["species"])
    stream = torch.cuda.Stream()
    out = {"workload": "lognormal 16^3 boxes of 16^3 cells, quadratic", "particles": nparts,
           "max_box_particles": int(wl["box_counts"].max()), "steps": steps}

    def timed(sim, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sim = pic.from_workload(wl, stream=stream.cuda_stream)
    sim.step(2)
    ms = timed(sim, steps)
    out["static_order"] = nparts * steps / (ms / 1e3)
    sim.close()
    tuned = None
    for name, cst in (("device_clock", pic.COST_DEVICE_CLOCK), ("kernel_time", pic.COST_KERNEL_TIME),
                      ("heuristic", pic.COST_HEURISTIC)):
        kw = dict(mode=pic.LB_DYNAMIC, interval=10, theta=0.10, policy=pic.POLICY_KNAPSACK, cost=cst,
                  sched=pic.SCHED_QUEUE)
        sim = pic.from_workload(wl, stream=stream.cuda_stream)
        sim.step(1)
        if name == "device_clock":
            clk, npb = sim.box_costs(pic.COST_DEVICE_CLOCK)
            kt, _ = sim.box_costs(pic.COST_KERNEL_TIME)
            out["spearman_device_clock_vs_np"] = float(spearmanr(clk, npb).correlation)
            out["spearman_kernel_time_vs_np"] = float(spearmanr(kt, npb).correlation)
        sim.rebalance(**dict(kw, theta=0.0))
        sim.set_lb_params(**kw)
        if tuned is None:
            tuned = sim.autotune(steps_per_candidate=2)
        else:
            sim.set_launch(**tuned)
        sim.step(2)
        ms = timed(sim, steps)
        out[name] = nparts * steps / (ms / 1e3)
        sim.close()
    out["launch"] = tuned
    out["speedup_balanced_over_static"] = out["device_clock"] / out["static_order"]
    return out


def run_server(args, seed=4):
    """Serving arm: independent 2D3V thermal-plasma requests (the serving
    recipe: 1000 requests, grid side in {64,128,256,512}, ppc in {1,..,64},
    steps U[100, 2000]) through the continuous-batching server; first all at
    once (saturated throughput), then Poisson arrivals at 0.8x that rate (and
    at 0.5x with --server-half)."""
    import numpy as np
    from paper_2104_11385_gb300.server import Server
    from paper_2104_11385_gb300 import _lib as L
    rng = np.random.default_rng(seed)
    n = args.server_requests
    reqs = []
    for i in range(n):
        side = int(rng.choice([64, 128, 256, 512]))
        ppc = int(rng.choice([1, 2, 4, 8, 16, 32, 64]))
        steps = int(rng.integers(100, args.server_steps_max + 1))
        reqs.append(dict(ncell=(side, 1, side), box=(32, 1, 32), dx=(0.2, 1.0, 0.2), nsteps=steps,
                         plasma=dict(ppc=ppc, density=1.0, u_th=0.02, ripple=0.01, seed=1000 + i)))
    work = sum(r["ncell"][0] * r["ncell"][2] * r["plasma"]["ppc"] * r["nsteps"] for r in reqs)

    def serve(arrivals):
        srv = Server(dim=2, max_active=64, hbm_budget_bytes=160 << 30)
        t0 = time.perf_counter()
        ids, k, done = {}, 0, {}
        while len(done) < n:
            now = time.perf_counter() - t0
            while k < n and arrivals[k] <= now:
                ids[srv.submit(**reqs[k])] = k
                k += 1
            a, p = srv.tick()
            for rid, i in list(ids.items()):
                st = srv.poll(rid)
                if st["state"] == L.REQ_DONE:
                    done[i] = st["t_done"] - st["t_submit"]
                    srv.release(rid)
                    del ids[rid]
            if a == 0 and p == 0 and k < n:
                time.sleep(max(0.0, min(0.05, arrivals[k] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        lat = np.array([done[i] for i in range(n)])
        return wall, lat, stats

    wall_sat, lat_sat, st_sat = serve([0.0] * n)
    sat_rate = n / wall_sat
    out = {"requests": n,
           "mix": "2D3V, side {64..512}, ppc {1..64}, steps U[100,%d], 32x32 boxes, FP64, linear" % args.server_steps_max,
           "particle_updates": int(work),
           "saturated_requests_per_s": sat_rate, "saturated_particle_updates_per_s": work / wall_sat}
    out["arrival_rates"] = "0.8x and 0.5x the saturated rate" if args.server_half else (
        "0.8x the saturated rate (the 0.5x pass is left out of the default run for time: --server-half)")
    for frac in ((0.8, 0.5) if args.server_half else (0.8,)):
        lam = frac * sat_rate
        arr = np.cumsum(rng.exponential(1.0 / lam, n))
        arr -= arr[0]
        wall, lat, st = serve(list(arr))
        r = {"poisson_lambda_per_s": lam, "p50_s": float(np.percentile(lat, 50)),
             "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
             "throughput_requests_per_s": n / wall, "throughput_particle_updates_per_s": work / wall,
             "ticks": st["ticks"], "packed_particle_launches": st["particle_launches"]}
        if frac == 0.8:
            out.update(r)  # the headline arrival rate
        else:
            out["at_0.5x"] = r
    return out


def _oracle_sample(wl_name, seed_offset=0):
    """A bounded sample of the workload for the CPU oracle: the same recipe at
    reduced extents (the full ones take minutes per step on one core)."""
    from paper_2104_11385_gb300 import workloads as W
    if wl_name == "foil_at_scale":
        return (W.foil_at_scale(seed=5 + seed_offset, scale=8),
                "foil-at-scale recipe at 1/8 extents: 64x64x128 cells, foil 2 cells thick, 64 ppc per species")
    if wl_name == "foil256":
        return W.foil256(seed=2 + seed_offset, scale=4), "foil256 recipe at 1/4 extents: 64^3 cells, foil 2 cells thick"
    if wl_name == "uniform32":
        return W.uniform32(seed=1 + seed_offset), "uniform32 in full: 32^3 cells"
    if wl_name == "laser_ion_2d":
        return W.laser_ion_2d(seed=6 + seed_offset, scale=8), "laser-ion 2D recipe at 1/8 extents: 240^2 cells"
    return W.lognormal(seed=3 + seed_offset, nbox=(4, 4, 4)), "lognormal recipe on 4^3 boxes of 16^3"


def oracle_rate(wl_name, budget_s=15.0, steps=1, seed_offset=0):
    """The FP64 CPU oracle as it stands, on a bounded sample of the workload,
    timed over up to `steps` full PIC cycles within budget_s on one host core."""
    import oracle as orc
    wl, sample = _oracle_sample(wl_name, seed_offset)
    ref = orc.OracleSim(wl["dim"], wl["ncell"], wl["dx"], wl["dt"], wl["order"], wl["absorb"])
    for s in wl["species"]:
        ref.add_species(s["q"], s["m"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"], s["id"])
    if wl.get("laser"):
        L = wl["laser"]
        ref.set_laser(L["a0"], L["w0"], L["tau"], L["t_peak"], L["omega"], L["xc"], L["yc"], L["k_ant"])
    nparts = sum(len(s["x"]) for s in wl["species"])
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        ref.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    secs = time.perf_counter() - t0
    return nparts * done / secs, "%s, %d particles, %d step(s)" % (sample, nparts, done), secs


def _oracle_worker(task):
    """One host core's share of the all-core baseline (a process of its own)."""
    wl_name, seed_offset, steps = task
    r, sample, secs = oracle_rate(wl_name, budget_s=1e9, steps=steps, seed_offset=seed_offset)
    return r, sample, secs


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baselines(wl_name):
    """The FP64 CPU oracle on the host: one core on a bounded sample; every core
    at once, each on an independent sample of the same recipe (one process per
    core, spawned); and the small uniform plasma in full on one core."""
    import multiprocessing as mp
    r, sample, secs = oracle_rate(wl_name, budget_s=25.0, steps=15)
    ncores = os.cpu_count() or 1
    out = {"value": r, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
           "sample": sample + " (%.1f s of CPU time)" % secs, "nproc": ncores, "cpu_model": cpu_model()}
    try:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(ncores) as pool:
            res = pool.map(_oracle_worker, [(wl_name, 100 + i, 4) for i in range(ncores)])
        wall = time.perf_counter() - t0
        out["all_cores"] = {"value": sum(x[0] for x in res), "unit": "particle-updates/s", "cores": ncores,
                            "sample": "%d independent samples at once (seeds offset 100..%d), each: %s"
                                      % (ncores, 99 + ncores, res[0][1]),
                            "wall_s": wall, "what": "sum of the per-process rates; one oracle process per core"}
    except Exception as e:  # the all-core figure is optional context
        out["all_cores"] = {"error": str(e)[:200]}
    r1, s1, secs1 = oracle_rate("uniform32", budget_s=60.0, steps=50)
    out["uniform32_full"] = {"value": r1, "unit": "particle-updates/s", "cores": 1,
                             "sample": s1 + " (%.1f s)" % secs1}
    return out


def run_timeline(args):
    """The paper's comparison of load-balancing modes over a run (Sec. 3.2):
    the same workload, launch and schedule under no balancing (the fixed
    equal-count Morton mapping), static balancing (once, at the first
    interval) and dynamic balancing (every interval, threshold theta), with
    the time per step and E (Eq. 1) of the mapping in force every interval.
    Dynamic balancing runs with both of the paper's policies: knapsack and
    the Morton space-filling curve."""
    import torch
    import paper_2104_11385_gb300 as pic
    wl = make_workload(args.workload, args.scale)
    interval = int(wl.get("lb_interval", 10))
    nint = max(1, args.timeline // interval)
    sched = pic.SCHED_LISTS if args.sched == "lists" else pic.SCHED_QUEUE
    stream = torch.cuda.Stream()
    out = {}
    known = {"none": (pic.LB_NONE, pic.POLICY_KNAPSACK, pic.COST_DEVICE_CLOCK),
             "static": (pic.LB_STATIC, pic.POLICY_KNAPSACK, pic.COST_DEVICE_CLOCK),
             "dynamic": (pic.LB_DYNAMIC, pic.POLICY_KNAPSACK, pic.COST_DEVICE_CLOCK),
             "dynamic_sfc": (pic.LB_DYNAMIC, pic.POLICY_SFC, pic.COST_DEVICE_CLOCK),
             "dynamic_heuristic": (pic.LB_DYNAMIC, pic.POLICY_KNAPSACK, pic.COST_HEURISTIC),
             "dynamic_kernel_time": (pic.LB_DYNAMIC, pic.POLICY_KNAPSACK, pic.COST_KERNEL_TIME)}
    modes = [m for m in args.timeline_modes.split(",") if m]
    for name in modes:
        mode, policy, cost = known[name]
        sim = pic.from_workload(wl, stream=stream.cuda_stream)
        sim.set_lb_params(mode=mode, interval=interval, theta=0.10, policy=policy,
                          cost=cost, split=args.split, sched=sched)
        sim.set_launch(threads=args.threads or 256, ctas_per_sm=args.ctas_per_sm or 2,
                       precision=args.precision)
        ms, eff = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(nint):
            nlog = len(sim.lb_log())
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(interval)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1) / interval)
            log = sim.lb_log()[nlog:]
            # E of the mapping used during this interval: the load-balancing
            # call at its end measured it (e_old); otherwise read it and start
            # a new cost window
            # (for dynamic_heuristic and dynamic_kernel_time that call's E is in
            # its own cost measure; the time per step is the common yardstick)
            eff.append(log[-1]["e_old"] if log else sim.efficiency(reset_window=True))
        lbl = sim.lb_log()
        sim.close()
        del sim
        torch.cuda.empty_cache()
        out[name] = {"total_ms": sum(ms) * interval, "ms_per_step": ms, "E": eff,
                     "mean_E": sum(eff) / len(eff),
                     "adopted": sum(1 for r in lbl if r["adopted"]), "lb_calls": len(lbl)}
    line = {"metric": "lb_timeline", "workload": workload_desc(wl), "steps_per_mode": nint * interval,
            "interval": interval, "sched": args.sched, "theta": 0.10,
            "launch": {"threads": args.threads or 256, "ctas_per_sm": args.ctas_per_sm or 2,
                       "precision": args.precision},
            "modes": out}
    for a, b, key in (("none", "static", "speedup_static_over_none"), ("none", "dynamic", "speedup_dynamic_over_none"),
                      ("static", "dynamic", "speedup_dynamic_over_static"),
                      ("dynamic_sfc", "dynamic", "speedup_knapsack_over_sfc"),
                      ("dynamic_heuristic", "dynamic", "speedup_device_clock_over_heuristic"),
                      ("dynamic_kernel_time", "dynamic", "speedup_device_clock_over_kernel_time")):
        if a in out and b in out:
            line[key] = out[a]["total_ms"] / out[b]["total_ms"]
    print(json.dumps(line, default=_jsonable), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm is the FP64 CPU oracle, timed as it stands on the host cores
        for _ in range(args.warmup):
            oracle_rate(args.workload, budget_s=5.0, steps=1)
        rates = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r, sample, _ = oracle_rate(args.workload, budget_s=5.0, steps=1)
            rates.append(r)
        secs = time.perf_counter() - t0
        v = statistics.median(rates)
        wl_name = workload_name(args)
        line = {"metric": "particle-updates/s", "value": v, "unit": "particle-updates/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / max(args.steps, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": wl_name + " (bounded sample)", "sample": sample},
                "cpu_baseline": {"value": v, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
                                 "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
                "e2e": {"value": v, "unit": "particle-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if args.timeline > 0:
        if rank == 0:
            run_timeline(args)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_ours(args, rank, world)
    sec = None
    if rank == 0 and args.secondary != "none" and args.secondary != args.workload:
        import torch
        torch.cuda.empty_cache()
        sec = run_ours(args, 0, 1, wl=make_workload(args.secondary, args.scale), full=False)
        sec = {"workload": sec["config"], "value": sec["value"], "unit": "particle-updates/s",
               "ms_per_step": sec["ms_per_step"], "step_time_spread": sec["step_time_spread"],
               "phase_ms_per_step": sec["phase_ms_per_step"], "static_order": sec["static_order"], "mixed_precision": sec["mixed_precision"],
               "fp32": sec["fp32"], "fdtd_cell_updates_per_s": sec["fdtd_cell_updates_per_s"],
               "hbm_frac_fp64": BYTES_PER_PARTICLE * sec["_nparts"]
               / (sec["phase_ms_per_step"]["particle"] / 1e3) / 1e9 / hbm_peak_gbs()}
    server = None
    if rank == 0 and not args.no_server:
        server = run_server(args)
    c3 = None
    if rank == 0 and not args.no_c3:
        c3 = run_c3(args)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baselines(args.workload)
    if rank == 0:
        line = {"metric": "particle-updates/s", "value": res["value"], "unit": "particle-updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["ms_per_step"], "step_time_spread": res["step_time_spread"],
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {1: "f64", 2: "float-float", 3: "f32"}[args.precision],
                "data": "synthetic (seeded PCG64 workload recipe)", "config": res["config"],
                "clocks": res["clocks"], "e2e": res.get("e2e"),
                "gpu_launches": res["gpu_launches"], "roofline": res["roofline"], "cpu_baseline": cpu,
                "static_order": res["static_order"], "cutting_vs_ordering": res.get("cutting_vs_ordering"),
                "other_schedule": res.get("other_schedule"),
                "cost_strategies": res.get("cost_strategies"), "mixed_precision": res["mixed_precision"],
                "fp32": res["fp32"], "secondary": sec,
                "batched_uneven_boxes": c3,
                "cell_updates_per_s": res["cell_updates_per_s"],
                "fdtd_cell_updates_per_s": res["fdtd_cell_updates_per_s"],
                "phase_ms_per_step": res["phase_ms_per_step"], "lb": res["lb"], "server": server}
        print(json.dumps(line, default=_jsonable), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def workload_name(args):
    names = {"foil_at_scale": "foil512x512x1024", "foil256": "foil256x256x256", "uniform32": "uniform32",
             "lognormal4096": "lognormal4096", "laser_ion_2d": "laser_ion_2d_1920"}
    return names.get(args.workload, args.workload)


if __name__ == "__main__":
    main()
