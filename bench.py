#!/usr/bin/env python
"""Benchmark of the extended Shan-Chen LB time step on GB300.

Default workload (one GPU): an 8192 x 8192 periodic D2Q9 box with 400
Poisson-disk gas bubbles (radii 8-64, log-uniform, edge gap >= 2), G = -5.5,
tau = 1, psi = 1 - exp(-rho), film barrier on (R_z = 4, relabel every
K = 10 steps). A "step" is one full time step of the method: the barrier
pipeline when due, then the fused pull-stream/force/collide kernel.

Prints one JSON line. `value` is whole-job MLUPS (FP32 storage) with the
state resident in HBM; the FP16-deviation-storage run and the every-step
barrier variant are reported beside it. `roofline` relates the fused step
kernel's algorithmic bytes (9 population reads + 9 writes + 1 mask byte per
cell) to the measured HBM copy bandwidth. `cpu_baseline` is the FP64 oracle
timed on the host cores on a bounded sample. `e2e` runs whole jobs through
the public C ABI from pinned host memory (density in, density out).

Multi-GPU: the path is run as independent replicas (one box per rank, no
collective in the data path); `value` sums all ranks' cell updates over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM roofline fraction (FP32 vs FP16-store) at 8192^2; served p50/p99"
WORKLOADS = {
    "c3": dict(n=8192, bubbles=400, rmin=8.0, rmax=64.0, seed=21,
               desc="8192^2 periodic D2Q9, 400 Poisson-disk bubbles r 8-64 log-uniform (gap>=2), "
                    "G=-5.5, tau=1, psi=1-exp(-rho), film barrier on (R_z=4)"),
    "small": dict(n=2048, bubbles=25, rmin=8.0, rmax=64.0, seed=21,
                  desc="2048^2 periodic D2Q9, 25 Poisson-disk bubbles r 8-64 (profiling case)"),
    "mid": dict(n=4096, bubbles=100, rmin=8.0, rmax=64.0, seed=21,
                desc="4096^2 periodic D2Q9, 100 Poisson-disk bubbles r 8-64 (profiling case, state > L2)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c3")
    ap.add_argument("--relabel-every", type=int, default=10)
    ap.add_argument("--storage", choices=["f32", "f16", "both"], default="both")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-k1", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-growth", action="store_true", help="skip the nucleation/growth leg")
    ap.add_argument("--no-2c", action="store_true", help="skip the two-component leg")
    ap.add_argument("--serve-requests", type=int, default=192)
    ap.add_argument("--serve-step-scale", type=float, default=0.1)
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    ap.add_argument("--serve-policy", default="hrrn",
                    choices=["work", "time", "lockstep", "tiered", "fifo", "express", "srpt", "hrrn"])
    ap.add_argument("--serve-age-weight", type=float, default=0.5,
                    help="srpt policy: requests are ordered by remaining GPU time minus this times the time waited")
    ap.add_argument("--serve-big-s", type=float, default=0.02,
                    help="tiered and express policies: requests with more GPU time left than this are served first come, "
                         "first served")
    ap.add_argument("--serve-big-slowdown", type=float, default=float("inf"),
                    help="tiered policy: past this slowdown of the oldest big request the small ones' share "
                         "is cut to --serve-late-share")
    ap.add_argument("--serve-late-share", type=float, default=0.0)
    ap.add_argument("--serve-small-share", type=float, default=0.5,
                    help="tiered policy: most of each quantum that small requests take while a big one runs")
    ap.add_argument("--serve-load", type=float, default=0.9,
                    help="offered load as a fraction of the one-box-at-a-time throughput")
    ap.add_argument("--batch-step-scale", type=float, default=1.0)
    ap.add_argument("--clocks-dir", default=os.path.join(ROOT, "bench_out"),
                    help="directory for the nvidia-smi clock samples taken during the timed region")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


TRAFFIC_SOURCES = {"step": ("step.cu", "lbm_internal.cuh", "tma.cuh"),
                   "step2": ("step2.cu", "lbm_internal.cuh", "tma.cuh")}


def sources_sha256(kind: str) -> str:
    """Hash of the code (comments and whitespace left out) of the sources a
    step kernel is built from."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[kind]:
        text = open(os.path.join(ROOT, "paper_1708_01613_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def kernel_traffic(key: str, cells: int):
    """DRAM bytes per launch of a fused step kernel ("f32", "f16" or
    "two_component") from the committed ncu summary, if it was taken on the
    current kernel sources and on a box of this many cells (else None)."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    entry = d.get(key, {})
    kind = "step2" if key == "two_component" else "step"
    if d.get("cells") != cells or d.get("sources_sha256", {}).get(kind) != sources_sha256(kind):
        return None
    v = entry.get("bytes_per_launch_full")
    return float(v) if v else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int, directory: str):
        self.index = index
        self.proc = None
        self.path = os.path.join(directory, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        return summarize_clocks(self.path)


def summarize_clocks(path: str):
    """Median SM clock, maximum clock and the throttle reasons seen in an
    nvidia-smi CSV (index, clocks.sm, clocks.max.sm, power, reasons mask,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap);
    None without samples."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v: float, device=None) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- GPU arm
def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import inputs
    from paper_1708_01613_gb300 import Simulation, make_config
    from paper_1708_01613_gb300 import lbm as L

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    n = wl["n"]
    N = n * n
    bub = inputs.poisson_disk_bubbles(n, n, wl["bubbles"], wl["rmin"], wl["rmax"], 2.0,
                                      seed=wl["seed"] + 1000 * rank)
    RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
    peak, peak_kind = measured_peaks()
    K = args.relabel_every

    def timed(storage: str, relabel_every: int, steps: int, warmup: int, sample_clocks: bool, growth=None):
        sim = Simulation(make_config(n, n, storage=storage, barrier=True, relabel_every=relabel_every,
                                     rho_ref=RL, growth=growth is not None), device=dev)
        sim.init_bubbles(bub, RL, RG, 4.0)
        if growth is not None:
            sim.set_growth(*growth)
        sim.step(warmup)
        sim.sync()
        stream = sim.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local, args.clocks_dir) if sample_clocks else None
        if sampler:
            sampler.start()
        barrier(world)
        torch.cuda.synchronize(dev)
        launches0 = sim.kernel_launches
        t_first = sim.steps_done
        t_all0.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        clocks = sampler.stop() if sampler else None
        launches = sim.kernel_launches - launches0
        sim.sync()  # raises on a device-side numeric fault
        total_ms = t_all0.elapsed_time(t_all1)
        per = [a.elapsed_time(b) for a, b in ev]
        plain = [d for k, d in enumerate(per) if (t_first + k) % relabel_every != 0]
        relab = [d for k, d in enumerate(per) if (t_first + k) % relabel_every == 0]
        st = sim.stats()
        released = sim.growth_released if growth is not None else 0.0
        del sim
        torch.cuda.empty_cache()
        return dict(total_ms=total_ms, per=per, plain=plain, relab=relab, launches=launches,
                    clocks=clocks, stats=st, released=released)

    def roofline(storage, r):
        eb = 4 if storage == "f32" else 2
        bytes_cell = 2 * 9 * eb + 1
        kern_ms = statistics.mean(r["plain"]) if r["plain"] else r["total_ms"] / args.steps
        achieved = bytes_cell * N / (kern_ms * 1e-3) / 1e9
        traffic = kernel_traffic(storage, N)
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else peak_kind,
                "algorithmic_bytes_per_cell": bytes_cell,
                "kernel": "k_step_dyn" if n % 16 == 0 else "k_step_strip",
                "kernel_ms_avg": round(kern_ms, 5),
                "kernel_mlups": round(N / (kern_ms * 1e-3) / 1e6, 1),
                "roofline_mlups": round(peak * 1e9 / bytes_cell / 1e6, 1)}

    results = {}
    storages = ["f32", "f16"] if args.storage == "both" else [args.storage]
    for s in storages:
        results[s] = timed(s, K, args.steps, args.warmup, sample_clocks=(s == storages[0]))
    primary = storages[0]
    r0 = results[primary]
    tmax = max_over_ranks(world, r0["total_ms"], dev)
    value = world * N * args.steps / (tmax * 1e-3) / 1e6
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tmax / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if primary == "f32" else "f16-storage/f32-math", "data": "synthetic",
        "config": {"workload": wl["desc"], "cells": N, "storage": primary, "relabel_every": K,
                   "zone_radius": 4, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: the resident state (>= 2.4 GB) is far larger than L2",
                   "per_rank_seed_offset": 1000},
        "roofline": roofline(primary, r0),
        "gpu_launches": int(r0["launches"]),
        "clocks": r0["clocks"],
        "relabel_ms_avg": round(statistics.mean(r0["relab"]) - statistics.mean(r0["plain"]), 4)
        if r0["relab"] and r0["plain"] else None,
        "bubbles_after": {"n": r0["stats"]["n_bubbles"], "gas_fraction": r0["stats"]["gas_fraction"]},
    }
    for s in storages[1:]:
        r = results[s]
        t = max_over_ranks(world, r["total_ms"], dev)
        out[s] = {"value": round(world * N * args.steps / (t * 1e-3) / 1e6, 1),
                  "ms_per_step": round(t / args.steps, 5), "roofline": roofline(s, r),
                  "gpu_launches": int(r["launches"])}
    if not args.no_k1:
        ksteps = max(5, min(args.steps, 20))
        r = timed(primary, 1, ksteps, min(args.warmup, 3), sample_clocks=False)
        t = max_over_ranks(world, r["total_ms"], dev)
        out["barrier_every_step"] = {"value": round(world * N * ksteps / (t * 1e-3) / 1e6, 1),
                                     "ms_per_step": round(t / ksteps, 5), "steps": ksteps,
                                     "relabel_every": 1}
    if not args.no_growth and "f32" in results:
        # nucleation/growth source (Sec. 2.1.3) on the same FP32 box: census with
        # every relabel, one growth launch after every step
        rate, budget = 100.0, 1e9
        r = timed("f32", K, args.steps, min(args.warmup, 3), sample_clocks=False, growth=(rate, budget))
        t = max_over_ranks(world, r["total_ms"], dev)
        base = results["f32"]
        out["growth"] = {"value": round(world * N * args.steps / (t * 1e-3) / 1e6, 1), "unit": "MLUPS",
                         "ms_per_step": round(t / args.steps, 5),
                         "release_per_step": rate, "released": r["released"],
                         "extra_ms_per_plain_step": round(statistics.mean(r["plain"]) - statistics.mean(base["plain"]), 5)
                         if r["plain"] and base["plain"] else None,
                         "extra_ms_per_relabel_step": round(statistics.mean(r["relab"]) - statistics.mean(base["relab"]), 5)
                         if r["relab"] and base["relab"] else None,
                         "storage": "f32", "gpu_launches": int(r["launches"])}
    if not args.no_2c:
        out["two_component"] = run_two_component(args, dev, n, bub, RL, RG, world, peak, peak_kind)
        if rank == 0 and not args.no_cpu:
            out["two_component"]["cpu_baseline"] = cpu_sample_two_component()
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, dev, n, bub, RL, RG, world)
    if not args.no_batch:
        out["batched"] = run_batched(args, dev, world, rank)
    if not args.no_serve:
        cap = out.get("batched", {}).get("sequential", 45000.0) * 1e6
        out["served"] = run_served(args, dev, world, rank, cap)
    return out


def run_two_component(args, dev, n, bub, RL, RG, world, peak, peak_kind):
    """Two-component variant (melt and gas lattices) on the benchmark box:
    melt density of the foam, a gas component filling the bubbles (0.3 inside,
    0.005 outside), G_mm = -5.5, G_mg = 1.0, FP32, barrier on, K as the main
    leg. Roofline of the fused two-lattice step: 2 x 18 x 4 + 1 = 145 B/cell."""
    import numpy as np
    import torch

    import inputs
    from paper_1708_01613_gb300 import Simulation, make_config

    N = n * n
    K = args.relabel_every
    sim = Simulation(make_config(n, n, components=2, barrier=True, relabel_every=K, G_mg=1.0), device=dev)
    prof = Simulation(make_config(n, n, barrier=False), device=dev)  # density of the foam, FP64 tanh profile
    prof.init_bubbles(bub, RL, RG, 4.0)
    rm = prof.read("rho", device=True)["rho"].to(torch.float64)
    del prof
    rg = 0.005 + 0.3 * (RL - rm) / (RL - RG)
    sim.init_density(rm.cpu().numpy(), rg.cpu().numpy())
    del rm, rg
    sim.step(min(args.warmup, 3))
    sim.sync()
    stream = sim.stream
    steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    t_first = sim.steps_done
    l0 = sim.kernel_launches
    for k in range(steps):
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    sim.sync()
    per = [a.elapsed_time(b) for a, b in ev]
    plain = [d for k, d in enumerate(per) if (t_first + k) % K != 0]
    kern_ms = statistics.mean(plain) if plain else sum(per) / steps
    total = max_over_ranks(world, sum(per), dev)
    bytes_cell = 2 * 18 * 4 + 1
    achieved = bytes_cell * N / (kern_ms * 1e-3) / 1e9
    out = {"value": round(world * N * steps / (total * 1e-3) / 1e6, 1), "unit": "MLUPS",
           "ms_per_step": round(total / steps, 5), "storage": "f32", "components": 2,
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": kernel_traffic("two_component", N),
                        "algorithmic_bytes_per_cell": bytes_cell,
                        "kernel": "k_step2_tma" if n % 16 == 0 and n >= 272 else "k_step2_strip",
                        "kernel_ms_avg": round(kern_ms, 5), "peak_kind": peak_kind},
           "gpu_launches": int(sim.kernel_launches - l0)}
    del sim
    torch.cuda.empty_cache()
    return out


def run_served(args, dev, world, rank, capacity_ups):
    """Continuous-batching server on a Poisson request stream (sides 128-4096
    log-uniform, 2-300 bubbles, 1k-20k steps scaled by `serve_step_scale`,
    half FP32 and half FP16 storage), offered load `serve_load` of the
    one-box-at-a-time throughput measured above; against the same stream run
    one at a time."""
    import math

    import torch

    import inputs
    from paper_1708_01613_gb300.serve import FoamServer, Request, run_one_at_a_time, summarize

    n = args.serve_requests
    scale = args.serve_step_scale
    raw = inputs.serving_requests(count=n, rate_per_s=1.0, seed=41 + 1000 * rank)
    work = [r["nx"] * r["ny"] * max(20, int(round(r["steps"] * scale))) for r in raw]
    rate = args.serve_load * capacity_ups / (sum(work) / len(work))
    reqs = []
    for r in raw:
        bub = inputs.request_bubbles(r)
        reqs.append(Request(r["id"], r["arrival_s"] / rate, r["nx"], r["ny"], bub,
                            max(20, int(round(r["steps"] * scale))), r["storage"],
                            inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55, True, 10))
    torch.cuda.synchronize(dev)
    server = FoamServer(memory_budget_bytes=int(args.serve_budget_gb * 2**30), max_boxes=32, device=str(dev),
                        policy=args.serve_policy, big_s=args.serve_big_s, small_share=args.serve_small_share,
                        big_slowdown=args.serve_big_slowdown, late_share=args.serve_late_share,
                        age_weight=args.serve_age_weight)
    served = summarize(server.run(reqs), server.stats["makespan_s"])
    alone_res, alone_span = run_one_at_a_time(reqs, device=str(dev))
    alone = summarize(alone_res, alone_span)
    reduced = n < 2000 or scale < 1.0
    return {"workload": ("reduced stream: " if reduced else "") +
                        f"{n} requests (the configuration: 2000), Poisson arrivals at offered load "
                        f"{args.serve_load} of the one-at-a-time throughput, sides "
                        "128-4096 log-uniform (any integer), 2-300 bubbles, 1k-20k steps x step_scale "
                        f"({scale}), FP32/FP16 50/50, barrier on (K=10)",
            "reduced": reduced,
            "step_scale": scale, "rate_per_s": round(rate, 3), "memory_budget_gb": args.serve_budget_gb,
            "policy": server.policy, "big_s": server.big_s, "small_share": server.small_share,
            "big_slowdown": server.big_slowdown, "late_share": server.late_share,
            "age_weight": server.age_weight, "quantum_s": server.quantum_s,
            "p50_s": served["p50_s"], "p99_s": served["p99_s"], "mean_s": served["mean_s"],
            "p50_by_size_s": served["p50_by_size_s"], "mlups": served["mlups"],
            "makespan_s": served["makespan_s"], "batch_rebuilds": server.stats["batch_rebuilds"],
            "server": {k: server.stats[k] for k in ("quanta", "admit_s", "step_s", "finish_s", "rate_mlups")},
            "peak_resident_gb": round(server.stats["peak_bytes"] / 2**30, 2),
            "one_at_a_time": {"p50_s": alone["p50_s"], "p99_s": alone["p99_s"], "mean_s": alone["mean_s"],
                              "p50_by_size_s": alone["p50_by_size_s"], "mlups": alone["mlups"],
                              "makespan_s": alone["makespan_s"]}}


def run_batched(args, dev, world, rank):
    """64 independent boxes of mixed size (sides 256-2048 log-uniform, 5-200
    bubbles, 1k-20k steps each, FP16-deviation storage, barrier on, K = 10):
    one batch (persistent launch per step, graphs, autotuned tiles) against the
    same boxes stepped one after another with lbm_step. Both time exactly
    sum_i cells_i * steps_i updates; `step_scale` shrinks all step counts."""
    import torch

    import inputs
    from paper_1708_01613_gb300 import Batch, Simulation, make_config

    RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
    specs = inputs.batch_instances(count=64, seed=31 + 1000 * rank)
    scale = args.batch_step_scale
    steps = [max(10, int(round(s["steps"] * scale))) for s in specs]

    def boxes():
        out = []
        for s in specs:
            sim = Simulation(make_config(s["nx"], s["ny"], storage="f16", barrier=True, relabel_every=10,
                                         rho_ref=RL), device=dev)
            sim.init_bubbles(s["bubbles"], RL, RG, 4.0)
            out.append(sim)
        return out

    updates = sum(s["nx"] * s["ny"] * k for s, k in zip(specs, steps))
    # one box after another, each with its own launches per step
    seq = boxes()
    for sim in seq:
        sim.step(1)
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    for sim, k in zip(seq, steps):
        sim.step(k)
    torch.cuda.synchronize(dev)
    t_seq = max_over_ranks(world, time.perf_counter() - t0, dev)
    for sim in seq:
        sim.sync()
    del seq
    torch.cuda.empty_cache()
    # the batch: tune tiles (as warm-up), then run every box for its own count
    bat_boxes = boxes()
    bat = Batch(bat_boxes)
    tune_ms = bat.tune(trial_steps=2)
    strip, rows = bat.tiles
    bat.sync()
    order = sorted(range(len(specs)), key=lambda i: steps[i])
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    done = 0
    for i in order:
        if steps[i] > done:
            bat.step(steps[i] - done)
            done = steps[i]
        bat.set_active(i, False)
    torch.cuda.synchronize(dev)
    t_bat = max_over_ranks(world, time.perf_counter() - t0, dev)
    bat.sync()
    launches = bat.kernel_launches
    bat.close()
    del bat, bat_boxes
    torch.cuda.empty_cache()
    return {"workload": "64 boxes, sides 256-2048 log-uniform (any integer), 5-200 Poisson-disk bubbles, "
                        "1k-20k steps each (log-uniform), FP16-deviation storage, barrier on (K=10, R_z=4)",
            "step_scale": scale, "cell_updates": updates,
            "value": round(world * updates / t_bat / 1e6, 1), "unit": "MLUPS",
            "sequential": round(world * updates / t_seq / 1e6, 1),
            "speedup_vs_sequential": round(t_seq / t_bat, 3),
            "seconds": {"batched": round(t_bat, 3), "sequential": round(t_seq, 3)},
            "tiles": {"strip_width": strip, "chunk_rows": rows, "tune_ms_per_step": round(tune_ms, 4)},
            "graphs": True, "kernel_launches": int(launches)}


def run_e2e(args, dev, n, bub, RL, RG, world):
    """Whole jobs through the C ABI from pinned host memory: density in
    (FP64), `job_steps` steps, density out (FP32), synchronised."""
    import numpy as np
    import torch

    import inputs
    from paper_1708_01613_gb300 import lbm as L

    N = n * n
    job_steps = 100
    lib = L.load_library()
    cfg = L.make_config(n, n, storage="f32", barrier=True, relabel_every=args.relabel_every, rho_ref=RL)
    nbytes = L.lbm_workspace_bytes(cfg)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = C.c_void_p()
    L._check(lib.lbm_create(C.byref(cfg), C.c_void_p((ws.data_ptr() + 255) // 256 * 256), nbytes,
                            C.c_void_p(stream.cuda_stream), C.byref(h)))
    rho_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    out_host = torch.empty(N, dtype=torch.float32, pin_memory=True)
    # the initial density of the job (made once on the host, outside the timing)
    sim_tmp = L.Simulation(cfg, device=dev)
    sim_tmp.init_bubbles(bub, RL, RG, 4.0)
    r = sim_tmp.read("rho")["rho"].astype(np.float64).ravel()
    rho_host.copy_(torch.from_numpy(r))
    del sim_tmp
    torch.cuda.empty_cache()

    def job():
        L._check(lib.lbm_init_density(h, C.c_void_p(rho_host.data_ptr()), 0), h)
        L._check(lib.lbm_step(h, job_steps), h)
        L._check(lib.lbm_read_fields(h, L.FIELD_RHO, C.c_void_p(out_host.data_ptr()), 4 * N, 0), h)

    job()
    iters = 3
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(iters):
        job()
    t1 = time.perf_counter()
    barrier(world)
    lib.lbm_destroy(h)
    dt = max_over_ranks(world, t1 - t0, dev)
    return {"value": round(world * N * job_steps * iters / dt / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": 8 * N // job_steps, "d2h_bytes_per_step": 4 * N // job_steps,
            "h2d_bytes_per_job": 8 * N, "d2h_bytes_per_job": 4 * N,
            "job": f"init_density(host FP64) + {job_steps} steps + read_fields(RHO, host)",
            "steps_per_job": job_steps, "jobs": iters}


# ----------------------------------------------------------------- oracle (CPU)
def cpu_sample(steps: int, warmup: int, budget_s: float | None):
    """The FP64 oracle on a 512^2 box with the benchmark's bubble density
    (bubbles per area of the 8192^2 workload, about 1.6 per 512^2: 2 here),
    barrier on, K = 10."""
    import inputs
    import oracle as O

    n = 512
    bub = inputs.poisson_disk_bubbles(n, n, 2, 8.0, 64.0, 2.0, seed=21)
    P = O.make_params(n, n, barrier=True, relabel_every=10)
    s = O.OracleSim(P)
    s.init_density(O.init_bubbles(P, bub, inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55, 4.0))
    s.step(warmup)
    if budget_s is not None:
        t0 = time.perf_counter()
        s.step(2)
        per = (time.perf_counter() - t0) / 2
        steps = max(2, int(budget_s / per))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return n * n * steps / dt / 1e6, steps, dt, O.max_threads()


def cpu_spinodal_config():
    """The FP64 oracle on the spinodal configuration as stated: 128^2,
    rho = 0.7 (1 + 0.01 U[-1, 1)), G = -5.5, 2000 steps (seed 1)."""
    import inputs
    import oracle as O

    n, steps = 128, 2000
    s = O.OracleSim(O.make_params(n, n, G=-5.5))
    s.init_density(inputs.noise_density(n, n, seed=1))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return {"value": round(n * n * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": O.max_threads(),
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": "the whole spinodal run: 128^2, 2000 steps, rho = 0.7 (1 + 0.01 U[-1,1)), G = -5.5"}


def cpu_sample_two_component(budget_s: float = 4.0):
    """The FP64 two-component oracle on a 256^2 box of the two-component
    leg's kind (one melt bubble filled with gas, G_mm = -5.5, G_mg = 1.0,
    barrier on, K = 10), timed for about `budget_s` seconds."""
    import inputs
    import oracle as O

    n = 256
    RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
    rm = O.init_bubbles(O.make_params(n, n), [[n / 2, n / 2, 30.0]], RL, RG, 4.0)
    rg = 0.005 + 0.3 * (RL - rm) / (RL - RG)
    s = O.OracleSim2(O.make_params2(n, n, G_mm=-5.5, G_mg=1.0, barrier=True, relabel_every=10))
    s.init_density(rm, rg)
    s.step(2)
    t0 = time.perf_counter()
    s.step(2)
    steps = max(2, int(budget_s / ((time.perf_counter() - t0) / 2)))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return {"value": round(n * n * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": O.max_threads(),
            "kind": "oracle", "sample": f"{steps} steps of a 256^2 two-component box ({dt:.1f} s, FP64 oracle, OpenMP)"}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        if rank != 0:
            return
        mlups, steps, dt, cores = cpu_sample(args.steps, args.warmup, None)
        out = {"metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / steps * 1e3, 3),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "impl": "reference",
               "config": {"workload": WORKLOADS[args.workload]["desc"],
                          "sample": "512^2 box at the workload's bubble density, barrier on, K=10"},
               "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{steps} steps of a 512^2 box (FP64 oracle, OpenMP)"},
               "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    out = run_gpu(args, world, rank, local)
    if rank == 0 and not args.no_cpu:
        mlups, steps, dt, cores = cpu_sample(0, 2, budget_s=12.0)
        out["cpu_baseline"] = {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                               "sample": f"{steps} steps of a 512^2 box at the workload's bubble density, "
                                         f"barrier on, K=10 ({dt:.1f} s, FP64 oracle, OpenMP)"}
        import oracle as O

        O.set_threads(1)
        m1, s1, d1, _ = cpu_sample(0, 1, budget_s=4.0)
        O.set_threads(cores)
        out["cpu_baseline"]["single_thread"] = {"value": round(m1, 3), "unit": "MLUPS", "cores": 1,
                                                "sample": f"{s1} steps of the same box ({d1:.1f} s, one thread)"}
        out["cpu_baseline"]["spinodal_128"] = cpu_spinodal_config()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
