"""Continuous-batching server for foam simulations on one GPU.

Requests (box size, bubbles, step count, storage) arrive over time. The
server keeps every admitted box resident in HBM, admits waiting requests in
arrival order as long as their workspace (lbm_workspace_bytes) fits the
memory budget and a box slot is free, and advances all resident boxes
together: one batch per storage type (each on its own stream, so the two
overlap on the device), in short quanta shared fairly by work, so that new
arrivals join within a quantum and small requests overtake large ones. A box
leaves at the end of the quantum in which its step count is reached; its
result is read then and its memory returned at the next admission. Every box evolves
bitwise as it would alone (batches keep the single-box arithmetic), so a
result does not depend on what else was in the mix.

`run_one_at_a_time` processes the same arrival stream with the plain method:
one request at a time, in arrival order, each stepped alone.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field

import numpy as np

from .lbm import Batch, Simulation, lbm_workspace_bytes, make_config


@dataclass
class Request:
    rid: int
    arrival_s: float
    nx: int
    ny: int
    bubbles: np.ndarray          # (n, 3) cx, cy, r
    steps: int
    storage: str = "f16"         # "f32" | "f16" | "bf16"
    rho_l: float = 2.306865
    rho_g: float = 0.104158
    barrier: bool = True
    relabel_every: int = 10


@dataclass
class Result:
    rid: int
    arrival_s: float
    admit_s: float
    done_s: float
    steps: int
    cells: int
    mass: float
    n_bubbles: int
    gas_fraction: float
    pops: np.ndarray | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def config_of(req: Request):
    return make_config(req.nx, req.ny, storage=req.storage, barrier=req.barrier,
                       relabel_every=req.relabel_every, rho_ref=req.rho_l)


def footprint_bytes(req: Request) -> int:
    """Device bytes a request holds while resident (its workspace)."""
    return int(lbm_workspace_bytes(config_of(req)))


def _make_box(req: Request, device) -> Simulation:
    sim = Simulation(config_of(req), device=device)
    sim.init_bubbles(req.bubbles, req.rho_l, req.rho_g, 4.0)
    return sim


def _finish(req: Request, sim: Simulation, t0: float, admit_s: float, keep_pops: bool) -> Result:
    st = sim.stats()
    pops = sim.read("pops")["pops"] if keep_pops else None
    return Result(req.rid, req.arrival_s, admit_s, time.perf_counter() - t0, req.steps, req.nx * req.ny,
                  st["mass"], st["n_bubbles"], st["gas_fraction"], pops)


@dataclass
class _Job:
    req: Request
    sim: Simulation
    remaining: int
    admit_s: float
    nbytes: int

    @property
    def cells(self) -> int:
        return self.req.nx * self.req.ny


def fair_steps(jobs: list[_Job], budget_updates: float) -> dict[int, int]:
    """Steps per job for one quantum: the cell-update budget is shared equally
    among the jobs (processor sharing by work), a job needing less than its
    share takes all its remaining steps and leaves the rest to the others
    (water-filling), and every job advances at least one step."""
    out: dict[int, int] = {}
    left = float(budget_updates)
    order = sorted(jobs, key=lambda j: j.remaining * j.cells)
    for k, j in enumerate(order):
        share = max(0.0, left) / (len(order) - k)
        s = j.remaining if j.remaining * j.cells <= share else max(1, int(share // j.cells))
        s = min(s, j.remaining)
        out[j.req.rid] = s
        left -= s * j.cells
    return out


@dataclass
class FoamServer:
    """Continuous batching: each quantum (about `quantum_s` of GPU time, from
    a running estimate of the update rate, or exactly `quantum_updates` cell
    updates when given) is split fairly between the resident boxes with
    `fair_steps`, and every batch runs its share as multi-rate steps
    (lbm_batch_step_each): small boxes take many cheap steps while large ones
    take few, so a small request is not held to the pace of the largest box."""
    memory_budget_bytes: int
    max_boxes: int = 64
    quantum_s: float = 0.02
    quantum_updates: float | None = None
    device: str = "cuda"
    keep_pops: bool = False
    stats: dict = field(default_factory=dict)

    def run(self, requests: list[Request]) -> list[Result]:
        """Serves `requests` (arrival times relative to the call) to completion.

        Membership changes cost a batch rebuild (descriptor upload), so they
        are batched too: a box that finishes is only switched off in its
        batch and its memory is given back at the next admission, which
        rebuilds the batches once for every request admitted at that point."""
        import torch

        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque[Request] = collections.deque()
        active: dict[int, _Job] = {}
        parked: list[_Job] = []            # finished, still held by a batch
        batches: dict[str, tuple[Batch, list[_Job]]] = {}
        results: list[Result] = []
        used = 0                           # bytes of boxes still stepping
        peak_held = 0
        rebuilds = quanta = 0
        rate = 3e10                        # cell updates per second, refined as we go
        t_admit = t_step = t_finish = 0.0
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            admit: list[Request] = []
            want = used
            while waiting and len(active) + len(admit) < self.max_boxes:
                need = footprint_bytes(waiting[0])
                if need > self.memory_budget_bytes:
                    raise ValueError(f"request {waiting[0].rid} needs {need} bytes, more than the whole budget")
                if want + need > self.memory_budget_bytes:
                    break
                admit.append(waiting.popleft())
                want += need
            if admit:
                ta = time.perf_counter()
                for b, _ in batches.values():
                    b.close()
                batches = {}
                if parked:
                    parked.clear()
                    torch.cuda.empty_cache()
                for r in admit:
                    active[r.rid] = _Job(r, _make_box(r, self.device), r.steps, time.perf_counter() - t0,
                                         footprint_bytes(r))
                used = want
                peak_held = max(peak_held, used)
                groups: dict[str, list[_Job]] = collections.defaultdict(list)
                for j in active.values():
                    groups[j.req.storage].append(j)
                for storage, jobs in groups.items():
                    batches[storage] = (Batch([j.sim for j in jobs]), jobs)
                rebuilds += 1
                t_admit += time.perf_counter() - ta
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival_s - (time.perf_counter() - t0)))
                continue
            budget = self.quantum_updates if self.quantum_updates else rate * self.quantum_s
            share = fair_steps(list(active.values()), budget)
            ts = time.perf_counter()
            live = []
            for b, jobs in batches.values():
                plan = [share.get(j.req.rid, 0) if j.remaining > 0 else 0 for j in jobs]
                if any(plan):
                    b.step_each(plan)  # each batch on its own stream: the storage classes overlap
                    live.append((b, jobs, plan))
            for b, _, _ in live:
                b.sync()
            dt = time.perf_counter() - ts
            t_step += dt
            done = sum(share[r] * active[r].cells for r in share)
            rate = 0.7 * rate + 0.3 * done / max(dt, 1e-6)
            quanta += 1
            tf = time.perf_counter()
            for b, jobs, plan in live:
                for i, (j, s) in enumerate(zip(jobs, plan)):
                    if s == 0:
                        continue
                    j.remaining -= s
                    if j.remaining == 0:
                        b.set_active(i, False)
                        active.pop(j.req.rid)
                        results.append(_finish(j.req, j.sim, t0, j.admit_s, self.keep_pops))
                        used -= j.nbytes
                        parked.append(j)
            t_finish += time.perf_counter() - tf
        for b, _ in batches.values():
            b.close()
        self.stats = {"makespan_s": time.perf_counter() - t0, "peak_bytes": peak_held,
                      "batch_rebuilds": rebuilds, "quanta": quanta, "admit_s": round(t_admit, 4),
                      "step_s": round(t_step, 4), "finish_s": round(t_finish, 4),
                      "rate_mlups": round(rate / 1e6, 1)}
        return results


def run_one_at_a_time(requests: list[Request], device: str = "cuda", keep_pops: bool = False):
    """The plain method: requests in arrival order, each stepped alone."""
    import torch

    results = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival_s):
        wait = r.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        admit = time.perf_counter() - t0
        sim = _make_box(r, device)
        sim.step(r.steps)
        results.append(_finish(r, sim, t0, admit, keep_pops))
        del sim
        torch.cuda.empty_cache()
    return results, time.perf_counter() - t0


def summarize(results: list[Result], makespan_s: float) -> dict:
    lat = sorted(r.latency_s for r in results)
    updates = sum(r.cells * r.steps for r in results)

    def pct(p):
        k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[k]

    return {"requests": len(results), "p50_s": round(pct(50), 4), "p99_s": round(pct(99), 4),
            "mean_s": round(statistics.mean(lat), 4), "makespan_s": round(makespan_s, 3),
            "mlups": round(updates / makespan_s / 1e6, 1), "cell_updates": updates}
