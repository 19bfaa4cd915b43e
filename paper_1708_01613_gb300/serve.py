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
    return _water_fill(jobs, budget_updates, lambda j: float(j.cells))


def fair_time_steps(jobs: list[_Job], budget_s: float, launch_s: float, s_per_update: float) -> dict[int, int]:
    """Like `fair_steps`, but the shares are GPU time: a step of job j is
    taken to cost launch_s + s_per_update * cells (a small box's step is
    bound by the launch, not by its cells)."""
    return _water_fill(jobs, budget_s, lambda j: launch_s + s_per_update * j.cells)


def lockstep_steps(jobs: list[_Job], budget_s: float, launch_s: float, s_per_update: float) -> dict[int, int]:
    """Every job steps in every launch (until its count is reached); the
    number of launches L is the largest whose predicted time, the sum over
    launches of launch_s + s_per_update * (cells still stepping), fits the
    budget (at least one launch)."""
    by_rem = sorted((j.remaining, j.cells) for j in jobs)
    live = float(sum(c for _, c in by_rem))
    t, L, k = 0.0, 0, 0
    while k < len(by_rem):
        nxt = by_rem[k][0]  # launches L .. nxt-1 step the same set of jobs
        per = launch_s + s_per_update * live
        fit = int((budget_s - t) // per)
        if L + fit < nxt:
            L += max(0, fit)
            break
        t += per * (nxt - L)
        L = nxt
        while k < len(by_rem) and by_rem[k][0] == nxt:
            live -= by_rem[k][1]
            k += 1
    L = max(1, L)
    return {j.req.rid: min(j.remaining, L) for j in jobs}


def tiered_steps(jobs: list[_Job], budget_updates: float, big_updates: float, small_share: float = 0.5) -> dict[int, int]:
    """Two classes: a job with at least `big_updates` cell updates left is
    big. Small jobs share up to `small_share` of the budget by work
    (`fair_steps`; all of it when no big job is resident); the oldest big job
    (by arrival) takes the rest, and the other big jobs wait (0 steps), so
    big requests are served first come, first served at nearly the full rate
    while small ones keep overtaking them."""
    small = [j for j in jobs if j.remaining * j.cells < big_updates]
    big = sorted((j for j in jobs if j.remaining * j.cells >= big_updates), key=lambda j: (j.req.arrival_s, j.req.rid))
    out = {j.req.rid: 0 for j in jobs}
    used = 0.0
    if small:
        share = fair_steps(small, budget_updates * (small_share if big else 1.0))
        out.update(share)
        used = sum(share[j.req.rid] * j.cells for j in small)
    if big:
        j = big[0]
        out[j.req.rid] = min(j.remaining, max(1, int(max(0.0, budget_updates - used) // j.cells)))
    return out


def ordered_steps(jobs: list[_Job], budget_updates: float, key) -> dict[int, int]:
    """Greedy fill in the order `key`: each job in turn takes all its
    remaining steps, or as many as the cell-update budget still allows (at
    least one step for the first job of the order); the jobs after the
    budget runs out wait (0 steps). With `key` the arrival this is first
    come, first served with batching; with the remaining work it is shortest
    remaining processing time first."""
    out = {j.req.rid: 0 for j in jobs}
    left = float(budget_updates)
    for k, j in enumerate(sorted(jobs, key=key)):
        if left <= 0.0 and k > 0:
            break
        s = min(j.remaining, max(1, int(left // j.cells)))
        out[j.req.rid] = s
        left -= s * j.cells
    return out


def order_key(policy: str, now: float, s_per_update: float, age_weight: float = 0.5, big_s: float = 0.02):
    """Sort key of the ordered policies at time `now` (seconds since the
    stream started); ties go to the earlier arrival, then the lower id.
    "fifo": arrival order; "express": jobs with less than `big_s` of GPU
    time left first, arrival order within each class; "srpt": remaining GPU
    time less `age_weight` times the time waited; "hrrn": the highest
    response ratio, time since arrival over remaining GPU time, first."""
    def left(j):
        return j.remaining * j.cells * s_per_update

    if policy == "fifo":
        return lambda j: (j.req.arrival_s, j.req.rid)
    if policy == "express":
        return lambda j: (left(j) >= big_s, j.req.arrival_s, j.req.rid)
    if policy == "srpt":
        return lambda j: (left(j) - age_weight * (now - j.req.arrival_s), j.req.arrival_s, j.req.rid)
    if policy == "hrrn":
        return lambda j: (-(now - j.req.arrival_s) / max(left(j), 1e-9), j.req.arrival_s, j.req.rid)
    raise ValueError(f"no ordered policy {policy!r}")


def _water_fill(jobs: list[_Job], budget: float, cost) -> dict[int, int]:
    out: dict[int, int] = {}
    left = float(budget)
    order = sorted(jobs, key=lambda j: j.remaining * cost(j))
    for k, j in enumerate(order):
        share = max(0.0, left) / (len(order) - k)
        c = cost(j)
        s = j.remaining if j.remaining * c <= share else max(1, int(share // c))
        s = min(s, j.remaining)
        out[j.req.rid] = s
        left -= s * c
    return out


class _CostModel:
    """Quantum time ~ launch_s * launches + s_per_update * updates, fitted
    by least squares over the recent quanta."""

    def __init__(self, launch_s=1e-5, s_per_update=1.0 / 5e10, keep=64):
        self.launch_s, self.s_per_update, self.keep = launch_s, s_per_update, keep
        self.obs: list[tuple[float, float, float]] = []

    def add(self, launches: int, updates: float, seconds: float) -> None:
        self.obs = (self.obs + [(float(launches), float(updates), float(seconds))])[-self.keep:]
        if len(self.obs) < 4:
            return
        A = np.array([[o[0], o[1]] for o in self.obs])
        y = np.array([o[2] for o in self.obs])
        sol, *_ = np.linalg.lstsq(A, y, rcond=None)
        if sol[0] > 0 and sol[1] > 0:
            self.launch_s, self.s_per_update = float(sol[0]), float(sol[1])


@dataclass
class FoamServer:
    """Continuous batching in quanta of about `quantum_s` of GPU time (from a
    cost model fitted to the quanta so far). Each quantum's steps per box
    follow `policy`: "work" shares the cell updates equally (`fair_steps`;
    `quantum_updates` fixes the budget), "time" shares GPU time counting a
    launch cost per step (`fair_time_steps`), "lockstep" steps every box in
    every launch (`lockstep_steps`), "tiered" serves big jobs first come,
    first served beside equally shared small ones (`tiered_steps`), "fifo"
    and "srpt" fill each quantum in arrival or shortest-remaining-work order
    (`ordered_steps`; "srpt" credits each job `age_weight` times the time
    it has waited, so the largest jobs are not starved), "express" puts the
    jobs with less than `big_s` of work left first and keeps arrival order
    otherwise, "hrrn" fills it in order of the ratio of time since arrival to
    remaining work, and "tiered"
    cuts the small ones' share to `late_share` while the oldest big job's
    projected latency exceeds `big_slowdown` times its work alone. Every batch runs its plan as multi-rate
    steps (lbm_batch_step_each), so small boxes can take many cheap steps
    while large ones take few."""
    memory_budget_bytes: int
    max_boxes: int = 64
    quantum_s: float = 0.01
    quantum_updates: float | None = None
    policy: str = "work"            # "work" | "time" | "lockstep" | "tiered" | "fifo" | "express" | "srpt" | "hrrn"
    big_s: float = 0.05             # "tiered": a job with more work left than this much GPU time is big
    small_share: float = 0.5        # "tiered": most of a quantum the small jobs take while a big one runs
    big_slowdown: float = float("inf")  # "tiered": once the oldest big job's projected latency exceeds
                                        # this many times its work alone, the small jobs' share is
    late_share: float = 0.0             # cut to late_share (they still move a step per quantum)
    age_weight: float = 0.0         # "srpt": order by remaining GPU time minus this times the time waited
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
        model = _CostModel()               # quantum time vs launches and updates
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
            jobs_now = list(active.values())
            if self.policy == "work":
                budget = self.quantum_updates if self.quantum_updates else self.quantum_s / model.s_per_update
                share = fair_steps(jobs_now, budget)
            elif self.policy == "time":
                share = fair_time_steps(jobs_now, self.quantum_s, model.launch_s, model.s_per_update)
            elif self.policy == "lockstep":
                share = lockstep_steps(jobs_now, self.quantum_s, model.launch_s, model.s_per_update)
            elif self.policy in ("fifo", "express", "srpt", "hrrn"):
                budget = self.quantum_updates if self.quantum_updates else self.quantum_s / model.s_per_update
                key = order_key(self.policy, now, model.s_per_update, self.age_weight, self.big_s)
                share = ordered_steps(jobs_now, budget, key)
            elif self.policy == "tiered":
                budget = self.quantum_updates if self.quantum_updates else self.quantum_s / model.s_per_update
                big_updates = self.big_s / model.s_per_update
                small_share = self.small_share
                bigs = [j for j in jobs_now if j.remaining * j.cells >= big_updates]
                if bigs:
                    # projected latency of the oldest big job at the full rate
                    # from now on, against its work alone: past the bound it
                    # takes the whole quantum (small jobs still move a step)
                    j0 = min(bigs, key=lambda j: (j.req.arrival_s, j.req.rid))
                    alone = j0.req.steps * j0.cells * model.s_per_update
                    projected = (now - j0.req.arrival_s) + j0.remaining * j0.cells * model.s_per_update
                    if projected > self.big_slowdown * alone:
                        small_share = min(small_share, self.late_share)
                share = tiered_steps(jobs_now, budget, big_updates, small_share)
            else:
                raise ValueError(f"unknown policy {self.policy!r}")
            ts = time.perf_counter()
            live = []
            for b, jobs in batches.values():
                plan = [share.get(j.req.rid, 0) if j.remaining > 0 else 0 for j in jobs]
                movers = [i for i, n in enumerate(plan) if n > 0]
                if len(movers) == 1:
                    # a single box moves: its own step path, which a batch's per-step
                    # launches only slow down
                    b.step_one(movers[0], plan[movers[0]])
                    live.append((b, jobs, plan))
                elif movers:
                    b.step_each(plan)  # each batch on its own stream: the storage classes overlap
                    live.append((b, jobs, plan))
            for b, _, _ in live:
                b.sync()
            dt = time.perf_counter() - ts
            t_step += dt
            done = sum(share[r] * active[r].cells for r in share)
            model.add(max(share.values()), done, dt)
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
                      "policy": self.policy, "launch_us": round(model.launch_s * 1e6, 2),
                      "rate_mlups": round(1e-6 / model.s_per_update, 1)}
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


def _pct(vals: list[float], p: float) -> float:
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(round(p / 100.0 * (len(v) - 1)))))]


def summarize(results: list[Result], makespan_s: float) -> dict:
    """Latency percentiles (nearest rank), mean, throughput, and the median
    latency of the smallest, middle and largest third of the requests by
    work (cells x steps)."""
    lat = [r.latency_s for r in results]
    updates = sum(r.cells * r.steps for r in results)
    by_work = sorted(results, key=lambda r: r.cells * r.steps)
    k = len(by_work)
    thirds = [by_work[: k // 3], by_work[k // 3: 2 * k // 3], by_work[2 * k // 3:]]
    return {"requests": len(results), "p50_s": round(float(_pct(lat, 50)), 4), "p99_s": round(float(_pct(lat, 99)), 4),
            "mean_s": round(float(statistics.mean(lat)), 4), "makespan_s": round(makespan_s, 3),
            "mlups": round(updates / makespan_s / 1e6, 1), "cell_updates": updates,
            "p50_by_size_s": [round(float(_pct([r.latency_s for r in t], 50)), 4) if t else None for t in thirds]}
