"""Counter-based seeded generators for the synthetic foam workloads.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``k`` of stream ``seed`` is ``mix(seed + (k + 1) * gamma)``
with the published finaliser ``mix``, turned into a double in [0, 1) from its
top 53 bits. The same (seed, k) always gives the same number, on any machine.

Workload recipes (lattice units, periodic boxes):

* spinodal noise: ``rho = rho_mean * (1 + amp * U[-1, 1))`` per cell, drawn in
  row-major cell order (draw k = y * nx + x);
* Poisson-disk bubbles: dart throwing on the torus, radius uniform or
  log-uniform, an edge gap of at least ``gap_min`` to every placed bubble;
* clustered bubbles: each new bubble touches a random placed bubble at an
  edge gap drawn from U[gap_lo, gap_hi] in a random direction, and is
  rejected if its gap to any other bubble is below ``gap_lo``;
* batched instances and serving requests: sides, bubble counts and step
  counts drawn log-uniformly (sides rounded to the nearest integer).

The liquid and gas densities used to initialise bubbles are plain numbers
here (``RHO_LIQ_G55``, ``RHO_GAS_G55``); the tests check them against the
equal-area construction computed by the oracle and against the oracle's own
flat-interface run.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

# Coexisting densities for psi = 1 - exp(-rho), G = -5.5, tau = 1 (D2Q9,
# velocity-shift forcing), as reached by a flat liquid slab run to rest.
RHO_GAS_G55 = 0.104158
RHO_LIQ_G55 = 2.306865


def splitmix64_uniform(seed: int, k) -> np.ndarray:
    """Uniform doubles in [0, 1) for draws ``k`` (int or int array) of ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (k + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class _Stream:
    """Sequential draws from one SplitMix64 counter stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.k = 0

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = float(splitmix64_uniform(self.seed, self.k))
        self.k += 1
        return lo + (hi - lo) * u

    def log_uniform(self, lo: float, hi: float) -> float:
        return math.exp(self.uniform(math.log(lo), math.log(hi)))


def noise_density(nx: int, ny: int, seed: int, rho_mean: float = 0.7,
                  amp: float = 0.01) -> np.ndarray:
    """Row-major (ny, nx) FP64 density ``rho_mean * (1 + amp * U[-1, 1))``."""
    k = np.arange(nx * ny, dtype=np.uint64)
    u = splitmix64_uniform(seed, k)
    return (rho_mean * (1.0 + amp * (2.0 * u - 1.0))).reshape(ny, nx)


def _torus_gap(b, c, nx, ny):
    dx = abs(b[0] - c[0])
    dy = abs(b[1] - c[1])
    dx = min(dx, nx - dx)
    dy = min(dy, ny - dy)
    return math.hypot(dx, dy) - b[2] - c[2]


def poisson_disk_bubbles(nx: int, ny: int, n: int, rmin: float, rmax: float,
                         gap_min: float, seed: int, log_uniform: bool = True,
                         max_tries: int = 200000) -> np.ndarray:
    """(n, 3) array of (cx, cy, r): dart throwing on the nx-by-ny torus."""
    s = _Stream(seed)
    out: list[tuple[float, float, float]] = []
    tries = 0
    while len(out) < n:
        if tries >= max_tries:
            raise RuntimeError(f"placed only {len(out)} of {n} bubbles")
        tries += 1
        cx = s.uniform(0.0, nx)
        cy = s.uniform(0.0, ny)
        r = s.log_uniform(rmin, rmax) if log_uniform else s.uniform(rmin, rmax)
        b = (cx, cy, r)
        if 2.0 * r + gap_min > min(nx, ny):
            continue
        if all(_torus_gap(b, c, nx, ny) >= gap_min for c in out):
            out.append(b)
    return np.asarray(out, dtype=np.float64).reshape(-1, 3)


def clustered_bubbles(nx: int, ny: int, n: int, rmin: float, rmax: float,
                      gap_lo: float, gap_hi: float, seed: int,
                      max_tries: int = 200000) -> np.ndarray:
    """(n, 3) array of (cx, cy, r), each bubble touching an earlier one at a gap in [gap_lo, gap_hi]."""
    s = _Stream(seed)
    r0 = s.uniform(rmin, rmax)
    out = [(s.uniform(0.0, nx), s.uniform(0.0, ny), r0)]
    tries = 0
    while len(out) < n:
        if tries >= max_tries:
            raise RuntimeError(f"placed only {len(out)} of {n} bubbles")
        tries += 1
        j = min(int(s.uniform() * len(out)), len(out) - 1)
        theta = s.uniform(0.0, 2.0 * math.pi)
        gap = s.uniform(gap_lo, gap_hi)
        r = s.uniform(rmin, rmax)
        pj = out[j]
        dist = pj[2] + r + gap
        cx = (pj[0] + dist * math.cos(theta)) % nx
        cy = (pj[1] + dist * math.sin(theta)) % ny
        b = (cx, cy, r)
        if all(_torus_gap(b, c, nx, ny) >= gap_lo - 1e-9 for c in out):
            out.append(b)
    return np.asarray(out, dtype=np.float64).reshape(-1, 3)


def log_uniform_sides(count: int, lo: int, hi: int, seed: int, multiple: int = 1) -> list[int]:
    """``count`` box sides drawn log-uniformly in [lo, hi], rounded to ``multiple``
    (1: any integer side)."""
    s = _Stream(seed)
    out = []
    for _ in range(count):
        v = s.log_uniform(lo, hi)
        out.append(int(min(hi, max(lo, multiple * round(v / multiple)))))
    return out


def batch_instances(count: int = 64, side_lo: int = 256, side_hi: int = 2048,
                    bub_lo: int = 5, bub_hi: int = 200, steps_lo: int = 1000,
                    steps_hi: int = 20000, seed: int = 31) -> list[dict]:
    """Mixed-size independent foam instances (square boxes)."""
    s = _Stream(seed)
    out = []
    for i in range(count):
        side = int(min(side_hi, max(side_lo, round(s.log_uniform(side_lo, side_hi)))))
        nb = int(round(s.log_uniform(bub_lo, bub_hi)))
        steps = int(round(s.log_uniform(steps_lo, steps_hi)))
        # keep the bubble area below ~35 % of the box
        rmax = max(6.0, min(48.0, 0.33 * side / math.sqrt(max(nb, 1)) ))
        rmin = min(6.0, rmax)
        bubbles = poisson_disk_bubbles(side, side, nb, rmin, rmax, 2.0,
                                       seed * 1000003 + i, log_uniform=True)
        out.append({"nx": side, "ny": side, "bubbles": bubbles, "steps": steps,
                    "seed": seed * 1000003 + i})
    return out


def nucleation_schedule(nx: int, ny: int, count: int, t_max: int, r_lo: float = 3.0, r_hi: float = 8.0,
                        seed: int = 61) -> np.ndarray:
    """Random nucleation events (the paper's "time random subroutine"): rows
    (step, cx, cy, r), steps uniform in [0, t_max), sites uniform over the
    box, radii log-uniform in [r_lo, r_hi], sorted by step (stable)."""
    s = _Stream(seed)
    rows = []
    for _ in range(count):
        t = min(t_max - 1, int(s.uniform() * t_max))
        rows.append((float(t), s.uniform() * nx, s.uniform() * ny, s.log_uniform(r_lo, r_hi)))
    rows.sort(key=lambda r: r[0])
    return np.array(rows, dtype=np.float64).reshape(-1, 4)


def serving_requests(count: int = 2000, rate_per_s: float = 10.0, side_lo: int = 128,
                     side_hi: int = 4096, bub_lo: int = 2, bub_hi: int = 300,
                     steps_lo: int = 1000, steps_hi: int = 20000, seed: int = 41,
                     fp16_fraction: float = 0.5) -> list[dict]:
    """Poisson arrival stream of foam-simulation requests.

    Bubble lists are not drawn here (they are cheap to draw at admission
    time from the request's ``seed``); each request carries its own seed.
    """
    s = _Stream(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - s.uniform()) / rate_per_s
        side = int(min(side_hi, max(side_lo, round(s.log_uniform(side_lo, side_hi)))))
        nb = int(round(s.log_uniform(bub_lo, bub_hi)))
        steps = int(round(s.log_uniform(steps_lo, steps_hi)))
        fp16 = s.uniform() < fp16_fraction
        out.append({"id": i, "arrival_s": t, "nx": side, "ny": side, "n_bubbles": nb,
                    "steps": steps, "storage": "f16" if fp16 else "f32",
                    "seed": seed * 1000003 + i})
    return out


def request_bubbles(req: dict) -> np.ndarray:
    """Bubble list of one serving request (Poisson-disk, log-uniform radii).

    The requested count is capped so that bubbles of radius 5 cover at most
    a fifth of the box (radii start at 4); dart throwing then always
    succeeds."""
    side = req["nx"]
    cap = max(1, int(0.2 * req["nx"] * req["ny"] / (math.pi * 5.0**2)))
    nb = min(req["n_bubbles"], cap)
    rmax = max(4.0, min(48.0, 0.33 * side / math.sqrt(max(nb, 1))))
    rmin = min(4.0, rmax)
    return poisson_disk_bubbles(req["nx"], req["ny"], nb, rmin, rmax, 2.0, req["seed"])
