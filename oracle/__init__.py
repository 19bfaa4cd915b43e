"""Python access to the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The CUDA library and its binding
never import it.

``OracleSim`` holds one periodic box: FP64 populations ``f[9, ny, nx]`` (the
incoming populations at the start of the next step) and the barrier state
(labels, owners, rupture signs, open flags, blocked-edge mask). The numpy
arrays are owned here and handed to the C functions by pointer.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Cited paper constants (arXiv 1708.01613, Sec. 2.1.2): critical point of
# p = rho/3 + G psi^2/6 with psi = 1 - exp(-rho).
G_CRITICAL = -4.0
RHO_CRITICAL = math.log(2.0)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                   "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("barrier", C.c_int32),
                ("relabel_every", C.c_int32), ("zone_radius", C.c_int32),
                ("stop_on_first_rupture", C.c_int32), ("tau", C.c_double),
                ("G", C.c_double), ("rho0", C.c_double), ("gas_threshold", C.c_double),
                ("rupture_eps", C.c_double), ("growth_rate", C.c_double),
                ("growth_budget", C.c_double)]


class _State(C.Structure):
    _fields_ = [("f", C.c_void_p), ("f_next", C.c_void_p), ("rho", C.c_void_p),
                ("jx", C.c_void_p), ("jy", C.c_void_p), ("psi", C.c_void_p),
                ("Fx", C.c_void_p), ("Fy", C.c_void_p), ("label", C.c_void_p),
                ("owner", C.c_void_p), ("sgn", C.c_void_p), ("open", C.c_void_p),
                ("mask", C.c_void_p), ("t", C.c_int64), ("opened_total", C.c_int64),
                ("opened_last", C.c_int32), ("halted", C.c_int32), ("gas", C.c_void_p),
                ("n_gas", C.c_int64), ("injected", C.c_double), ("merges_total", C.c_int64)]


class Params2(C.Structure):
    """Two-component (melt / gas lattices) parameters; see ``orc2_params``."""
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("barrier", C.c_int32),
                ("relabel_every", C.c_int32), ("zone_radius", C.c_int32), ("reserved", C.c_int32),
                ("tau_m", C.c_double), ("tau_g", C.c_double), ("G_mm", C.c_double),
                ("G_mg", C.c_double), ("G_gg", C.c_double), ("rho0", C.c_double),
                ("gas_threshold", C.c_double), ("rupture_eps", C.c_double)]


class _State2(C.Structure):
    _fields_ = [("fm", C.c_void_p), ("fg", C.c_void_p), ("fm_next", C.c_void_p), ("fg_next", C.c_void_p),
                ("rm", C.c_void_p), ("rg", C.c_void_p), ("psim", C.c_void_p), ("psig", C.c_void_p),
                ("pr", C.c_void_p), ("label", C.c_void_p), ("owner", C.c_void_p), ("sgn", C.c_void_p),
                ("open", C.c_void_p), ("mask", C.c_void_p), ("t", C.c_int64), ("opened_total", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER(Params)
        S = C.POINTER(_State)
        vp = C.c_void_p
        sig = {
            "orc_set_threads": (None, [C.c_int]),
            "orc_max_threads": (C.c_int, []),
            "orc_lattice": (None, [vp, vp, vp]),
            "orc_psi": (C.c_double, [C.c_double, C.c_double]),
            "orc_pressure": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_equilibrium": (None, [C.c_double, C.c_double, C.c_double, vp]),
            "orc_moments": (None, [P, vp, vp, vp, vp]),
            "orc_force": (None, [P, vp, vp, vp, vp]),
            "orc_label": (None, [P, vp, vp]),
            "orc_owner": (None, [P, vp, vp]),
            "orc_rupture": (None, [P, vp, vp, vp, vp, vp]),
            "orc_mask": (None, [P, vp, vp, vp]),
            "orc_relabel": (None, [P, S]),
            "orc_gas_census": (None, [P, S]),
            "orc_nucleate": (None, [P, S, vp, C.c_int32, C.c_double]),
            "orc_init_state": (None, [P, S, vp]),
            "orc_step": (C.c_int, [P, S]),
            "orc_run": (C.c_int64, [P, S, C.c_int64]),
            "orc_fields": (None, [P, S, vp, vp, vp, vp]),
            "orc_step_cells": (None, [P, vp, vp, vp, C.c_int64, vp]),
            "orc_init_bubbles": (None, [P, vp, C.c_int32, C.c_double, C.c_double,
                                        C.c_double, vp]),
            "orc_stats": (C.c_int32, [P, vp, vp, vp, vp, vp, vp, C.c_int32, C.c_double,
                                      C.c_double]),
            "orc_merges": (C.c_int32, [P, vp, vp]),
        }
        P2 = C.POINTER(Params2)
        S2 = C.POINTER(_State2)
        sig.update({
            "orc2_pressure": (C.c_double, [P2, C.c_double, C.c_double]),
            "orc2_init_state": (None, [P2, S2, vp, vp]),
            "orc2_relabel": (None, [P2, S2]),
            "orc2_step": (None, [P2, S2]),
            "orc2_run": (None, [P2, S2, C.c_int64]),
            "orc2_fields": (None, [P2, S2, vp, vp, vp, vp, vp]),
        })
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def make_params(nx, ny, *, tau=1.0, G=-5.5, rho0=1.0, barrier=False, relabel_every=1,
                zone_radius=4, stop_on_first_rupture=False, gas_threshold=None,
                rupture_eps=1e-6, growth_rate=0.0, growth_budget=0.0) -> Params:
    if gas_threshold is None:
        gas_threshold = RHO_CRITICAL
    return Params(nx=nx, ny=ny, barrier=int(bool(barrier)), relabel_every=relabel_every,
                  zone_radius=zone_radius, stop_on_first_rupture=int(bool(stop_on_first_rupture)),
                  tau=tau, G=G, rho0=rho0, gas_threshold=gas_threshold, rupture_eps=rupture_eps,
                  growth_rate=growth_rate, growth_budget=growth_budget)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def lattice():
    ex = np.zeros(9, np.int32)
    ey = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    lib().orc_lattice(_p(ex), _p(ey), _p(w))
    return ex, ey, w


def psi(rho: float, rho0: float = 1.0) -> float:
    return lib().orc_psi(float(rho), float(rho0))


def pressure(rho: float, G: float = -5.5, rho0: float = 1.0) -> float:
    return lib().orc_pressure(float(rho), float(G), float(rho0))


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9, np.float64)
    lib().orc_equilibrium(float(rho), float(ux), float(uy), _p(out))
    return out


def force(params: Params, psi_field: np.ndarray, mask: np.ndarray | None = None):
    psi_field = np.ascontiguousarray(psi_field, dtype=np.float64)
    Fx = np.zeros_like(psi_field)
    Fy = np.zeros_like(psi_field)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    lib().orc_force(C.byref(params), _p(psi_field), _p(m), _p(Fx), _p(Fy))
    return Fx, Fy


def label(params: Params, rho: np.ndarray) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty(rho.shape, np.int32)
    lib().orc_label(C.byref(params), _p(rho), _p(out))
    return out


def owner(params: Params, labels: np.ndarray) -> np.ndarray:
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    out = np.empty(labels.shape, np.int32)
    lib().orc_owner(C.byref(params), _p(labels), _p(out))
    return out


def rupture(params: Params, rho, owners, sgn, open_):
    """In-place update of ``sgn`` and ``open_``; returns the count newly opened."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    owners = np.ascontiguousarray(owners, dtype=np.int32)
    n = C.c_int32(0)
    lib().orc_rupture(C.byref(params), _p(rho), _p(owners), _p(sgn), _p(open_), C.byref(n))
    return int(n.value)


def mask(params: Params, owners, open_) -> np.ndarray:
    owners = np.ascontiguousarray(owners, dtype=np.int32)
    open_ = np.ascontiguousarray(open_, dtype=np.uint8)
    out = np.empty(owners.shape, np.uint8)
    lib().orc_mask(C.byref(params), _p(owners), _p(open_), _p(out))
    return out


def init_bubbles(params: Params, bubbles, rho_l: float, rho_g: float, width: float = 4.0):
    b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(-1, 3))
    out = np.empty((params.ny, params.nx), np.float64)
    lib().orc_init_bubbles(C.byref(params), _p(b), int(b.shape[0]), float(rho_l), float(rho_g),
                           float(width), _p(out))
    return out


def merges(params: Params, before: np.ndarray, now: np.ndarray) -> int:
    """Components of the labelling `now` holding gas of two or more
    components of `before` (coalescence events)."""
    before = np.ascontiguousarray(before, dtype=np.int32)
    now = np.ascontiguousarray(now, dtype=np.int32)
    return int(lib().orc_merges(C.byref(params), _p(before), _p(now)))


def step_cells(params: Params, f: np.ndarray, cells, mask_arr: np.ndarray | None = None):
    """Next-step incoming populations at ``cells`` (flat indices) -> (len, 9)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty((cells.shape[0], 9), np.float64)
    m = None if mask_arr is None else np.ascontiguousarray(mask_arr, dtype=np.uint8)
    lib().orc_step_cells(C.byref(params), _p(f), _p(m), _p(cells), int(cells.shape[0]), _p(out))
    return out


def stats(params: Params, labels: np.ndarray, nbins: int = 16, dmin: float = 1.0,
          dmax: float = 256.0) -> dict:
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    N = labels.size
    gf = C.c_double(0.0)
    md = C.c_double(0.0)
    areas = np.zeros(N, np.float64)
    diam = np.zeros(N, np.float64)
    hist = np.zeros(max(nbins, 1), np.float64)
    n = lib().orc_stats(C.byref(params), _p(labels), C.byref(gf), C.byref(md), _p(areas),
                        _p(diam), _p(hist), int(nbins), float(dmin), float(dmax))
    return {"n_bubbles": int(n), "gas_fraction": gf.value, "mean_diameter": md.value,
            "areas": areas[:n].copy(), "diameters": diam[:n].copy(), "hist": hist[:nbins].copy()}


class OracleSim:
    """One periodic box advanced by the FP64 oracle."""

    def __init__(self, params: Params):
        self.params = params
        nx, ny = params.nx, params.ny
        self.f = np.zeros((9, ny, nx), np.float64)
        self.f_next = np.zeros_like(self.f)
        self.rho = np.zeros((ny, nx), np.float64)
        self.jx = np.zeros_like(self.rho)
        self.jy = np.zeros_like(self.rho)
        self.psi = np.zeros_like(self.rho)
        self.Fx = np.zeros_like(self.rho)
        self.Fy = np.zeros_like(self.rho)
        self.label = np.full((ny, nx), -1, np.int32)
        self.owner = np.full((ny, nx), -1, np.int32)
        self.sgn = np.zeros((ny, nx), np.int8)
        self.open = np.zeros((ny, nx), np.uint8)
        self.mask = np.zeros((ny, nx), np.uint8)
        self.gas = np.zeros((ny, nx), np.uint8)
        self._s = _State(f=_p(self.f), f_next=_p(self.f_next), rho=_p(self.rho), jx=_p(self.jx),
                         jy=_p(self.jy), psi=_p(self.psi), Fx=_p(self.Fx), Fy=_p(self.Fy),
                         label=_p(self.label), owner=_p(self.owner), sgn=_p(self.sgn),
                         open=_p(self.open), mask=_p(self.mask), t=0, opened_total=0,
                         opened_last=0, halted=0, gas=_p(self.gas), n_gas=0, injected=0.0,
                         merges_total=0)

    def init_density(self, rho: np.ndarray) -> None:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (self.params.ny, self.params.nx)
        lib().orc_init_state(C.byref(self.params), C.byref(self._s), _p(rho))

    def load_populations(self, f: np.ndarray) -> None:
        self.f[...] = f

    def relabel(self) -> None:
        lib().orc_relabel(C.byref(self.params), C.byref(self._s))

    def nucleate(self, nuclei, rho_g: float) -> None:
        """Cells within r of a nucleus (cx, cy, r) become gas at rest (rho_g)."""
        b = np.ascontiguousarray(np.asarray(nuclei, dtype=np.float64).reshape(-1, 3))
        lib().orc_nucleate(C.byref(self.params), C.byref(self._s), _p(b), int(b.shape[0]), float(rho_g))

    @property
    def injected(self) -> float:
        return float(self._s.injected)

    @property
    def n_gas(self) -> int:
        return int(self._s.n_gas)

    def step(self, n: int = 1) -> int:
        return int(lib().orc_run(C.byref(self.params), C.byref(self._s), int(n)))

    @property
    def t(self) -> int:
        return int(self._s.t)

    @property
    def halted(self) -> bool:
        return bool(self._s.halted)

    @property
    def opened_total(self) -> int:
        return int(self._s.opened_total)

    @property
    def opened_last(self) -> int:
        return int(self._s.opened_last)

    @property
    def merges_total(self) -> int:
        """Coalescence events counted by the relabels so far."""
        return int(self._s.merges_total)

    def fields(self):
        ny, nx = self.params.ny, self.params.nx
        rho = np.empty((ny, nx))
        ux = np.empty((ny, nx))
        uy = np.empty((ny, nx))
        pr = np.empty((ny, nx))
        lib().orc_fields(C.byref(self.params), C.byref(self._s), _p(rho), _p(ux), _p(uy), _p(pr))
        return {"rho": rho, "ux": ux, "uy": uy, "p": pr}

    def mass(self) -> float:
        return float(np.sum(self.f))

    def momentum(self):
        """Sum over the box of j + F/2 (the physical momentum)."""
        fl = self.fields()
        return (float(np.sum(fl["rho"] * fl["ux"])), float(np.sum(fl["rho"] * fl["uy"])))

    def labels_now(self) -> np.ndarray:
        """Labels of the current density (the same threshold as the barrier)."""
        lib().orc_moments(C.byref(self.params), _p(self.f), _p(self.rho), None, None)
        return label(self.params, self.rho)


def make_params2(nx, ny, *, tau_m=1.0, tau_g=1.0, G_mm=-5.5, G_mg=0.0, G_gg=0.0, rho0=1.0, barrier=False,
                 relabel_every=1, zone_radius=4, gas_threshold=None, rupture_eps=1e-6) -> Params2:
    if gas_threshold is None:
        gas_threshold = RHO_CRITICAL
    return Params2(nx=nx, ny=ny, barrier=int(bool(barrier)), relabel_every=relabel_every,
                   zone_radius=zone_radius, reserved=0, tau_m=tau_m, tau_g=tau_g, G_mm=G_mm, G_mg=G_mg,
                   G_gg=G_gg, rho0=rho0, gas_threshold=gas_threshold, rupture_eps=rupture_eps)


class OracleSim2:
    """Two-component box (melt and gas lattices) advanced by the FP64 oracle."""

    def __init__(self, params: Params2):
        self.params = params
        nx, ny = params.nx, params.ny
        self.fm = np.zeros((9, ny, nx), np.float64)
        self.fg = np.zeros_like(self.fm)
        self.fm_next = np.zeros_like(self.fm)
        self.fg_next = np.zeros_like(self.fm)
        self.rm = np.zeros((ny, nx), np.float64)
        self.rg = np.zeros_like(self.rm)
        self.psim = np.zeros_like(self.rm)
        self.psig = np.zeros_like(self.rm)
        self.pr = np.zeros_like(self.rm)
        self.label = np.full((ny, nx), -1, np.int32)
        self.owner = np.full((ny, nx), -1, np.int32)
        self.sgn = np.zeros((ny, nx), np.int8)
        self.open = np.zeros((ny, nx), np.uint8)
        self.mask = np.zeros((ny, nx), np.uint8)
        self._s = _State2(fm=_p(self.fm), fg=_p(self.fg), fm_next=_p(self.fm_next), fg_next=_p(self.fg_next),
                          rm=_p(self.rm), rg=_p(self.rg), psim=_p(self.psim), psig=_p(self.psig), pr=_p(self.pr),
                          label=_p(self.label), owner=_p(self.owner), sgn=_p(self.sgn), open=_p(self.open),
                          mask=_p(self.mask), t=0, opened_total=0)

    def init_density(self, rho_m: np.ndarray, rho_g: np.ndarray) -> None:
        rho_m = np.ascontiguousarray(rho_m, dtype=np.float64)
        rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
        assert rho_m.shape == rho_g.shape == (self.params.ny, self.params.nx)
        lib().orc2_init_state(C.byref(self.params), C.byref(self._s), _p(rho_m), _p(rho_g))

    def step(self, n: int = 1) -> None:
        lib().orc2_run(C.byref(self.params), C.byref(self._s), int(n))

    @property
    def t(self) -> int:
        return int(self._s.t)

    @property
    def opened_total(self) -> int:
        return int(self._s.opened_total)

    def fields(self) -> dict:
        ny, nx = self.params.ny, self.params.nx
        out = {k: np.empty((ny, nx)) for k in ("rho_m", "rho_g", "ux", "uy", "p")}
        lib().orc2_fields(C.byref(self.params), C.byref(self._s), _p(out["rho_m"]), _p(out["rho_g"]),
                          _p(out["ux"]), _p(out["uy"]), _p(out["p"]))
        return out

    def masses(self):
        return float(np.sum(self.fm)), float(np.sum(self.fg))

    def momentum(self):
        fl = self.fields()
        r = fl["rho_m"] + fl["rho_g"]
        return float(np.sum(r * fl["ux"])), float(np.sum(r * fl["uy"]))


def pressure2(params: Params2, rho_m: float, rho_g: float) -> float:
    return lib().orc2_pressure(C.byref(params), float(rho_m), float(rho_g))
