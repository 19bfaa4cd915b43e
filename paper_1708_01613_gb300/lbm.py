"""Thin ctypes binding of liblbm (include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA
library. PyTorch supplies the device workspace (one uint8 tensor) and the
CUDA stream. There is no CPU fallback: if the library cannot be loaded or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENUMERIC, LBM_ETIMEOUT, LBM_ENOTSUP = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ENUMERIC",
                5: "LBM_ETIMEOUT", 6: "LBM_ENOTSUP"}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}

FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_P = 1 << 0, 1 << 1, 1 << 2, 1 << 3
FIELD_LABEL, FIELD_OWNER, FIELD_MASK, FIELD_OPEN, FIELD_POPS = 1 << 4, 1 << 5, 1 << 6, 1 << 7, 1 << 8
FIELD_RHO_GAS = 1 << 9
FIELDS = {"rho": (FIELD_RHO, np.float32), "ux": (FIELD_UX, np.float32), "uy": (FIELD_UY, np.float32),
          "p": (FIELD_P, np.float32), "label": (FIELD_LABEL, np.int32),
          "owner": (FIELD_OWNER, np.int32), "mask": (FIELD_MASK, np.uint8),
          "open": (FIELD_OPEN, np.uint8), "pops": (FIELD_POPS, np.float32),
          "rho_gas": (FIELD_RHO_GAS, np.float32)}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class lbm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("storage", C.c_int32),
                ("barrier", C.c_int32), ("relabel_every", C.c_int32), ("zone_radius", C.c_int32),
                ("stop_on_first_rupture", C.c_int32), ("growth", C.c_int32),
                ("tau", C.c_double), ("G", C.c_double), ("rho0", C.c_double),
                ("rho_ref", C.c_double), ("gas_threshold", C.c_double),
                ("rupture_eps", C.c_double), ("components", C.c_int32), ("reserved2", C.c_int32),
                ("tau_g", C.c_double), ("G_mg", C.c_double), ("G_gg", C.c_double)]


class lbm_bubble(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double)]


class lbm_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_bubbles", C.c_int32), ("reserved", C.c_int32),
                ("n_open", C.c_int64), ("gas_fraction", C.c_double),
                ("mean_eq_diameter", C.c_double), ("mass", C.c_double), ("n_merges", C.c_int64)]


# Every entry point of include/lbm.h with its ctypes signature.
_vp = C.c_void_p
SIGNATURES = {
    "lbm_config_default": (None, [C.POINTER(lbm_config)]),
    "lbm_workspace_bytes": (C.c_size_t, [C.POINTER(lbm_config)]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_config), _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "lbm_init_density": (C.c_int, [_vp, _vp, C.c_int]),
    "lbm_init_bubbles": (C.c_int, [_vp, _vp, C.c_int32, C.c_double, C.c_double, C.c_double]),
    "lbm_load_populations": (C.c_int, [_vp, _vp, C.c_int]),
    "lbm_step": (C.c_int, [_vp, C.c_int64]),
    "lbm_steps_done": (C.c_int64, [_vp]),
    "lbm_kernel_launches": (C.c_int64, [_vp]),
    "lbm_set_step_variant": (C.c_int, [_vp, C.c_int]),
    "lbm_halted": (C.c_int, [_vp]),
    "lbm_fields_bytes": (C.c_size_t, [_vp, C.c_uint32]),
    "lbm_read_fields": (C.c_int, [_vp, C.c_uint32, _vp, C.c_size_t, C.c_int]),
    "lbm_mass": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "lbm_nucleate": (C.c_int, [_vp, _vp, C.c_int32, C.c_double]),
    "lbm_set_growth": (C.c_int, [_vp, C.c_double, C.c_double]),
    "lbm_growth_released": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "lbm_bubble_stats": (C.c_int, [_vp, C.POINTER(lbm_stats), _vp, C.c_int32, C.c_double,
                                   C.c_double]),
    "lbm_bubble_areas": (C.c_int, [_vp, C.c_int32, _vp, _vp, C.POINTER(C.c_int32)]),
    "lbm_sync": (C.c_int, [_vp]),
    "lbm_last_error": (C.c_char_p, [_vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_mass_noalloc": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, _vp, _vp,
                                   C.c_char_p, C.c_size_t]),
    "lbm_batch_workspace_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "lbm_batch_create": (C.c_int, [_vp, C.c_int32, _vp, C.c_size_t, C.POINTER(_vp)]),
    "lbm_batch_set_tiles": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "lbm_batch_get_tiles": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_batch_tune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_float)]),
    "lbm_batch_use_graph": (C.c_int, [_vp, C.c_int]),
    "lbm_batch_set_active": (C.c_int, [_vp, C.c_int32, C.c_int]),
    "lbm_batch_step": (C.c_int, [_vp, C.c_int64]),
    "lbm_batch_step_each": (C.c_int, [_vp, _vp, C.c_int32]),
    "lbm_batch_step_one": (C.c_int, [_vp, C.c_int32, C.c_int64]),
    "lbm_batch_sync": (C.c_int, [_vp]),
    "lbm_batch_steps_done": (C.c_int64, [_vp]),
    "lbm_batch_kernel_launches": (C.c_int64, [_vp]),
    "lbm_batch_last_error": (C.c_char_p, [_vp]),
    "lbm_batch_destroy": (None, [_vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_needed: bool = True) -> C.CDLL:
    """Load liblbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise OSError(f"liblbm.so not found at {_build.LIB}; run build()")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(code: int, handle=None) -> None:
    if code != LBM_OK:
        msg = ""
        if handle is not None:
            m = load_library().lbm_last_error(handle)
            msg = m.decode() if m else ""
        raise LbmError(code, msg)


def lbm_config_default() -> lbm_config:
    c = lbm_config()
    load_library().lbm_config_default(C.byref(c))
    return c


def make_config(nx: int, ny: int, *, storage: str = "f32", barrier: bool = False, relabel_every: int = 1,
                zone_radius: int = 4, stop_on_first_rupture: bool = False, tau: float = 1.0,
                G: float = -5.5, rho0: float = 1.0, rho_ref: float = 1.0,
                gas_threshold: float = math.log(2.0), rupture_eps: float = 1e-6,
                growth: bool = False, components: int = 1, tau_g: float = 1.0, G_mg: float = 0.0,
                G_gg: float = 0.0) -> lbm_config:
    c = lbm_config_default()
    c.nx, c.ny = int(nx), int(ny)
    c.storage = STORAGE[storage]
    c.barrier = int(bool(barrier))
    c.relabel_every = int(relabel_every)
    c.zone_radius = int(zone_radius)
    c.stop_on_first_rupture = int(bool(stop_on_first_rupture))
    c.tau, c.G, c.rho0, c.rho_ref = float(tau), float(G), float(rho0), float(rho_ref)
    c.gas_threshold, c.rupture_eps = float(gas_threshold), float(rupture_eps)
    c.growth = int(bool(growth))
    c.components = int(components)
    c.tau_g, c.G_mg, c.G_gg = float(tau_g), float(G_mg), float(G_gg)
    return c


def lbm_workspace_bytes(cfg: lbm_config) -> int:
    return int(load_library().lbm_workspace_bytes(C.byref(cfg)))


class Simulation:
    """One periodic box on one GPU, driven through the C ABI.

    The workspace is a torch uint8 tensor owned by this object; the stream is
    torch's current stream on ``device`` unless one is given.
    """

    def __init__(self, cfg: lbm_config, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; no CPU fallback exists")
        lib = load_library()
        self.cfg = cfg
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = lbm_workspace_bytes(cfg)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid configuration")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            base = self.workspace.data_ptr()
            self._ws_ptr = (base + 255) // 256 * 256
            h = C.c_void_p()
            _check(lib.lbm_create(C.byref(cfg), C.c_void_p(self._ws_ptr), nbytes,
                                  C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.handle = h
        self.nx, self.ny = cfg.nx, cfg.ny

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "handle", None):
            load_library().lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def _call(self, name, *args):
        import torch

        with torch.cuda.device(self.device):
            _check(getattr(load_library(), name)(self.handle, *args), self.handle)

    @property
    def components(self) -> int:
        return 2 if self.cfg.components == 2 else 1

    def init_density(self, rho, rho_gas=None) -> None:
        """Rest equilibrium at the FP64 densities; with two components the
        gas density `rho_gas` is required too (melt first)."""
        import torch

        if self.components == 2:
            if rho_gas is None:
                raise LbmError(LBM_EINVAL, "two components need rho and rho_gas")
            rho = np.concatenate([np.asarray(rho, np.float64).ravel(), np.asarray(rho_gas, np.float64).ravel()])
        elif rho_gas is not None:
            raise LbmError(LBM_EINVAL, "rho_gas is for two-component boxes")
        n = self.nx * self.ny * self.components
        if isinstance(rho, torch.Tensor) and rho.is_cuda:
            t = rho.to(torch.float64).contiguous()
            assert t.numel() == n
            self._call("lbm_init_density", C.c_void_p(t.data_ptr()), 1)
            self.stream.synchronize()
        else:
            a = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
            assert a.size == n
            self._call("lbm_init_density", C.c_void_p(a.ctypes.data), 0)
            self.stream.synchronize()

    def init_bubbles(self, bubbles, rho_l: float, rho_g: float, width: float = 4.0) -> None:
        b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(-1, 3))
        self._call("lbm_init_bubbles", C.c_void_p(b.ctypes.data) if len(b) else None, int(len(b)),
                   float(rho_l), float(rho_g), float(width))

    def load_populations(self, f) -> None:
        import torch

        if isinstance(f, torch.Tensor) and f.is_cuda:
            t = f.to(torch.float32).contiguous()
            assert t.numel() == 9 * self.components * self.nx * self.ny
            self._call("lbm_load_populations", C.c_void_p(t.data_ptr()), 1)
        else:
            a = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
            assert a.size == 9 * self.components * self.nx * self.ny
            self._call("lbm_load_populations", C.c_void_p(a.ctypes.data), 0)

    def set_step_variant(self, variant: int) -> None:
        """0 automatic, 1 plain loads, 2 one-cell staged, 3 two-cell staged,
        4 two-cell staged with dynamically drawn row chunks (3 and 4 need nx % 16 == 0)."""
        self._call("lbm_set_step_variant", int(variant))

    def step(self, n: int = 1) -> None:
        self._call("lbm_step", C.c_int64(int(n)))

    @property
    def steps_done(self) -> int:
        return int(load_library().lbm_steps_done(self.handle))

    @property
    def kernel_launches(self) -> int:
        return int(load_library().lbm_kernel_launches(self.handle))

    @property
    def halted(self) -> bool:
        return bool(load_library().lbm_halted(self.handle))

    def read(self, *names: str, device: bool = False) -> dict:
        """Fields by name (rho, ux, uy, p, label, owner, mask, open, pops, rho_gas).

        Host numpy arrays by default; with ``device=True`` torch CUDA tensors
        written directly by the library."""
        import torch

        out = {}
        lib = load_library()
        for name in names:
            bit, dt = FIELDS[name]
            nb = int(lib.lbm_fields_bytes(self.handle, bit))
            shape = (9 * self.components, self.ny, self.nx) if name == "pops" else (self.ny, self.nx)
            if device:
                t = torch.empty(shape, dtype=getattr(torch, np.dtype(dt).name), device=self.device)
                self._call("lbm_read_fields", C.c_uint32(bit), C.c_void_p(t.data_ptr()), nb, 1)
                out[name] = t
            else:
                a = np.empty(shape, dtype=dt)
                self._call("lbm_read_fields", C.c_uint32(bit), C.c_void_p(a.ctypes.data), nb, 0)
                out[name] = a
        return out

    def mass(self) -> float:
        v = C.c_double(0.0)
        self._call("lbm_mass", C.byref(v))
        return float(v.value)

    def nucleate(self, nuclei, rho_g: float) -> None:
        """Cells within r of a nucleus (cx, cy, r) become gas at rest (rho_g)."""
        b = np.ascontiguousarray(np.asarray(nuclei, dtype=np.float64).reshape(-1, 3))
        self._call("lbm_nucleate", C.c_void_p(b.ctypes.data) if len(b) else None, int(len(b)), float(rho_g))

    def set_growth(self, rate: float, budget: float) -> None:
        """Release `rate` of gas mass per step until `budget` is released."""
        self._call("lbm_set_growth", float(rate), float(budget))

    @property
    def growth_released(self) -> float:
        v = C.c_double(0.0)
        self._call("lbm_growth_released", C.byref(v))
        return float(v.value)

    def stats(self, nbins: int = 0, dmin: float = 1.0, dmax: float = 256.0) -> dict:
        st = lbm_stats()
        hist = np.zeros(max(nbins, 1), np.float64)
        self._call("lbm_bubble_stats", C.byref(st), C.c_void_p(hist.ctypes.data) if nbins else None,
                   int(nbins), float(dmin), float(dmax))
        return {"step": st.step, "n_bubbles": st.n_bubbles, "n_open": st.n_open,
                "gas_fraction": st.gas_fraction, "mean_diameter": st.mean_eq_diameter,
                "mass": st.mass, "n_merges": st.n_merges, "hist": hist[:nbins].copy()}

    def bubble_areas(self):
        """(labels, areas) of the bubbles of the current density, in
        increasing label order (labels int32, areas float64 cell counts)."""
        n = C.c_int32(0)
        lib = load_library()
        import torch

        with torch.cuda.device(self.device):
            rc = lib.lbm_bubble_areas(self.handle, 0, None, None, C.byref(n))
        if rc not in (LBM_OK, LBM_EINVAL):
            _check(rc, self.handle)
        labels = np.zeros(max(n.value, 1), np.int32)
        areas = np.zeros(max(n.value, 1), np.float64)
        self._call("lbm_bubble_areas", int(len(labels)), C.c_void_p(labels.ctypes.data),
                   C.c_void_p(areas.ctypes.data), C.byref(n))
        return labels[:n.value].copy(), areas[:n.value].copy()

    def sync(self) -> None:
        self._call("lbm_sync")


class Batch:
    """Several Simulation boxes advanced together (lbm_batch_*).

    Every step is one persistent launch over all active boxes; blocks of a
    relabel period are replayed as CUDA graphs. Boxes evolve bitwise as they
    would alone. The workspace is a torch uint8 tensor owned by this object.
    """

    def __init__(self, sims):
        import torch

        self.sims = list(sims)
        lib = load_library()
        arr = (C.c_void_p * len(self.sims))(*[s.handle.value for s in self.sims])
        self._arr = arr
        nbytes = int(lib.lbm_batch_workspace_bytes(arr, len(self.sims)))
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid batch")
        dev = self.sims[0].device
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.lbm_batch_create(arr, len(self.sims), C.c_void_p(ptr), nbytes, C.byref(h)))
        self.handle = h
        self.device = dev

    def _call(self, name, *args):
        import torch

        lib = load_library()
        with torch.cuda.device(self.device):
            code = getattr(lib, name)(self.handle, *args)
        if code != LBM_OK:
            m = lib.lbm_batch_last_error(self.handle)
            raise LbmError(code, m.decode() if m else "")

    @property
    def period(self) -> int:
        """Steps covered by one captured graph: the relabel period with the
        barrier on, else 16."""
        c = self.sims[0].cfg
        return int(c.relabel_every) if c.barrier else 16

    def set_tiles(self, strip_width: int, chunk_rows: int) -> None:
        self._call("lbm_batch_set_tiles", int(strip_width), int(chunk_rows))

    @property
    def tiles(self):
        a, b = C.c_int32(), C.c_int32()
        load_library().lbm_batch_get_tiles(self.handle, C.byref(a), C.byref(b))
        return int(a.value), int(b.value)

    def tune(self, trial_steps: int = 3) -> float:
        ms = C.c_float(0.0)
        self._call("lbm_batch_tune", int(trial_steps), C.byref(ms))
        return float(ms.value)

    def use_graph(self, enable: bool) -> None:
        self._call("lbm_batch_use_graph", int(bool(enable)))

    def set_active(self, index: int, active: bool) -> None:
        self._call("lbm_batch_set_active", int(index), int(bool(active)))

    def step(self, n: int = 1) -> None:
        self._call("lbm_batch_step", C.c_int64(int(n)))

    def step_each(self, nsteps) -> None:
        """Box i advances nsteps[i] steps (0 = sits out), asynchronously."""
        a = np.ascontiguousarray(np.asarray(nsteps, dtype=np.int64))
        if a.shape != (len(self.sims),):
            raise LbmError(LBM_EINVAL, f"need {len(self.sims)} step counts")
        self._call("lbm_batch_step_each", C.c_void_p(a.ctypes.data), len(self.sims))

    def step_one(self, index: int, n: int) -> None:
        """Box `index` advances n steps alone (its own step path), asynchronously."""
        self._call("lbm_batch_step_one", int(index), C.c_int64(int(n)))

    def sync(self) -> None:
        self._call("lbm_batch_sync")

    @property
    def steps_done(self) -> int:
        return int(load_library().lbm_batch_steps_done(self.handle))

    @property
    def kernel_launches(self) -> int:
        return int(load_library().lbm_batch_kernel_launches(self.handle))

    def close(self) -> None:
        if getattr(self, "handle", None):
            load_library().lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
