"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol include/lbm.h declares; configuration validation and workspace sizing
work without a GPU. No compute call is made here."""
import ctypes as C
import os
import re

import pytest

from paper_1708_01613_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    names = _declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding knows every declared entry point, under the same name
    assert set(names) == set(lbm.SIGNATURES)


def test_config_defaults():
    c = lbm.lbm_config_default()
    assert (c.nx, c.ny, c.storage, c.barrier, c.relabel_every, c.zone_radius) == (256, 256, 0, 0, 1, 4)
    assert c.tau == 1.0 and c.G == -5.5 and c.rho0 == 1.0
    assert abs(c.gas_threshold - 0.6931471805599453) < 1e-15 and c.rupture_eps == 1e-6


def test_workspace_bytes_and_validation():
    N = 512 * 256
    c = lbm.make_config(512, 256)
    b32 = lbm.lbm_workspace_bytes(c)
    assert b32 >= 2 * 9 * N * 4 + 8 * N
    c16 = lbm.make_config(512, 256, storage="f16")
    assert lbm.lbm_workspace_bytes(c16) < b32
    cb = lbm.make_config(512, 256, barrier=True)
    assert lbm.lbm_workspace_bytes(cb) >= b32 + 7 * N
    for bad in (dict(nx=3, ny=64), dict(nx=64, ny=64, tau=0.5), dict(nx=64, ny=64, relabel_every=0),
                dict(nx=8, ny=64, zone_radius=4, barrier=True), dict(nx=64, ny=64, rho0=0.0)):
        nx, ny = bad.pop("nx"), bad.pop("ny")
        assert lbm.lbm_workspace_bytes(lbm.make_config(nx, ny, **bad)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_config(8, 64, zone_radius=4)) > 0  # R unused without barrier
    c.storage = 7
    assert lbm.lbm_workspace_bytes(c) == 0


def test_config_rules_of_the_variants():
    """The rules of the growth source and the two-component mode, and the
    field ranges, are checked on the host before any device work."""
    ok = lbm.make_config(256, 64, components=2, barrier=True, G_mg=1.0)
    assert lbm.lbm_workspace_bytes(ok) > 2 * lbm.lbm_workspace_bytes(lbm.make_config(256, 64))
    bad = [
        dict(components=2, storage="f16"),                  # two components: FP32 only
        dict(components=2, growth=True),                    # no growth source with two lattices
        dict(components=2, tau_g=0.5),                      # tau_g > 0.5
        dict(components=2, G_mg=float("nan")),
        dict(components=3),
        dict(components=2, barrier=True, zone_radius=17),   # two-lattice barrier: tiled pipeline, R_z <= 16
        dict(nx=65536, ny=65536),                           # nx * ny beyond int32
        dict(G=float("inf")),
        dict(rupture_eps=float("nan")),
        dict(barrier=True, zone_radius=-1),
        dict(barrier=True, zone_radius=32),                 # 2 R_z + 1 must stay below ny = 64
    ]
    for kw in bad:
        nx, ny = kw.pop("nx", 256), kw.pop("ny", 64)
        assert lbm.lbm_workspace_bytes(lbm.make_config(nx, ny, **kw)) == 0, kw
    c = lbm.make_config(256, 64)
    c.barrier = 2
    assert lbm.lbm_workspace_bytes(c) == 0
    c = lbm.make_config(256, 64)
    c.growth = 3
    assert lbm.lbm_workspace_bytes(c) == 0
    # growth reserves a gas-point list of 4 bytes per cell
    g = lbm.lbm_workspace_bytes(lbm.make_config(256, 64, growth=True, barrier=True))
    assert g >= lbm.lbm_workspace_bytes(lbm.make_config(256, 64, barrier=True)) + 4 * 256 * 64


def test_create_rejects_bad_arguments_without_gpu_work():
    lib = lbm.load_library()
    c = lbm.make_config(64, 64)
    h = C.c_void_p()
    assert lib.lbm_create(C.byref(c), None, 1 << 20, None, C.byref(h)) == lbm.LBM_EINVAL
    assert lib.lbm_create(C.byref(c), C.c_void_p(0x1001), 1 << 30, None, C.byref(h)) == lbm.LBM_EINVAL
    assert lib.lbm_create(C.byref(c), C.c_void_p(0x1000), 16, None, C.byref(h)) == lbm.LBM_ENOMEM
    assert not h.value
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_last_error(None) == b"handle is NULL"
    lib.lbm_destroy(None)


def test_product_path_does_not_use_the_oracle():
    """The package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1708_01613_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "lbm_oracle" not in txt and "liboracle" not in txt, f
