"""The allocation-free mass entry point, lbm_mass_noalloc.

Some callers may not allocate device memory of their own: their device
memory is owned by another allocator or pool, or cudaMalloc's implicit
synchronisation is not acceptable in their loop. They cannot hand the
library a workspace, so lbm_mass_noalloc keeps its reduction scratch in a
fixed file-scope device array instead. This test calls it through the C ABI
twice in a row on the same buffer and compares each result with the
workspace-based lbm_mass of the same state. It lives in its own file, named
to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import inputs
from paper_1708_01613_gb300 import Simulation, make_config
from paper_1708_01613_gb300 import lbm as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_mass_noalloc_matches_workspace_mass_twice(storage):
    """512 x 300 cells (three 65,536-cell reduction blocks) of populations
    from a stepped box. The 16-bit buffer handed to lbm_mass_noalloc holds
    the deviations g = f - w_i rho_ref rounded to the storage type (the
    conversion lbm_load_populations applies), so lbm_mass of a box loaded with
    the same populations sums the same stored values."""
    import torch

    nx, ny = 512, 300
    rho = inputs.noise_density(nx, ny, seed=11)
    rho_ref = float(np.mean(rho))
    sim = Simulation(make_config(nx, ny, storage=storage, rho_ref=rho_ref))
    sim.init_density(rho)
    sim.step(25)
    f = sim.read("pops", device=True)["pops"]  # FP32 [9][ny][nx] on the device
    sim.load_populations(f)
    ref = sim.mass()  # the existing entry point (workspace scratch)
    if storage == "f32":
        buf = f.contiguous()
    else:
        _, _, w = inputs_lattice_weights()
        wref = torch.tensor([np.float32(wi * rho_ref) for wi in w], dtype=torch.float32, device=f.device)
        dt = torch.float16 if storage == "f16" else torch.bfloat16
        buf = (f - wref[:, None, None]).to(dt).contiguous()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=f.device)
    lib = L.load_library()
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream(f.device)
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.lbm_mass_noalloc(C.c_void_p(buf.data_ptr()), nx, ny, L.STORAGE[storage], rho_ref,
                                  C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()), err, 256)
        assert rc == L.LBM_OK, err.value
        stream.synchronize()
        got = float(out.item())
        # the same stored values summed in FP64 in another order
        assert got == pytest.approx(ref, rel=1e-12, abs=0.0)
    assert ref == pytest.approx(float(np.sum(rho)), rel=1e-5 if storage == "f32" else 2e-3)


def inputs_lattice_weights():
    """D2Q9 directions and weights (Eqs. 15-16) as the lattice tables of the
    test suite give them."""
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    return ex, ey, w


def test_mass_noalloc_rejects_oversize_and_bad_arguments():
    import torch

    lib = L.load_library()
    err = C.create_string_buffer(256)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    pops = torch.zeros(9 * 16, dtype=torch.float32, device="cuda")
    rc = lib.lbm_mass_noalloc(C.c_void_p(pops.data_ptr()), 1 << 15, 1 << 14, 0, 1.0, None,
                              C.c_void_p(out.data_ptr()), err, 256)
    assert rc == L.LBM_EINVAL and b"static scratch limit" in err.value
    rc = lib.lbm_mass_noalloc(None, 4, 4, 0, 1.0, None, C.c_void_p(out.data_ptr()), err, 256)
    assert rc == L.LBM_EINVAL
