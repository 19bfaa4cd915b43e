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


def test_mass_noalloc_matches_workspace_mass_twice():
    import torch

    nx, ny = 300, 70
    rho = inputs.noise_density(nx, ny, seed=11)
    sim = Simulation(make_config(nx, ny))
    sim.init_density(rho)
    sim.step(25)
    ref = sim.mass()  # the existing entry point (workspace scratch)
    pops = sim.read("pops", device=True)["pops"]  # FP32 [9][ny][nx] on the device
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=pops.device)
    lib = L.load_library()
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream(pops.device)
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.lbm_mass_noalloc(C.c_void_p(pops.data_ptr()), nx, ny, L.STORAGE["f32"], 1.0,
                                  C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()), err, 256)
        assert rc == L.LBM_OK, err.value
        stream.synchronize()
        got = float(out.item())
        # same FP32 values summed in FP64 in another order
        assert got == pytest.approx(ref, rel=1e-12, abs=0.0)
    assert ref == pytest.approx(float(np.sum(rho)), rel=1e-5)


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
