"""GB300 (sm_103a) implementation of the time step of the extended Shan-Chen
lattice Boltzmann method for metal-foam bubbles (arXiv 1708.01613).

The compute path is the CUDA library ``liblbm.so`` (C ABI in include/lbm.h);
``paper_1708_01613_gb300.lbm`` is its ctypes binding.
"""
from .lbm import (  # noqa: F401
    Batch,
    LbmError,
    Simulation,
    lbm_config,
    lbm_bubble,
    lbm_stats,
    load_library,
    make_config,
    lbm_config_default,
    lbm_workspace_bytes,
)
