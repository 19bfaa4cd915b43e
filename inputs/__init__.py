"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module draws random numbers and places bubbles. It holds none of the
lattice Boltzmann arithmetic: no equilibrium, force, pseudopotential or
pressure. Both sides receive exactly the arrays and bubble lists made here.
"""
from .synth import (  # noqa: F401
    GOLDEN_GAMMA,
    splitmix64_uniform,
    noise_density,
    poisson_disk_bubbles,
    clustered_bubbles,
    log_uniform_sides,
    batch_instances,
    nucleation_schedule,
    serving_requests,
    RHO_GAS_G55,
    RHO_LIQ_G55,
    request_bubbles,
)
