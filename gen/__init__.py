"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path (no solver code)."""
from .surfaces import icosphere, unit_icosphere, bumpy_surface
from .sites import Sites, random_multipoles
from .configs import Params, Problem, WORKLOADS, sphere_r4_1280, sphere_r10_20480, bumpy_r14_81920, \
    binding_triples, bumpy_r24_327680, small_bumpy, small_triple, two_body, sphere_random, bumpy_problem, \
    with_params

__all__ = [
    "icosphere", "unit_icosphere", "bumpy_surface", "Sites", "random_multipoles", "Params",
    "Problem", "WORKLOADS", "sphere_r4_1280", "sphere_r10_20480", "bumpy_r14_81920", "binding_triples",
    "bumpy_r24_327680", "small_bumpy", "small_triple", "two_body", "sphere_random", "bumpy_problem",
    "with_params",
]
