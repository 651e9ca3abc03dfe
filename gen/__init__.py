"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path (no solver code)."""
from .surfaces import icosphere, unit_icosphere, bumpy_surface
from .sites import Sites, random_multipoles
from .configs import Params, Problem, CONFIGS, config1, config2, config3, config4, config5, \
    small_bumpy, small_triple, two_body, sphere_random, bumpy_problem, with_params

__all__ = [
    "icosphere", "unit_icosphere", "bumpy_surface", "Sites", "random_multipoles", "Params",
    "Problem", "CONFIGS", "config1", "config2", "config3", "config4", "config5", "small_bumpy",
    "small_triple", "two_body",
    "sphere_random", "bumpy_problem", "with_params",
]
