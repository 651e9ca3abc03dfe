"""The benchmark workloads as seeded synthetic problems.

Every random draw uses ``numpy.random.default_rng(1810036980 + k)`` where k is the
workload number below, so the oracle and the CUDA path see identical inputs.

  1  sphere R=4 A, icosphere subdivision 3 (1,280 panels), two fixed sites
  2  sphere R=10 A, subdivision 5 (20,480 panels), 100 random sites in r <= 8 A
  3  bumpy star surface R=14 A, subdivision 6 (81,920 panels), 2,000 sites
  5  bumpy star surface R=24 A, subdivision 7 (327,680 panels), 10,000 sites

The paper's own workloads are protein surfaces meshed with msms at 4 vertices
per square angstrom carrying AMOEBA multipoles; these stand in for them with
matching panel counts and site densities.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .surfaces import icosphere, bumpy_surface, mesh_stats
from .sites import Sites, random_multipoles, sample_ball, sample_inside, StarSurfaceInside

SEED_BASE = 1810036980


@dataclass
class Params:
    eps_in: float = 1.0
    eps_out: float = 80.0
    kappa: float = 0.125          # 1/A
    gauss_k: int = 4              # Gauss points per panel for far-away pairs
    near_factor: float = 2.0      # near-singular threshold: |x_i - c_j| < near_factor * sqrt(A_i)
    theta: float = 0.5            # treecode multipole acceptance
    order: int = 5                # treecode Taylor order P
    leaf: int = 256               # treecode leaf size (panels)
    gmres_tol: float = 1e-8
    gmres_restart: int = 100
    gmres_maxit: int = 500
    scf_tol: float = 1e-8         # RMS change of the induced dipoles, e*A
    sor_omega: float = 0.7
    scf_maxit: int = 200
    thole_a: float = 0.39


@dataclass
class Problem:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    sites: Sites
    params: Params
    meta: dict = field(default_factory=dict)

    @property
    def n_panels(self) -> int:
        return int(self.tris.shape[0])


def config1() -> Problem:
    """Sphere R=4, subdivision 3; charge+dipole at the centre, polarizable charge at (1.5,0,0)."""
    v, f = icosphere(4.0, 3)
    sites = Sites(
        pos=np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0]]),
        q=np.array([1.0, -0.5]),
        d=np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 0.0]]),
        Q=np.zeros((2, 3, 3)),
        alpha=np.array([0.0, 1.0]),
    )
    p = Params(gmres_tol=1e-8, scf_tol=1e-8)
    return Problem("sphere_r4_sub3_1280p_2sites", v, f, sites, p,
                   meta={"radius": 4.0, "subdiv": 3, "kind": "sphere"})


def sphere_random(radius: float, subdiv: int, n_sites: int, r_sites: float, min_sep: float,
                  seed_index: int) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_index)
    v, f = icosphere(radius, subdiv)
    pos = sample_ball(rng, n_sites, r_sites, min_sep)
    q, d, Q, alpha = random_multipoles(rng, n_sites)
    sites = Sites(pos=pos, q=q, d=d, Q=Q, alpha=alpha)
    p = Params()
    return Problem(f"sphere_r{radius:g}_sub{subdiv}_{f.shape[0]}p_{n_sites}sites", v, f, sites, p,
                   meta={"radius": radius, "subdiv": subdiv, "kind": "sphere"})


def config2() -> Problem:
    """Sphere R=10, subdivision 5 (20,480 panels), 100 sites uniform in r <= 8, min separation 1.5."""
    pr = sphere_random(10.0, 5, 100, 8.0, 1.5, 2)
    pr.params = Params(gmres_tol=1e-8, scf_tol=1e-8, theta=0.5, order=5)
    return pr


def bumpy_problem(radius: float, subdiv: int, n_sites: int, seed_index: int,
                  min_surface: float = 1.5, min_sep: float = 1.2, alpha_range=(0.5, 1.5)) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_index)
    v, f, coeffs = bumpy_surface(radius, subdiv, rng)
    surf = StarSurfaceInside(v, f, subdiv)
    # sites must also clear the near-singular radius 2 sqrt(A) of every panel
    _, area, _ = mesh_stats(v, f)
    min_surface = max(min_surface, 2.0 * float(np.sqrt(area.max())) + 0.2)
    rmax = radius * 1.12 - min_surface
    pos = sample_inside(rng, surf, n_sites, rmax, min_surface, min_sep)
    q, d, Q, alpha = random_multipoles(rng, n_sites, alpha_range=alpha_range)
    sites = Sites(pos=pos, q=q, d=d, Q=Q, alpha=alpha)
    return Problem(f"bumpy_r{radius:g}_sub{subdiv}_{f.shape[0]}p_{n_sites}sites", v, f, sites, Params(),
                   meta={"radius": radius, "subdiv": subdiv, "kind": "bumpy", "coeffs": coeffs})


# Dense bumpy workloads (2,000 sites at >= 1.2 A in ~8,200 A^3, about five times a
# protein's atom density) draw polarizabilities from U(0.25, 0.75) A^3: with
# U(0.5, 1.5) the damped dipole coupling 4 pi alpha T has an eigenvalue near -2.7,
# outside the range (> 1 - 2/omega = -1.86) where the relaxation
# mu <- (1 - omega) mu + omega 4 pi alpha E converges for omega = 0.7.
DENSE_ALPHA = (0.25, 0.75)


def config3() -> Problem:
    """Bumpy surface R=14, subdivision 6 (81,920 panels), 2,000 sites; tree theta=0.5, P=5."""
    pr = bumpy_problem(14.0, 6, 2000, 3, alpha_range=DENSE_ALPHA)
    pr.params = Params(gmres_tol=1e-6, scf_tol=1e-6, theta=0.5, order=5)
    return pr


def config5() -> Problem:
    """Bumpy surface R=24, subdivision 7 (327,680 panels), 10,000 sites."""
    pr = bumpy_problem(24.0, 7, 10000, 5, alpha_range=DENSE_ALPHA)
    pr.params = Params(gmres_tol=1e-6, scf_tol=1e-6, theta=0.5, order=5)
    return pr


def small_bumpy(subdiv: int = 3, n_sites: int = 40, radius: float = 8.0, seed_index: int = 103) -> Problem:
    """A small bumpy case for quick parity runs (several tiles, ragged tail)."""
    pr = bumpy_problem(radius, subdiv, n_sites, seed_index)
    return pr


def with_params(pr: Problem, **kw) -> Problem:
    return replace(pr, params=replace(pr.params, **kw))


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}
