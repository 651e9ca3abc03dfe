"""The benchmark workloads as seeded synthetic problems.

Every random draw uses ``numpy.random.default_rng(1810036980 + k)`` where k is the
workload number below, so the oracle and the CUDA path see identical inputs.

  1  sphere R=4 A, icosphere subdivision 3 (1,280 panels), two fixed sites
  2  sphere R=10 A, subdivision 5 (20,480 panels), 100 random sites in r <= 8 A
  3  bumpy star surface R=14 A, subdivision 6 (81,920 panels), 2,000 sites
  4  16 triples (A, B, AB) of bumpy bodies, subdivisions 3-6, R 6-14 A; in AB the
     two bodies are 3 A apart along x and share one solvent
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
    damp_permanent: bool = False  # Thole-damp the permanent moments' polarising field (AMOEBA; not the paper's rule)
    near_rule: str = "exact"      # near pairs off the self panel: "exact" (semi-analytical) or "gauss19"


@dataclass
class Problem:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    sites: Sites
    params: Params
    meta: dict = field(default_factory=dict)
    panel_body: np.ndarray = None   # [N] int32 body of each panel (None: one body)

    @property
    def n_panels(self) -> int:
        return int(self.tris.shape[0])


def sphere_r4_1280() -> Problem:
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


def sphere_r10_20480() -> Problem:
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


def bumpy_r14_81920() -> Problem:
    """Bumpy surface R=14, subdivision 6 (81,920 panels), 2,000 sites; tree theta=0.5, P=5."""
    pr = bumpy_problem(14.0, 6, 2000, 3, alpha_range=DENSE_ALPHA)
    pr.params = Params(gmres_tol=1e-6, scf_tol=1e-6, theta=0.5, order=5)
    return pr


def bumpy_r24_327680() -> Problem:
    """Bumpy surface R=24, subdivision 7 (327,680 panels), 10,000 sites."""
    pr = bumpy_problem(24.0, 7, 10000, 5, alpha_range=DENSE_ALPHA)
    pr.params = Params(gmres_tol=1e-6, scf_tol=1e-6, theta=0.5, order=5)
    return pr


def small_bumpy(subdiv: int = 3, n_sites: int = 40, radius: float = 8.0, seed_index: int = 103) -> Problem:
    """A small bumpy case for quick parity runs (several tiles, ragged tail)."""
    pr = bumpy_problem(radius, subdiv, n_sites, seed_index)
    return pr


def two_body(a: Problem, b: Problem, gap: float = 3.0) -> Problem:
    """The complex AB of two bodies in one solvent (Sec. "Calculation of the binding
    energy"): B is moved along +x until the slab between A's largest x and B's smallest
    x is ``gap`` wide, so no point of one surface is closer than ``gap`` to the other.
    Panels and sites keep their order (A first); B's sites get body 1 and their own
    polarisation groups."""
    shift = float(a.verts[:, 0].max() - b.verts[:, 0].min() + gap)
    off = np.array([shift, 0.0, 0.0])
    verts = np.vstack([a.verts, b.verts + off])
    tris = np.vstack([a.tris, b.tris + a.verts.shape[0]]).astype(a.tris.dtype)
    sa, sb = a.sites, b.sites
    sites = Sites(pos=np.vstack([sa.pos, sb.pos + off]), q=np.concatenate([sa.q, sb.q]),
                  d=np.vstack([sa.d, sb.d]), Q=np.concatenate([sa.Q, sb.Q]),
                  alpha=np.concatenate([sa.alpha, sb.alpha]),
                  group=np.concatenate([sa.group, sb.group + int(sa.group.max()) + 1]).astype(np.int32),
                  body=np.concatenate([np.zeros(sa.n, np.int32), np.ones(sb.n, np.int32)]))
    body = np.concatenate([np.zeros(a.n_panels, np.int32), np.ones(b.n_panels, np.int32)])
    return Problem(f"complex[{a.name}+{b.name}]", verts, tris, sites, a.params,
                   meta={"kind": "complex", "shift": shift, "gap": gap}, panel_body=body)


# Sites per body of the binding workload: 0.06 per A^3 of the ball of radius R,
# clamped to [50, 2000].  Coarse meshes need a wider site-free shell (2 sqrt(A_max)),
# which the 81,920-panel workload's density of 0.17 per A^3 would not leave room for.
TRIPLE_SITE_DENSITY = 0.06


def binding_triples(n_triples: int = 16, subdivs=(3, 4, 5, 6), radius=(6.0, 14.0)):
    """Binding workload: ``n_triples`` triples (A, B, AB).  Per body: subdivision uniform
    over ``subdivs``, R ~ U(radius), sites proportional to the volume; AB puts B 3 A
    from A along x.  Returns a list of (A, B, AB)."""
    rng = np.random.default_rng(SEED_BASE + 4)
    out = []
    for t in range(n_triples):
        pair = []
        for k in range(2):
            sub = int(rng.choice(np.asarray(subdivs)))
            R = float(rng.uniform(*radius))
            ns = int(np.clip(round(TRIPLE_SITE_DENSITY * 4.0 / 3.0 * np.pi * R ** 3), 50, 2000))
            pr = bumpy_problem(R, sub, ns, 4000 + 2 * t + k, alpha_range=DENSE_ALPHA)
            pr.params = Params(gmres_tol=1e-6, scf_tol=1e-6, theta=0.5, order=5)
            pair.append(pr)
        out.append((pair[0], pair[1], two_body(pair[0], pair[1])))
    return out


def small_triple(seed_index: int = 401, subdiv: int = 2, radius: float = 6.0, n_sites: int = 12,
                 gap: float = 3.0):
    """A triple small enough for the dense oracle (two bodies of 20 * 4^subdiv panels)."""
    a = bumpy_problem(radius, subdiv, n_sites, seed_index)
    b = bumpy_problem(radius * 0.8, subdiv, max(2, n_sites // 2), seed_index + 1)
    return a, b, two_body(a, b, gap)


def with_params(pr: Problem, **kw) -> Problem:
    return replace(pr, params=replace(pr.params, **kw))


WORKLOADS = {f.__name__: f for f in (sphere_r4_1280, sphere_r10_20480, bumpy_r14_81920, bumpy_r24_327680)}
