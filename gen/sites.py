"""Seeded AMOEBA-like multipole sites inside a closed surface.

Each site carries a charge q (e), a permanent dipole d (e*A), a traceless
symmetric quadrupole Q (e*A^2, in the paper's convention Q = int rho (3 r r -
r^2 I), the one used by the multipole potential of Sec. "Computation of the
right-hand side"), a polarizability alpha (A^3) and a polarisation group.

No solver arithmetic lives here: only sampling, rejection and plain geometry.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

from .surfaces import point_triangle_distance, mesh_stats, unit_icosphere


@dataclass
class Sites:
    pos: np.ndarray          # [Ns, 3] float64, A
    q: np.ndarray            # [Ns] float64, e
    d: np.ndarray            # [Ns, 3] float64, e*A (permanent dipole)
    Q: np.ndarray            # [Ns, 3, 3] float64, e*A^2 (traceless symmetric)
    alpha: np.ndarray        # [Ns] float64, A^3
    group: np.ndarray = field(default=None)   # [Ns] int32 polarisation group
    body: np.ndarray = field(default=None)    # [Ns] int32 body index

    def __post_init__(self):
        n = self.pos.shape[0]
        if self.group is None:
            self.group = np.arange(n, dtype=np.int32)
        if self.body is None:
            self.body = np.zeros(n, dtype=np.int32)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def random_multipoles(rng: np.random.Generator, n: int, q_range=(-1.0, 1.0), d_sigma=0.3,
                      Q_sigma=0.2, alpha_range=(0.5, 1.5)):
    """Draw q ~ U, d ~ N(0, d_sigma), traceless symmetric Q (entries N(0, Q_sigma)), alpha ~ U."""
    q = rng.uniform(q_range[0], q_range[1], size=n)
    d = rng.normal(0.0, d_sigma, size=(n, 3))
    A = rng.normal(0.0, Q_sigma, size=(n, 3, 3))
    Q = np.triu(A) + np.swapaxes(np.triu(A, 1), 1, 2)
    tr = np.trace(Q, axis1=1, axis2=2)
    Q = Q - (tr / 3.0)[:, None, None] * np.eye(3)[None]
    alpha = rng.uniform(alpha_range[0], alpha_range[1], size=n)
    return q, d, Q, alpha


class StarSurfaceInside:
    """Inside test and surface distance for a mesh mapped radially from a unit icosphere.

    The ray from the centre in direction w crosses exactly the mapped triangle
    whose unit-icosphere triangle contains w, so inside <=> |p - c| is below the
    ray-plane intersection distance of that triangle.
    """

    def __init__(self, verts, tris, subdiv, center=(0.0, 0.0, 0.0)):
        self.center = np.asarray(center, dtype=np.float64)
        self.verts = verts
        self.tris = tris
        u, f = unit_icosphere(subdiv)
        if not np.array_equal(f, tris):
            raise ValueError("mesh topology does not match the icosphere of this subdivision")
        self.u = u
        uc = u[f].mean(axis=1)
        uc /= np.linalg.norm(uc, axis=1, keepdims=True)
        self.unit_tree = cKDTree(uc)
        cen, area, rad = mesh_stats(verts, tris)
        self.cen = cen
        self.max_rad = float(rad.max())
        self.tri_tree = cKDTree(cen)

    def inside(self, p: np.ndarray) -> np.ndarray:
        w = p - self.center
        r = np.linalg.norm(w, axis=1)
        wd = w / np.maximum(r, 1e-300)[:, None]
        k = min(12, self.tris.shape[0])
        _, cand = self.unit_tree.query(wd, k=k)
        out = np.zeros(p.shape[0], dtype=bool)
        found = np.zeros(p.shape[0], dtype=bool)
        for j in range(k):
            t = cand[:, j]
            a, b, c = self.u[self.tris[t, 0]], self.u[self.tris[t, 1]], self.u[self.tris[t, 2]]
            s1 = np.einsum("ij,ij->i", wd, np.cross(a, b))
            s2 = np.einsum("ij,ij->i", wd, np.cross(b, c))
            s3 = np.einsum("ij,ij->i", wd, np.cross(c, a))
            hit = (s1 >= 0) & (s2 >= 0) & (s3 >= 0) & ~found
            if np.any(hit):
                A = self.verts[self.tris[t[hit], 0]] - self.center
                B = self.verts[self.tris[t[hit], 1]] - self.center
                C = self.verts[self.tris[t[hit], 2]] - self.center
                n = np.cross(B - A, C - A)
                tdist = np.einsum("ij,ij->i", n, A) / np.einsum("ij,ij->i", n, wd[hit])
                out[hit] = r[hit] < tdist
                found |= hit
        if not np.all(found):
            raise RuntimeError("ray-triangle search failed")
        return out

    def distance(self, p: np.ndarray, cap: float) -> np.ndarray:
        """Exact distance to the mesh for points closer than ``cap``; ``>= cap`` otherwise."""
        out = np.full(p.shape[0], np.inf)
        lists = self.tri_tree.query_ball_point(p, cap + self.max_rad)
        for i, lst in enumerate(lists):
            if not lst:
                continue
            t = np.asarray(lst)
            a = self.verts[self.tris[t, 0]]
            b = self.verts[self.tris[t, 1]]
            c = self.verts[self.tris[t, 2]]
            pp = np.repeat(p[i][None], t.size, axis=0)
            out[i] = point_triangle_distance(pp, a, b, c).min()
        return out


def _greedy_min_sep(kept, nkept, cands, n, min_sep):
    """Append candidates in order when they are >= min_sep from every kept point."""
    s2 = min_sep * min_sep
    for p in cands:
        if nkept >= n:
            break
        if nkept and np.min(np.sum((kept[:nkept] - p) ** 2, axis=1)) < s2:
            continue
        kept[nkept] = p
        nkept += 1
    return nkept


def sample_inside(rng: np.random.Generator, surf: StarSurfaceInside, n: int, rmax: float,
                  min_surface: float, min_sep: float, batch: int = 4096, max_rounds: int = 5000):
    """Uniform points in the ball of radius rmax that are inside the surface, at least
    ``min_surface`` from it and at least ``min_sep`` from each other."""
    kept = np.zeros((n, 3))
    nkept = 0
    for _ in range(max_rounds):
        if nkept >= n:
            break
        c = rng.uniform(-rmax, rmax, size=(batch, 3))
        c = c[np.sum(c * c, axis=1) <= rmax * rmax] + surf.center
        if c.shape[0]:
            c = c[surf.inside(c)]
        if c.shape[0]:
            c = c[surf.distance(c, min_surface) >= min_surface]
        nkept = _greedy_min_sep(kept, nkept, c, n, min_sep)
    if nkept < n:
        raise RuntimeError("site sampling did not reach the requested count")
    return kept


def sample_ball(rng: np.random.Generator, n: int, rmax: float, min_sep: float,
                center=(0.0, 0.0, 0.0)):
    """Uniform points in a ball with pairwise separation >= min_sep (greedy rejection)."""
    kept = np.zeros((n, 3))
    nkept = 0
    for _ in range(10000):
        if nkept >= n:
            break
        c = rng.uniform(-rmax, rmax, size=(4 * n, 3))
        c = c[np.sum(c * c, axis=1) <= rmax * rmax]
        nkept = _greedy_min_sep(kept, nkept, c, n, min_sep)
    if nkept < n:
        raise RuntimeError("site sampling did not reach the requested count")
    return kept + np.asarray(center, dtype=np.float64)
