"""Seeded synthetic surfaces: icospheres and star-shaped bumpy surfaces.

These generators produce the triangle meshes that both the FP64 oracle and
the CUDA path consume.  They hold no boundary-integral arithmetic: only mesh
construction (icosahedron subdivision, a radial map) and plain geometry.

Conventions
-----------
* ``verts`` is float64 ``[Nv, 3]`` in angstrom.
* ``tris`` is int32 ``[N, 3]``; each triangle is counter-clockwise seen from
  outside, so ``(v1 - v0) x (v2 - v0)`` points out of the enclosed region
  (the paper's normal points from the solute into the solvent, Eq. (1)).
* Subdivision ``s`` gives ``N = 20 * 4**s`` triangles.
"""
from __future__ import annotations

import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def _subdivide(v, f):
    """Split every triangle into four at its edge midpoints (projected to the unit sphere)."""
    nv = v.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    e_sorted = np.sort(e, axis=1)
    key = e_sorted[:, 0] * (nv + 1) + e_sorted[:, 1]
    uniq, inv = np.unique(key, return_inverse=True)
    a = uniq // (nv + 1)
    b = uniq % (nv + 1)
    mid = v[a] + v[b]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    nf = f.shape[0]
    m01 = nv + inv[:nf]
    m12 = nv + inv[nf:2 * nf]
    m20 = nv + inv[2 * nf:]
    f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
    newf = np.concatenate(
        [
            np.stack([f0, m01, m20], axis=1),
            np.stack([f1, m12, m01], axis=1),
            np.stack([f2, m20, m12], axis=1),
            np.stack([m01, m12, m20], axis=1),
        ],
        axis=0,
    )
    return np.concatenate([v, mid], axis=0), newf


def unit_icosphere(subdiv: int):
    """Unit icosphere with ``20 * 4**subdiv`` triangles, vertices on the unit sphere."""
    if subdiv < 0:
        raise ValueError("subdiv must be >= 0")
    v, f = _icosahedron()
    for _ in range(subdiv):
        v, f = _subdivide(v, f)
    # orient every face outward (the base table is already CCW from outside,
    # the check keeps it that way under subdivision)
    c = v[f].mean(axis=1)
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, c) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f.astype(np.int32)


def icosphere(radius: float, subdiv: int, center=(0.0, 0.0, 0.0)):
    """Icosphere of the given radius: vertices on the sphere, flat triangles inside it."""
    v, f = unit_icosphere(subdiv)
    return v * float(radius) + np.asarray(center, dtype=np.float64), f


# ----------------------------------------------------------------------------
# real orthonormal spherical harmonics (own recurrence, no library dependency)
# ----------------------------------------------------------------------------

def real_sph_harm(lmax: int, unit_dirs: np.ndarray):
    """Real orthonormal spherical harmonics Y_lm for 0 <= l <= lmax at unit directions.

    Returns a dict ``{(l, m): values}`` with ``-l <= m <= l``.  Normalised so that
    the integral of ``Y_lm**2`` over the unit sphere is 1.  Built from the
    standard three-term recurrence of the normalised associated Legendre functions.
    """
    x, y, z = unit_dirs[:, 0], unit_dirs[:, 1], unit_dirs[:, 2]
    ct = np.clip(z, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    phi = np.arctan2(y, x)
    # fully normalised P_l^m (including sqrt((2l+1)/(4pi) (l-m)!/(l+m)!)), no Condon-Shortley phase
    P = {}
    P[(0, 0)] = np.full_like(ct, np.sqrt(1.0 / (4.0 * np.pi)))
    for m in range(1, lmax + 1):
        P[(m, m)] = np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[(m - 1, m - 1)]
    for m in range(0, lmax):
        P[(m + 1, m)] = np.sqrt(2.0 * m + 3.0) * ct * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[(l, m)] = a * (ct * P[(l - 1, m)] - b * P[(l - 2, m)])
    Y = {}
    for l in range(lmax + 1):
        Y[(l, 0)] = P[(l, 0)]
        for m in range(1, l + 1):
            Y[(l, m)] = np.sqrt(2.0) * P[(l, m)] * np.cos(m * phi)
            Y[(l, -m)] = np.sqrt(2.0) * P[(l, m)] * np.sin(m * phi)
    return Y


def bumpy_surface(radius: float, subdiv: int, rng: np.random.Generator,
                  amplitude: float = 0.12, lmin: int = 2, lmax: int = 6,
                  center=(0.0, 0.0, 0.0)):
    """Star-shaped surface r(w) = R (1 + amplitude * S(w)) mapped radially from an icosphere.

    ``S = sum_{l=lmin..lmax, m} c_lm Y_lm`` with ``c_lm ~ N(0, 1)``, scaled so that
    ``max |S|`` over the mesh vertices is 1 (so r stays in R(1 +- amplitude)).
    Returns ``verts, tris, coeffs`` (coeffs maps (l, m) to the scaled c_lm).
    """
    u, f = unit_icosphere(subdiv)
    Y = real_sph_harm(lmax, u)
    coeffs = {}
    S = np.zeros(u.shape[0])
    for l in range(lmin, lmax + 1):
        for m in range(-l, l + 1):
            c = rng.standard_normal()
            coeffs[(l, m)] = c
            S += c * Y[(l, m)]
    scale = 1.0 / np.max(np.abs(S))
    S *= scale
    coeffs = {k: c * scale for k, c in coeffs.items()}
    r = radius * (1.0 + amplitude * S)
    return u * r[:, None] + np.asarray(center, dtype=np.float64), f, coeffs


# ----------------------------------------------------------------------------
# plain geometry helpers used by the site sampler
# ----------------------------------------------------------------------------

def point_triangle_distance(p: np.ndarray, a: np.ndarray, b: np.ndarray, c: np.ndarray):
    """Exact Euclidean distance from points ``p`` to triangles ``(a, b, c)`` (broadcast, rows).

    Region-based closest-point construction (vertex, edge and face regions).
    """
    ab = b - a
    ac = c - a
    ap = p - a
    d1 = np.einsum("ij,ij->i", ab, ap)
    d2 = np.einsum("ij,ij->i", ac, ap)
    bp = p - b
    d3 = np.einsum("ij,ij->i", ab, bp)
    d4 = np.einsum("ij,ij->i", ac, bp)
    cp = p - c
    d5 = np.einsum("ij,ij->i", ab, cp)
    d6 = np.einsum("ij,ij->i", ac, cp)
    va = d3 * d6 - d5 * d4
    vb = d5 * d2 - d1 * d6
    vc = d1 * d4 - d3 * d2
    n = p.shape[0]
    q = np.empty((n, 3))
    done = np.zeros(n, dtype=bool)

    def put(mask, val):
        nonlocal done
        m = mask & ~done
        q[m] = val[m]
        done |= m

    put((d1 <= 0) & (d2 <= 0), a)
    put((d3 >= 0) & (d4 <= d3), b)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = d1 / (d1 - d3)
        put((vc <= 0) & (d1 >= 0) & (d3 <= 0), a + v[:, None] * ab)
        put((d6 >= 0) & (d5 <= d6), c)
        w = d2 / (d2 - d6)
        put((vb <= 0) & (d2 >= 0) & (d6 <= 0), a + w[:, None] * ac)
        w2 = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        put((va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0), b + w2[:, None] * (c - b))
        denom = 1.0 / (va + vb + vc)
        vv = vb * denom
        ww = vc * denom
        put(np.ones(n, dtype=bool), a + ab * vv[:, None] + ac * ww[:, None])
    return np.linalg.norm(p - q, axis=1)


def mesh_stats(verts: np.ndarray, tris: np.ndarray):
    """Areas and circumradius bound (max vertex distance from centroid) of every triangle."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cen = (a + b + c) / 3.0
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    rad = np.max(np.stack([np.linalg.norm(a - cen, axis=1),
                           np.linalg.norm(b - cen, axis=1),
                           np.linalg.norm(c - cen, axis=1)], axis=1), axis=1)
    return cen, area, rad
