"""Panel geometry and quadrature rules (Sec. "The boundary element method").

The surface is discretised into flat triangles with piecewise-constant phi and
dphi/dn, collocated at the panel centroids.  Far-away panels are integrated
with 1, 3 or 4 Gauss nodes; panels closer than ``near_factor * sqrt(A_i)`` to
the collocation point x_i (A_i the area of the collocation point's own panel)
are integrated accurately (see ``panel.py``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np


def panel_geometry(verts: np.ndarray, tris: np.ndarray):
    """Centroid x_i, unit outward normal n_i and area A_i of every triangle.

    Written with separate products and sums (no fused operations), in the order
    centroid = (v0 + v1 + v2) / 3, cross = (v1 - v0) x (v2 - v0), A = |cross| / 2.
    """
    v0 = verts[tris[:, 0]]
    v1 = verts[tris[:, 1]]
    v2 = verts[tris[:, 2]]
    cen = (v0 + v1 + v2) / 3.0
    e1 = v1 - v0
    e2 = v2 - v0
    cr = np.empty_like(e1)
    cr[:, 0] = e1[:, 1] * e2[:, 2] - e1[:, 2] * e2[:, 1]
    cr[:, 1] = e1[:, 2] * e2[:, 0] - e1[:, 0] * e2[:, 2]
    cr[:, 2] = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    nrm = np.sqrt(cr[:, 0] * cr[:, 0] + cr[:, 1] * cr[:, 1] + cr[:, 2] * cr[:, 2])
    area = 0.5 * nrm
    normal = cr / nrm[:, None]
    return cen, normal, area


def gauss_rule(k: int):
    """Barycentric nodes and weights (summing to 1) of the K-node triangle rule.

    K=1: centroid.  K=3: (2/3, 1/6, 1/6) and permutations, degree 2.
    K=4: centroid with weight -27/48 and (3/5, 1/5, 1/5) permutations with
    weight 25/48, degree 3.  The paper names 1, 3 or 4 nodes without giving the
    rules; these are the classical Strang-Fix rules.
    """
    if k == 1:
        lam = np.array([[1 / 3, 1 / 3, 1 / 3]])
        w = np.array([1.0])
    elif k == 3:
        lam = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
        w = np.array([1 / 3, 1 / 3, 1 / 3])
    elif k == 4:
        lam = np.array([[1 / 3, 1 / 3, 1 / 3], [0.6, 0.2, 0.2], [0.2, 0.6, 0.2], [0.2, 0.2, 0.6]])
        w = np.array([-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0])
    else:
        raise ValueError("gauss_k must be 1, 3 or 4")
    return lam, w


def gauss_points(verts: np.ndarray, tris: np.ndarray, k: int):
    """Gauss-node positions y_jg [N, K, 3] and weights W_jg = w_g * A_j [N, K].

    The centroid node of the K=1 and K=4 rules is placed at the panel centroid
    itself, computed exactly as the collocation point ((v0 + v1) + v2) / 3: the
    node then coincides with its own panel's collocation point to the last bit,
    so that pair has r = 0 and contributes nothing (a product form
    v0/3 + v1/3 + v2/3 would miss the centroid by rounding and leave a spurious
    1/r ~ 1e16 term)."""
    lam, w = gauss_rule(k)
    v0 = verts[tris[:, 0]]
    v1 = verts[tris[:, 1]]
    v2 = verts[tris[:, 2]]
    y = (lam[None, :, 0, None] * v0[:, None, :] + lam[None, :, 1, None] * v1[:, None, :]
         + lam[None, :, 2, None] * v2[:, None, :])
    if k in (1, 4):
        y[:, 0, :] = (v0 + v1 + v2) / 3.0
    _, _, area = panel_geometry(verts, tris)
    return y, w[None, :] * area[:, None]


def near_pairs(cen: np.ndarray, area: np.ndarray, near_factor: float):
    """CSR of near pairs: j is near target i when |x_i - c_j|^2 < near_factor^2 * A_i.

    The comparison is made on squared distances in FP64, with the squared
    distance summed as dx*dx + dy*dy + dz*dz in that order.  Includes j = i.
    Returns (row_ptr [N+1] int64, cols int32 sorted ascending per row).
    Candidates come from a k-d tree ball query with a radius above every
    threshold (so no near pair is missed); each candidate then gets the exact test.
    """
    from scipy.spatial import cKDTree

    n = cen.shape[0]
    thr = (near_factor * near_factor) * area
    radius = float(np.sqrt(thr.max())) * (1.0 + 1e-6) + 1e-12
    cand = cKDTree(cen).query_ball_point(cen, radius)
    counts = np.array([len(c) for c in cand], dtype=np.int64)
    ci = np.repeat(np.arange(n), counts)
    cj = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if n else np.zeros(0, np.int64)
    dx = cen[ci, 0] - cen[cj, 0]
    dy = cen[ci, 1] - cen[cj, 1]
    dz = cen[ci, 2] - cen[cj, 2]
    keep = (dx * dx + dy * dy + dz * dz) < thr[ci]
    ci, cj = ci[keep], cj[keep]
    order = np.lexsort((cj, ci))
    ci, cj = ci[order], cj[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(np.bincount(ci, minlength=n))
    return ptr, cj.astype(np.int32)
