"""Panel geometry and quadrature rules (Sec. "The boundary element method").

The surface is discretised into flat triangles with piecewise-constant phi and
dphi/dn, collocated at the panel centroids.  Far-away panels are integrated
with 1, 3 or 4 Gauss nodes (19 for the paper's nearly-singular variant); panels
closer than ``near_factor * sqrt(A_i)`` to the collocation point x_i (A_i the area of
the collocation point's own panel) are integrated accurately (see ``panel.py``).

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
    elif k == 19:
        lam, w = _rule19()
    else:
        raise ValueError("gauss_k must be 1, 3, 4 or 19")
    return lam, w


def _rule19():
    """The fully symmetric 19-node rule of degree 9 for the paper's nearly-singular pairs
    ("finer quadrature rules with 19 Gauss nodes", Sec. "Comparison with Tinker-APBS"; the
    paper gives no table).  Orbits: the centroid, four (a, a, 1-2a) orbits of 3 nodes and one
    (b, c, 1-b-c) orbit of 6 nodes, 12 parameters in all; the S3-invariant polynomials of
    degree <= 9 give exactly 12 independent moment equations,
    int l1^i l2^j l3^k dA / A = 2 i! j! k! / (i+j+k+2)!,
    so the degree-9 rule with positive weights and interior nodes is an isolated solution
    (Dunavant, Int. J. Numer. Meth. Eng. 21 (1985) 1129, 19 points, degree 9).  It is solved
    here by least squares on the monomial moments from that table's values rounded to 3
    digits; the solve, not the rounded start, fixes every digit.  Cached."""
    global _RULE19
    if _RULE19 is not None:
        return _RULE19
    from math import factorial
    from scipy.optimize import least_squares

    def nodes(p):
        w0, a1, a2, a3, a4, w1, w2, w3, w4, b, c, w5 = p
        lam, w = [(1 / 3, 1 / 3, 1 / 3)], [w0]
        for a, wa in ((a1, w1), (a2, w2), (a3, w3), (a4, w4)):
            lam += [(a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)]
            w += [wa / 3] * 3
        d = 1 - b - c
        lam += [(b, c, d), (b, d, c), (c, b, d), (c, d, b), (d, b, c), (d, c, b)]
        w += [w5 / 6] * 6
        return np.array(lam), np.array(w)

    mons = [(i, j, k) for i in range(10) for j in range(10) for k in range(10) if i + j + k <= 9 and i >= j >= k]
    exact = np.array([2.0 * factorial(i) * factorial(j) * factorial(k) / factorial(i + j + k + 2) for i, j, k in mons])

    def resid(p):
        lam, w = nodes(p)
        got = np.array([np.sum(w * lam[:, 0] ** i * lam[:, 1] ** j * lam[:, 2] ** k) for i, j, k in mons])
        return got / exact - 1.0  # relative: the high moments are ~1e-7 and must count as much

    # start: the table's centroid weight, orbit parameters and orbit weights (sum of the
    # orbit's node weights), to 3 digits
    p0 = np.array([0.0971, 0.490, 0.437, 0.188, 0.0447, 0.094, 0.233, 0.239, 0.0767, 0.0368, 0.222, 0.260])
    r = least_squares(resid, p0, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=2000)
    lam, w = nodes(r.x)
    if not (np.abs(resid(r.x)).max() < 1e-13 and w.min() > 0 and lam.min() > 0):
        raise RuntimeError("the 19-node degree-9 rule did not converge")
    _RULE19 = (lam, w)
    return _RULE19


_RULE19 = None


def gauss_points(verts: np.ndarray, tris: np.ndarray, k: int):
    """Gauss-node positions y_jg [N, K, 3] and weights W_jg = w_g * A_j [N, K].

    The centroid node of the K=1, K=4 and K=19 rules is placed at the panel centroid
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
    if k in (1, 4, 19):
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
