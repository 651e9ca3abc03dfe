"""The seeded synthetic workloads meet the input recipe they are documented with.

The checks are independent of the generators' own logic. Mesh closure and orientation
come from the directed-edge multiset and the signed volume. Sites inside a surface are
found by ray casting (Moller-Trumbore), and their distance to it by exact point-triangle
distances. The remaining checks cover separations, moment conventions (symmetric traceless
quadrupoles), parameter ranges, and the panel and site totals of the binding batch.
"""
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import gen


def _closed_oriented(tris, nv):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    key = e[:, 0].astype(np.int64) * nv + e[:, 1]
    rev = e[:, 1].astype(np.int64) * nv + e[:, 0]
    return np.unique(key).size == key.size and np.array_equal(np.sort(key), np.sort(rev))


def _volume(verts, tris):
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c)))) / 6.0


def _seg_dist(p, a, b):
    ab = b - a
    t = np.clip(np.einsum("ij,ij->i", p - a, ab) / np.einsum("ij,ij->i", ab, ab), 0.0, 1.0)
    return np.linalg.norm(p - (a + t[:, None] * ab), axis=1)


def _point_triangle_dist(p, a, b, c):
    """Exact distance from p to triangles (a, b, c), row-aligned."""
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    h = np.einsum("ij,ij->i", p - a, n)
    q = p - h[:, None] * n
    inside = ((np.einsum("ij,ij->i", np.cross(b - a, q - a), n) >= 0)
              & (np.einsum("ij,ij->i", np.cross(c - b, q - b), n) >= 0)
              & (np.einsum("ij,ij->i", np.cross(a - c, q - c), n) >= 0))
    edge = np.minimum(np.minimum(_seg_dist(p, a, b), _seg_dist(p, b, c)), _seg_dist(p, c, a))
    return np.where(inside, np.abs(h), edge)


def _min_dist_to_surface(points, verts, tris, radius):
    """Smallest distance from each point to the surface, exact for distances below `radius`."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cen = (a + b + c) / 3.0
    circ = np.max(np.stack([np.linalg.norm(v - cen, axis=1) for v in (a, b, c)]), axis=0).max()
    cand = cKDTree(cen).query_ball_point(points, radius + circ)
    out = np.full(points.shape[0], np.inf)
    for i, js in enumerate(cand):
        if js:
            js = np.asarray(js)
            out[i] = _point_triangle_dist(np.repeat(points[i][None], js.size, axis=0), a[js], b[js], c[js]).min()
    return out


def _inside(points, verts, tris, direction=(0.3141, 0.5926, 0.7418)):
    """Parity of ray crossings along a fixed generic direction (odd = inside)."""
    d = np.asarray(direction) / np.linalg.norm(direction)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    e1, e2 = b - a, c - a
    pv = np.cross(d[None], e2)
    det = np.einsum("ij,ij->i", e1, pv)
    out = np.zeros(points.shape[0], dtype=bool)
    for i, p in enumerate(points):
        t = p - a
        u = np.einsum("ij,ij->i", t, pv) / det
        qv = np.cross(t, e1)
        v = (qv @ d) / det
        s = np.einsum("ij,ij->i", e2, qv) / det
        hits = (u >= 0) & (v >= 0) & (u + v <= 1) & (s > 0)
        out[i] = np.count_nonzero(hits) % 2 == 1
    return out


def _check_moments(sites, alpha_range):
    Q = sites.Q
    assert np.allclose(Q, np.transpose(Q, (0, 2, 1)), atol=1e-14)
    assert np.allclose(np.trace(Q, axis1=1, axis2=2), 0.0, atol=1e-13)
    assert np.all(np.abs(sites.q) <= 1.0)
    assert np.all(sites.alpha >= alpha_range[0]) and np.all(sites.alpha <= alpha_range[1])


def _min_pair_dist(pos):
    d, _ = cKDTree(pos).query(pos, k=2)
    return float(d[:, 1].min())


def test_sphere_20480_recipe():
    pr = gen.sphere_r10_20480()
    assert pr.n_panels == 20480 and pr.sites.n == 100
    assert _closed_oriented(pr.tris, len(pr.verts))
    assert _volume(pr.verts, pr.tris) == pytest.approx(4.0 / 3.0 * np.pi * 1000.0, rel=2e-3)
    assert np.all(np.linalg.norm(pr.sites.pos, axis=1) <= 8.0)
    assert _min_pair_dist(pr.sites.pos) >= 1.5
    _check_moments(pr.sites, (0.5, 1.5))


def test_bumpy_81920_recipe():
    pr = gen.bumpy_r14_81920()
    assert pr.n_panels == 81920 and pr.sites.n == 2000
    assert _closed_oriented(pr.tris, len(pr.verts))
    assert _volume(pr.verts, pr.tris) > 0.0
    r = np.linalg.norm(pr.verts, axis=1)
    assert 14.0 * 0.6 < r.min() and r.max() < 14.0 * 1.4       # bumps of a few tens of percent
    assert np.ptp(r) > 0.1 * 14.0                               # and really bumpy
    assert _min_pair_dist(pr.sites.pos) >= 1.2
    dist = _min_dist_to_surface(pr.sites.pos, pr.verts, pr.tris, 3.0)
    assert dist.min() >= 1.5
    sample = np.random.default_rng(5).choice(pr.sites.n, size=60, replace=False)
    assert np.all(_inside(pr.sites.pos[sample], pr.verts, pr.tris))
    _check_moments(pr.sites, gen.configs.DENSE_ALPHA)


def test_inside_test_sees_outside_points():
    pr = gen.sphere_r4_1280()
    pts = np.array([[0.0, 0.0, 0.0], [3.5, 0.0, 0.0], [4.5, 0.0, 0.0], [0.0, 0.0, -6.0]])
    assert _inside(pts, pr.verts, pr.tris).tolist() == [True, True, False, False]


@pytest.mark.slow
def test_binding_batch_recipe():
    triples = gen.binding_triples()
    assert len(triples) == 16
    systems = [p for t in triples for p in t]
    assert sum(p.n_panels for p in systems) == 2531840
    assert sum(p.sites.n for p in systems) == 14968
    for a, b, ab in triples:
        for body in (a, b):
            assert body.n_panels in (1280, 5120, 20480, 81920)
            assert 50 <= body.sites.n <= 2000
            assert _closed_oriented(body.tris, len(body.verts))
        assert ab.n_panels == a.n_panels + b.n_panels and ab.sites.n == a.sites.n + b.sites.n
        nb = ab.panel_body
        va = ab.verts[np.unique(ab.tris[nb == 0])]
        vb = ab.verts[np.unique(ab.tris[nb == 1])]
        assert vb[:, 0].min() - va[:, 0].max() >= 3.0 - 1e-9   # the 3 A slab between the partners


def test_kirkwood_golden_matches_the_sphere_workload():
    """tests/golden/kirkwood_sphere_r10_100sites.json (written by make_kirkwood_sphere_r10.py
    from oracle.kirkwood) belongs to the sites the 20,480-panel workload generates now, and
    its value is the closed form's (Born-like sign and size: |Delta G| of a few hundred to a
    few thousand kcal/mol for 100 unit-scale multipoles in a 10 A cavity)."""
    import hashlib
    import json
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "kirkwood_sphere_r10_100sites.json")))
    st = gen.sphere_r10_20480().sites
    h = hashlib.sha256()
    for a in (st.pos, st.q, st.d, st.Q, st.alpha):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    assert h.hexdigest() == gold["sites_sha256"]
    assert gold["n_sites"] == st.n == 100
    assert -5000.0 < gold["dG_kcal"] < -100.0
