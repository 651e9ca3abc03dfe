"""Pins for the oracle's panel integrals and quadrature rules (Sec. "The boundary element method").

Each check compares against something the mathematics fixes independently of
the oracle: solid angles of closed polyhedra (double-layer identity), brute
force 2-D adaptive quadrature, the planar closed form of int 1/R, the exactness
degree of the Gauss rules.
"""
import numpy as np
import pytest
from scipy import integrate

import gen
from oracle import geometry, panel

FOUR_PI = 4.0 * np.pi


def _closed_meshes():
    v0, f0 = gen.icosphere(1.0, 0)
    v1, f1 = gen.icosphere(2.0, 1)
    rng = np.random.default_rng(7)
    v2, f2, _ = gen.bumpy_surface(3.0, 1, rng, amplitude=0.2)
    return [(v0, f0), (v1, f1), (v2, f2)]


@pytest.mark.parametrize("mesh_id", [0, 1, 2])
def test_double_layer_solid_angle(mesh_id):
    """sum_j int_Tj dG_L/dn_y = -1 inside, -1/2 at a panel centroid, 0 outside (closed surface)."""
    v, f = _closed_meshes()[mesh_id]
    cen, nrm, area = geometry.panel_geometry(v, f)
    n = f.shape[0]
    V0, V1, V2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    for x in (np.zeros(3), np.array([0.2, -0.15, 0.1])):
        _, kl, _, _ = panel.panel_integrals(np.repeat(x[None], n, 0), V0, V1, V2, 0.125)
        assert abs(kl.sum() + 1.0) < 1e-13
    for i in (0, n // 3, n - 1):
        _, kl, _, _ = panel.panel_integrals(np.repeat(cen[i][None], n, 0), V0, V1, V2, 0.125,
                                            self_panel=np.arange(n) == i)
        assert abs(kl.sum() + 0.5) < 1e-13
        assert kl[i] == 0.0
    x = np.array([5.0, 1.0, -2.0])
    _, kl, _, _ = panel.panel_integrals(np.repeat(x[None], n, 0), V0, V1, V2, 0.125)
    assert abs(kl.sum()) < 1e-13


def _brute(x, a, b, c, kappa):
    cr = np.cross(b - a, c - a)
    j2 = np.linalg.norm(cr)
    n = cr / j2

    def f(t, s, which):
        y = a + s * (b - a) + t * (1.0 - s) * (c - a)
        r = x - y
        R = np.linalg.norm(r)
        e = np.exp(-kappa * R)
        val = (1.0 / R, n @ r / R ** 3, e / R, n @ r * (1.0 + kappa * R) * e / R ** 3)[which]
        return val * j2 * (1.0 - s) / FOUR_PI

    return [integrate.dblquad(lambda t, s: f(t, s, w), 0, 1, 0, 1, epsabs=1e-15, epsrel=1e-13)[0]
            for w in range(4)]


TRI = (np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.1, 0.0]), np.array([0.2, 0.9, 0.1]))


@pytest.mark.parametrize("x", [
    [0.3, 0.3, 0.5],        # above the interior
    [0.4, 0.3, 0.02],       # nearly singular, foot inside
    [0.5, 0.05, -0.01],     # nearly singular, foot close to an edge
    [1.5, 1.2, -0.3],       # foot outside
    [-0.3, -0.2, 0.1],      # foot outside, behind a vertex
])
def test_panel_integrals_vs_brute_force(x):
    x = np.asarray(x, dtype=float)
    a, b, c = TRI
    got = panel.panel_integrals(x[None], a[None], b[None], c[None], 0.125)
    ref = _brute(x, a, b, c, 0.125)
    for g, r in zip(got, ref):
        assert abs(g[0] - r) < 1e-12 * max(1.0, abs(r)), (g[0], r)


def _planar_int_invR(p, a, b, c):
    """Closed form of int_T 1/R dS for p in the plane of T: sum over edges of
    d_e * ln((t_b + s_b) / (t_a + s_a)), d_e the signed distance from p to edge e,
    t the position along the edge and s the distance to the edge's end points."""
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    tot = 0.0
    for P, Q in ((a, b), (b, c), (c, a)):
        L = np.linalg.norm(Q - P)
        u = (Q - P) / L
        d = np.dot(np.cross(P - p, Q - p), n) / L
        ta = np.dot(P - p, u)
        tb = np.dot(Q - p, u)
        sa = np.linalg.norm(P - p)
        sb = np.linalg.norm(Q - p)
        tot += d * np.log((tb + sb) / (ta + sa))
    return tot


def test_self_panel_single_layer_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, b, c = rng.normal(size=(3, 3))
        cen = (a + b + c) / 3.0
        vl, kl, vy, ky = panel.panel_integrals(cen[None], a[None], b[None], c[None], 0.125,
                                               self_panel=np.array([True]))
        ref = _planar_int_invR(cen, a, b, c) / FOUR_PI
        assert abs(vl[0] - ref) < 1e-13 * abs(ref)
        assert kl[0] == 0.0 and ky[0] == 0.0
        assert 0.0 < vy[0] < vl[0]


def test_double_layer_jump_across_panel():
    """Approaching the panel interior from either side, int dG_L/dn_y -> +-1/2 (the jump)."""
    a, b, c = TRI
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    foot = (a + b + c) / 3.0
    for h in (1e-3, 1e-5, 1e-7):
        _, kp, _, _ = panel.panel_integrals((foot + h * n)[None], a[None], b[None], c[None], 0.125)
        _, km, _, _ = panel.panel_integrals((foot - h * n)[None], a[None], b[None], c[None], 0.125)
        assert abs(kp[0] - 0.5) < 5 * h and abs(km[0] + 0.5) < 5 * h


def test_gauss_rules_exactness():
    """The K=1, 3, 4, 19 rules integrate polynomials of degree 1, 2, 3, 9 exactly over a triangle."""
    # exact: int over the unit right triangle of x^i y^j = i! j! / (i + j + 2)!
    from math import factorial
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    f = np.array([[0, 1, 2]], dtype=np.int32)
    for k, deg in ((1, 1), (3, 2), (4, 3), (19, 9)):
        y, w = geometry.gauss_points(v, f, k)
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                got = np.sum(w[0] * y[0, :, 0] ** i * y[0, :, 1] ** j)
                ref = factorial(i) * factorial(j) / factorial(i + j + 2)
                assert abs(got - ref) < 1e-15
        # and not one degree higher (the rule is exactly of that degree)
        got = np.sum(w[0] * y[0, :, 0] ** (deg + 1))
        ref = factorial(deg + 1) / factorial(deg + 3)
        assert abs(got - ref) > 1e-8
    lam, wb = geometry.gauss_rule(19)
    assert lam.shape == (19, 3) and np.all(wb > 0) and np.all(lam > 0)
    assert np.allclose(lam.sum(axis=1), 1.0, rtol=0, atol=1e-15)


def test_rule19_is_the_published_degree9_rule():
    """The moment equations of degree 9 fix the 19-node rule's 12 orbit parameters; the
    solution equals the published table (tests/golden/dunavant19_degree9.json, 15 digits)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "dunavant19_degree9.json")))
    lam, w = geometry.gauss_rule(19)
    assert abs(w[0] - gold["centroid_weight"]) < 1e-13
    assert np.allclose(lam[0], 1.0 / 3.0, rtol=0, atol=1e-16)
    for k, orb in enumerate(gold["orbits_aa"]):
        rows = lam[1 + 3 * k:4 + 3 * k]
        assert np.allclose(np.sort(rows, axis=1), [np.sort([orb["a"], orb["a"], 1 - 2 * orb["a"]])] * 3, rtol=0, atol=1e-13)
        assert np.allclose(w[1 + 3 * k:4 + 3 * k], orb["weight_per_node"], rtol=0, atol=1e-13)
    o = gold["orbit_abc"]
    want = np.sort([o["b"], o["c"], 1 - o["b"] - o["c"]])
    assert np.allclose(np.sort(lam[13:], axis=1), [want] * 6, rtol=0, atol=1e-13)
    assert np.allclose(w[13:], o["weight_per_node"], rtol=0, atol=1e-13)


def test_rule19_on_nearly_singular_pairs():
    """Near a panel (the paper applies 19 nodes within 1.25 sqrt(A) of the collocation point)
    the 19-node sums approach the exact integrals much faster than the 4-node rule."""
    a, b, c = TRI
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    verts = np.array([a, b, c])
    n = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(n)
    n /= np.linalg.norm(n)
    cen = (a + b + c) / 3.0
    err = {}
    for k in (4, 19):
        y, w = geometry.gauss_points(verts, tri, k)
        err[k] = []
        for dist in (1.25, 2.5):
            x = cen + dist * np.sqrt(area) * (0.6 * n + 0.8 * (b - a) / np.linalg.norm(b - a))
            ex = panel.panel_integrals(x[None], a[None], b[None], c[None], 0.125)
            kp = panel.kpoint_sums(x[None], y, w, n[None], 0.125)
            err[k].append(max(abs(kp[r][0] - ex[r][0]) / abs(ex[r][0]) for r in range(4)))
    assert err[19][0] < err[4][0] / 20 and err[19][1] < err[4][1] / 100
    assert err[19][1] < err[19][0] / 20


def test_kpoint_far_converges_to_exact():
    """Far from the panel the K-node sum approaches the exact integral at the rule's order."""
    a, b, c = TRI
    errs = []
    for dist in (2.0, 4.0, 8.0):
        x = np.array([0.4, 0.3, dist])
        ex = panel.panel_integrals(x[None], a[None], b[None], c[None], 0.125)
        y, w = geometry.gauss_points(np.array([a, b, c]), np.array([[0, 1, 2]], dtype=np.int32), 4)
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        kp = panel.kpoint_sums(x[None], y, w, n[None], 0.125)
        errs.append(abs(kp[0][0] - ex[0][0]) / ex[0][0])
    # degree-3 rule: relative error of 1/R falls like (size/dist)^4
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8


def test_near_pairs_threshold():
    v, f = gen.icosphere(4.0, 3)
    cen, _, area = geometry.panel_geometry(v, f)
    ptr, cols = geometry.near_pairs(cen, area, 2.0)
    n = f.shape[0]
    rng = np.random.default_rng(0)
    for i in rng.choice(n, 25, replace=False):
        d = np.linalg.norm(cen - cen[i], axis=1)
        ref = np.nonzero(d < 2.0 * np.sqrt(area[i]))[0]
        got = cols[ptr[i]:ptr[i + 1]]
        assert np.array_equal(np.sort(ref), got)
        assert i in got
    # about 4 pi panels within 2 sqrt(A)
    assert 8 < np.diff(ptr).mean() < 18
