"""The treecode's far-field coefficient table (bempol_far_coefficients, host only).

The library evaluates the Cartesian Taylor expansion of the Laplace and Yukawa kernels about a
cell centre (Sec. "The treecode algorithm") as sum_m g_m(|Delta|) sum_e Delta^e B_(m,e), with the
per-cell coefficients B formed from the cell's moments by this table.  Two pins, both independent
of the library's arithmetic:
- exactness: for one unit source at offset h, the table's expansion equals the Taylor polynomial
  of G(|Delta - h|) in h to order P, whose coefficients are computed here by symbolic
  differentiation (sympy), for G = 1/r and G = exp(-kappa r)/r;
- convergence: for a cluster of charges and dipoles the expansion approaches the direct sums of
  the single- and double-layer kernels, with the error falling like (rho / |Delta|)^(P + 1) and
  (rho / |Delta|)^P.
The radial sequence g_m = (1/r d/dr)^m G is also taken from sympy, not from the library.
"""
import math

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

KAPPA = 0.7
bp = None  # the binding, imported once the library is built


@pytest.fixture(scope="module", autouse=True)
def _library():
    from conftest import build_library
    build_library()
    global bp
    import paper_1810_03698_gb300
    bp = paper_1810_03698_gb300


def _multi_indices(P):
    """Moment order of the table: k = (a, b, n - a - b), n = 0..P, a = n..0, b = n - a..0."""
    return [(a, b, n - a - b) for n in range(P + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def _entries(P):
    """Entry order of the table: e = (a, b, c) ascending a, b, c with |e| <= P; m = |e| .. (P + |e|) // 2."""
    out = []
    for a in range(P + 1):
        for b in range(P + 1):
            for c in range(P + 1):
                d = a + b + c
                if d > P:
                    continue
                for m in range(d, (P + d) // 2 + 1):
                    out.append((m, (a, b, c)))
    return out


def _radial(P, yukawa):
    """g_0 .. g_P with g_m = (1/r d/dr)^m G, as functions of r (sympy, then lambdify)."""
    r = sp.symbols("r", positive=True)
    G = sp.exp(-KAPPA * r) / r if yukawa else 1 / r
    gs = [G]
    for _ in range(P):
        gs.append(sp.simplify(sp.diff(gs[-1], r) / r))
    return [sp.lambdify(r, g, "math") for g in gs]


def _expand(P, yukawa, delta, moments):
    """sum_m g_m(|Delta|) sum_e Delta^e B_(m,e)(moments) with the library's table."""
    ptr, mom, coef = bp.far_coefficients(P)
    ent = _entries(P)
    assert len(ptr) == len(ent) + 1
    B = np.array([np.dot(coef[ptr[q]:ptr[q + 1]], moments[mom[ptr[q]:ptr[q + 1]]]) for q in range(len(ent))])
    g = [f(float(np.linalg.norm(delta))) for f in _radial(P, yukawa)]
    return sum(g[m] * np.prod(delta ** np.array(e)) * B[q] for q, (m, e) in enumerate(ent))


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6])
def test_table_sizes(P):
    ptr, mom, coef = bp.far_coefficients(P)
    nb = sum((d + 1) * (d + 2) // 2 * ((P - d) // 2 + 1) for d in range(P + 1))
    assert len(ptr) == nb + 1 and ptr[0] == 0 and np.all(np.diff(ptr) >= 1)
    assert len(mom) == len(coef) == ptr[-1]
    assert mom.min() >= 0 and mom.max() < len(_multi_indices(P))


@pytest.mark.parametrize("P,yukawa", [(2, False), (4, False), (6, False), (3, True), (5, True)])
def test_expansion_equals_the_taylor_polynomial(P, yukawa):
    """One unit source at h: the expansion is sum_k a_k(Delta) h^k with a_k = (1/k!) d^k/dh^k G(|Delta - h|)."""
    delta = np.array([1.3, -0.7, 2.1])
    h = np.array([0.11, 0.07, -0.09])
    hx, hy, hz = sp.symbols("hx hy hz")
    R = sp.sqrt((delta[0] - hx) ** 2 + (delta[1] - hy) ** 2 + (delta[2] - hz) ** 2)
    G = sp.exp(-KAPPA * R) / R if yukawa else 1 / R
    taylor = 0.0
    moments = []
    for k in _multi_indices(P):
        d = sp.diff(G, hx, k[0], hy, k[1], hz, k[2]) if sum(k) else G
        a_k = float(d.subs({hx: 0, hy: 0, hz: 0})) / (math.factorial(k[0]) * math.factorial(k[1]) * math.factorial(k[2]))
        hk = float(np.prod(h ** np.array(k)))
        taylor += a_k * hk
        moments.append(hk)
    got = _expand(P, yukawa, delta, np.array(moments))
    assert abs(got - taylor) <= 1e-13 * abs(taylor)


@pytest.mark.parametrize("yukawa", [False, True])
def test_expansion_converges_to_the_direct_sums(yukawa):
    """Charges q and dipoles d in a ball of radius rho about the centre: the expansions of the
    single layer sum q G(|Delta - h|) and of the double layer sum d . grad_y G(|x - y|) (moments
    D_k = sum_j k_j d_j h^(k - e_j)) converge to the direct sums like (rho / |Delta|)^(P + 1)
    and (rho / |Delta|)^P."""
    rng = np.random.default_rng(7)
    rho = 0.6
    h = rng.normal(size=(40, 3))
    h *= (rho * rng.uniform(0.2, 1.0, size=40) / np.linalg.norm(h, axis=1))[:, None]
    q = rng.normal(size=40)
    dip = rng.normal(size=(40, 3))
    delta = np.array([2.4, 1.1, -1.6])
    r = np.linalg.norm(delta - h, axis=1)
    if yukawa:
        V = np.sum(q * np.exp(-KAPPA * r) / r)
        K = np.sum(np.einsum("ij,ij->i", dip, delta - h) * (1 + KAPPA * r) * np.exp(-KAPPA * r) / r ** 3)
    else:
        V = np.sum(q / r)
        K = np.sum(np.einsum("ij,ij->i", dip, delta - h) / r ** 3)
    ratio = rho / np.linalg.norm(delta)
    last = None
    for P in range(1, 7):
        ks = _multi_indices(P)
        M = np.array([np.sum(q * np.prod(h ** np.array(k), axis=1)) for k in ks])
        D = np.zeros(len(ks))
        for t, k in enumerate(ks):
            for j in range(3):
                if k[j] == 0:
                    continue
                km = list(k)
                km[j] -= 1
                D[t] += k[j] * np.sum(dip[:, j] * np.prod(h ** np.array(km), axis=1))
        eV = abs(_expand(P, yukawa, delta, M) - V) / abs(V)
        eK = abs(_expand(P, yukawa, delta, D) - K) / abs(K)
        # the double layer's moments of order k carry dipoles times h^(k-1): one order less
        assert eV < 2 * ratio ** (P + 1), (P, eV)
        assert eK < 10 * ratio ** P, (P, eK)
        last = (eV, eK)
    assert last[0] < 1e-5 and last[1] < 1e-3


def test_bad_order_is_rejected():
    with pytest.raises(bp.BempolError):
        bp.far_coefficients(0)
    with pytest.raises(bp.BempolError):
        bp.far_coefficients(7)
