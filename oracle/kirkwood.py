"""Closed-form solvation of point multipoles in a dielectric sphere (Kirkwood; Kong
and Ponder's multipole extension), used to pin the discrete BEM solution
(Sec. "Spherical cavity": the BEM error must fall with the mean panel area).

Sphere of radius a centred at the origin, permittivity eps1 inside, eps2 and
inverse Debye length kappa outside.  For a unit charge at s inside, the reaction
potential at r inside is

    G_R(r, s) = 1/(4 pi a) sum_n f_n T_n(r/a, s/a),
    T_n(r, s) = (|r||s|)^n P_n(r^ . s^),
    f_n = (1/eps1) ((n+1) eps1 + eps2 g_n) / (n eps1 - eps2 g_n),
    g_n = x k_n'(x) / k_n(x),  x = kappa a,

(k_n the modified spherical Bessel function of the second kind), obtained by
matching the interior and exterior solutions of Eq. (pde) at r = a.  With a Stern
(ion-exclusion) layer a < r < b of permittivity eps2 and no ions, as in the sphere
test of Sec. "Spherical cavity" (a = 4, b = 5), the layer's solution
C r^n + D r^-(n+1) is matched to the screened exterior at r = b and g_n becomes its
logarithmic derivative r phi'/phi at r = a:

    h_n = -(n+1) + (2n+1) u_n,   u_n = delta_n c_n / (delta_n c_n - (2n+1+delta_n)),
    delta_n = -(n+1) - g_n(kappa b) >= 0,   c_n = (a/b)^(2n+1),

which is g_n(kappa a) when b = a and -(n+1) (plain Laplace decay) when kappa = 0.  T_n obeys
(n+1) T_{n+1} = (2n+1)(r . s) T_n - n |r|^2 |s|^2 T_{n-1}; it is a polynomial in
r and s, so every derivative needed here is evaluated exactly by carrying
truncated bivariate Taylor jets (in eps along a direction u for r, and in
delta along v for s) through that recurrence.

A multipole (q, p, Q) at s acts as L_s = q + p . grad_s + (1/6) Q : grad_s grad_s on
the unit-charge solution (Eq. pot_multipole with traceless Q).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np

from . import multipole as mp

FOUR_PI = 4.0 * np.pi


def g_coeffs(nmax: int, x: float):
    """g_n = x k_n'(x)/k_n(x) for n = 0..nmax (g_n = -(n+1) when x = 0)."""
    n = np.arange(nmax + 1, dtype=np.float64)
    if x == 0.0:
        return -(n + 1.0)
    g = np.empty(nmax + 1)
    g[0] = -1.0 - x
    rho = x / (1.0 + x)          # k_0 / k_1
    for k in range(1, nmax + 1):
        g[k] = -(k + 1.0) - x * rho
        rho = 1.0 / (rho + (2.0 * k + 1.0) / x)   # k_k / k_{k+1}
    return g


def h_coeffs(nmax: int, kappa: float, a: float, b: float):
    """r phi'/phi at r = a+ of the order-n solution in a Stern layer a < r < b (no ions)
    matched at r = b to the screened exterior; n = 0..nmax."""
    if not b >= a:
        raise ValueError("the Stern radius b must be >= a")
    n = np.arange(nmax + 1, dtype=np.float64)
    delta = -(n + 1.0) - g_coeffs(nmax, kappa * b)
    c = np.exp((2.0 * n + 1.0) * np.log(a / b))       # (a/b)^(2n+1), underflows to 0
    u = delta * c / (delta * c - (2.0 * n + 1.0 + delta))
    return -(n + 1.0) + (2.0 * n + 1.0) * u


def f_coeffs(nmax, eps1, eps2, kappa, a, b=None):
    """f_n of the reaction Green's function; b = Stern radius (None: no layer)."""
    g = g_coeffs(nmax, kappa * a) if b is None else h_coeffs(nmax, kappa, a, b)
    n = np.arange(nmax + 1, dtype=np.float64)
    return ((n + 1.0) * eps1 + eps2 * g) / (eps1 * (n * eps1 - eps2 * g))


def _jmul(A, B):
    """Product of truncated jets A, B [..., 3, 3] (coefficients of eps^a delta^b, a, b <= 2)."""
    C = np.zeros(np.broadcast_shapes(A.shape, B.shape))
    for a1 in range(3):
        for b1 in range(3):
            Aa = A[..., a1, b1]
            for a2 in range(3 - a1):
                for b2 in range(3 - b1):
                    C[..., a1 + a2, b1 + b2] += Aa * B[..., a2, b2]
    return C


def reaction_jets(r0, u, s0, v, f, a):
    """Jets of G_R(r0 + eps u, s0 + delta v) for row-aligned arrays [M, 3]; returns [M, 3, 3]."""
    r0 = r0 / a
    s0 = s0 / a
    u = u / a
    v = v / a
    m = r0.shape[0]
    dot = lambda x, y: np.sum(x * y, axis=1)
    rs = np.zeros((m, 3, 3))
    rs[:, 0, 0] = dot(r0, s0)
    rs[:, 1, 0] = dot(u, s0)
    rs[:, 0, 1] = dot(r0, v)
    rs[:, 1, 1] = dot(u, v)
    rr = np.zeros((m, 3, 3))
    rr[:, 0, 0] = dot(r0, r0)
    rr[:, 1, 0] = 2.0 * dot(r0, u)
    rr[:, 2, 0] = dot(u, u)
    ss = np.zeros((m, 3, 3))
    ss[:, 0, 0] = dot(s0, s0)
    ss[:, 0, 1] = 2.0 * dot(s0, v)
    ss[:, 0, 2] = dot(v, v)
    rrss = _jmul(rr, ss)
    Tm = np.zeros((m, 3, 3))
    Tm[:, 0, 0] = 1.0
    T = rs.copy()
    acc = f[0] * Tm + f[1] * T
    for n in range(1, f.size - 1):
        Tn = ((2.0 * n + 1.0) * _jmul(rs, T) - n * _jmul(rrss, Tm)) / (n + 1.0)
        Tm, T = T, Tn
        acc += f[n + 1] * T
    return acc / (FOUR_PI * a)


def _operator_terms(q, p, Q):
    """L = q + p . grad + (1/6) Q : grad grad as (coef, direction, order) per site."""
    terms = []
    w, V = np.linalg.eigh(Q)
    for i in range(q.shape[0]):
        t = [(q[i], np.zeros(3), 0), (1.0, p[i], 1)]
        for k in range(3):
            t.append((w[i, k] / 6.0, V[i][:, k], 2))
        terms.append(t)
    return terms


_FACT = (1.0, 1.0, 2.0)


def _apply(pos_r, terms_r, pos_s, terms_s, f, a, pairs):
    """sum over (l, m) in pairs of L_r^(l) L_s^(m) G_R(r_l, r_m), per pair."""
    out = np.zeros(len(pairs))
    li = np.array([p[0] for p in pairs])
    mi = np.array([p[1] for p in pairs])
    nt_r = len(terms_r[0])
    nt_s = len(terms_s[0])
    for tr in range(nt_r):
        cr = np.array([terms_r[l][tr][0] for l in li])
        ur = np.array([terms_r[l][tr][1] for l in li])
        orr = terms_r[li[0]][tr][2]
        for ts in range(nt_s):
            cs = np.array([terms_s[m][ts][0] for m in mi])
            vs = np.array([terms_s[m][ts][1] for m in mi])
            os_ = terms_s[mi[0]][ts][2]
            J = reaction_jets(pos_r[li], ur, pos_s[mi], vs, f, a)
            out += cr * cs * _FACT[orr] * _FACT[os_] * J[:, orr, os_]
    return out


def solvation(sites, a, eps1, eps2, kappa, thole_a, nmax=None, polarizable=True, b=None):
    """Exact Delta G_solv (kcal/mol) of the sites in the sphere, with induced dipoles;
    b = radius of the Stern layer's outer surface (None: no layer).

    Induced dipoles solve mu = 4 pi alpha (E_reac + E_mult) directly; the
    multipole-multipole terms use the oracle's free-space tensors.
    Returns (dG_kcal, mu_diss, mu_vac).
    """
    pos = sites.pos
    ns = sites.n
    rmax = np.max(np.linalg.norm(pos, axis=1)) / a
    if nmax is None:
        nmax = 20
        while (nmax ** 4) * rmax ** (2 * nmax) > 1e-18 and nmax < 2000:
            nmax += 10
    f = f_coeffs(nmax, eps1, eps2, kappa, a, b)
    four_pi_alpha = FOUR_PI * sites.alpha
    pairs = [(l, m) for l in range(ns) for m in range(ns)]
    li = np.array([p[0] for p in pairs])
    mi = np.array([p[1] for p in pairs])

    class _P:  # parameter bundle for the multipole helpers
        pass
    par = _P()
    par.eps_in, par.thole_a, par.scf_tol, par.scf_maxit, par.sor_omega = eps1, thole_a, 1e-14, 1000, 0.7

    # reaction field at l of the permanent moments, and reaction matrix for dipoles
    zero_q = np.zeros(ns)
    zero_Q = np.zeros((ns, 3, 3))
    terms_perm = _operator_terms(sites.q, sites.d, sites.Q)
    E_reac_perm = np.zeros((ns, 3))
    M = np.zeros((ns, 3, ns, 3))
    for k in range(3):
        ek = np.zeros(3)
        ek[k] = 1.0
        terms_grad = [[(1.0, ek, 1)] for _ in range(ns)]
        g = _apply(pos, terms_grad, pos, terms_perm, f, a, pairs)
        np.add.at(E_reac_perm[:, k], li, -g)
        for c in range(3):
            ec = np.zeros(3)
            ec[c] = 1.0
            terms_dip = [[(1.0, ec, 1)] for _ in range(ns)]
            gg = _apply(pos, terms_grad, pos, terms_dip, f, a, pairs)
            M[li, k, mi, c] = -gg
    _, gperm, _ = mp.mult_potentials(pos, sites.q, sites.d, sites.Q, np.zeros((ns, 3)), sites.alpha,
                                     sites.group, sites.body, eps1, thole_a, masked=True,
                                     same_body_only=True)
    T = mp.thole_matrix(pos, sites.alpha, sites.body, eps1, thole_a, True)
    if polarizable:
        A = np.eye(3 * ns) - np.repeat(four_pi_alpha, 3)[:, None] * (M.reshape(3 * ns, 3 * ns) + T)
        b = (four_pi_alpha[:, None] * (E_reac_perm - gperm)).reshape(-1)
        mu = np.linalg.solve(A, b).reshape(ns, 3)
    else:
        mu = np.zeros((ns, 3))
    # energy: reaction part with sources p = d + mu, energy operator with permanent d
    terms_src = _operator_terms(sites.q, sites.d + mu, sites.Q)
    G_reac = 0.5 * np.sum(_apply(pos, terms_perm, pos, terms_src, f, a, pairs))
    mpot, mg, mh = mp.mult_potentials(pos, sites.q, sites.d, sites.Q, mu, sites.alpha, sites.group,
                                      sites.body, eps1, thole_a, masked=False, same_body_only=True)
    G_diss = G_reac + mp.site_energy(sites.q, sites.d, sites.Q, mpot, mg, mh)
    if polarizable:
        mu_v, _ = mp.vacuum_scf(sites, par, direct=True)
    else:
        mu_v = np.zeros((ns, 3))
    vp, vg, vh = mp.mult_potentials(pos, sites.q, sites.d, sites.Q, mu_v, sites.alpha, sites.group,
                                    sites.body, eps1, thole_a, masked=False, same_body_only=False)
    G_vac = mp.site_energy(sites.q, sites.d, sites.Q, vp, vg, vh)
    del zero_q, zero_Q
    return (G_diss - G_vac) * mp.KCAL_PER_UNIT, mu, mu_v


def born(q, a, eps1, eps2, kappa):
    """Born ion at the centre: (q^2 / (8 pi a)) (1/(eps2 (1 + kappa a)) - 1/eps1), in kcal/mol."""
    return q * q / (8.0 * np.pi * a) * (1.0 / (eps2 * (1.0 + kappa * a)) - 1.0 / eps1) * mp.KCAL_PER_UNIT


def born_stern(q, a, b, eps1, eps2, kappa):
    """Ion at the centre of a sphere of radius a with a Stern layer to radius b (kcal/mol):
    region potentials q/(4 pi eps r) + const matched at r = a and r = b to the screened
    q exp(-kappa (r - b)) / (4 pi eps2 (1 + kappa b) r) outside, which leaves the
    reaction potential (q / 4 pi) (1/(eps2 a) - 1/(eps1 a) - kappa/(eps2 (1 + kappa b)))."""
    phi = q / (4.0 * np.pi) * (1.0 / (eps2 * a) - 1.0 / (eps1 * a) - kappa / (eps2 * (1.0 + kappa * b)))
    return 0.5 * q * phi * mp.KCAL_PER_UNIT
