"""Pins for the closed-form sphere solution and, through it, the whole oracle chain.

The Kirkwood series is checked against scipy's Bessel functions, the Born and
centred-dipole closed forms, finite differences of a directly summed Legendre
series, and reciprocity.  The discrete BEM solution of the oracle must then
converge to it at the rate of a piecewise-constant method (error ~ mean panel
area, Sec. "Spherical cavity"), and Richardson extrapolation over three meshes
must land on it.
"""
import numpy as np
import pytest
from scipy import special

import gen
from oracle import kirkwood as kw, multipole as mp

FOUR_PI = 4.0 * np.pi


def test_g_coefficients_vs_scipy():
    for x in (0.05, 0.5, 1.0, 3.0):
        g = kw.g_coeffs(30, x)
        n = np.arange(31)
        ref = x * special.spherical_kn(n, x, derivative=True) / special.spherical_kn(n, x)
        assert np.allclose(g, ref, rtol=1e-12)
    g0 = kw.g_coeffs(5, 0.0)
    assert np.array_equal(g0, -(np.arange(6) + 1.0))


def test_born_and_centred_dipole():
    for eps1, eps2, kappa, a in ((1.0, 80.0, 0.125, 4.0), (2.0, 78.3, 0.0, 3.0)):
        s = gen.Sites(pos=np.zeros((1, 3)), q=np.array([1.3]), d=np.zeros((1, 3)), Q=np.zeros((1, 3, 3)),
                      alpha=np.zeros(1))
        got, _, _ = kw.solvation(s, a, eps1, eps2, kappa, 0.39)
        assert abs(got - kw.born(1.3, a, eps1, eps2, kappa)) < 1e-12 * abs(got)
        p = np.array([0.2, -0.4, 0.3])
        s = gen.Sites(pos=np.zeros((1, 3)), q=np.zeros(1), d=p[None], Q=np.zeros((1, 3, 3)), alpha=np.zeros(1))
        got, _, _ = kw.solvation(s, a, eps1, eps2, kappa, 0.39)
        f1 = kw.f_coeffs(1, eps1, eps2, kappa, a)[1]
        ref = 0.5 * f1 * (p @ p) / (FOUR_PI * a ** 3) * mp.KCAL_PER_UNIT
        assert abs(got - ref) < 1e-12 * abs(ref)
    # Born example: q = 1, a = 4 A, eps 1/80, no salt -> -40.99 kcal/mol
    assert abs(kw.born(1.0, 4.0, 1.0, 80.0, 0.0) + 40.99) < 0.01


def _series(r, s, f, a):
    rn, sn = np.linalg.norm(r), np.linalg.norm(s)
    c = r @ s / (rn * sn)
    n = np.arange(f.size)
    return np.sum(f * (rn * sn / a ** 2) ** n * special.eval_legendre(n, c)) / (FOUR_PI * a)


def test_reaction_jets_vs_fd_and_reciprocity():
    a = 4.0
    f = kw.f_coeffs(120, 1.0, 80.0, 0.125, a)
    rng = np.random.default_rng(8)
    r0 = rng.normal(size=3) * 1.2
    s0 = rng.normal(size=3) * 1.1
    u = rng.normal(size=3)
    v = rng.normal(size=3)
    J = kw.reaction_jets(r0[None], u[None], s0[None], v[None], f, a)[0]
    assert abs(J[0, 0] - _series(r0, s0, f, a)) < 1e-14
    assert abs(J[0, 0] - _series(s0, r0, f, a)) < 1e-14
    h = 1e-4
    G = lambda e, d: _series(r0 + e * u, s0 + d * v, f, a)
    d10 = (G(h, 0) - G(-h, 0)) / (2 * h)
    d01 = (G(0, h) - G(0, -h)) / (2 * h)
    d11 = (G(h, h) - G(h, -h) - G(-h, h) + G(-h, -h)) / (4 * h * h)
    d20 = (G(h, 0) - 2 * G(0, 0) + G(-h, 0)) / (h * h)
    assert abs(J[1, 0] - d10) < 1e-9
    assert abs(J[0, 1] - d01) < 1e-9
    assert abs(J[1, 1] - d11) < 1e-7
    assert abs(2 * J[2, 0] - d20) < 1e-6


def _problem_on(sub, sites, params, radius=4.0):
    v, f = gen.icosphere(radius, sub)
    return gen.Problem("sphere", v, f, sites, params)


@pytest.mark.slow
def test_oracle_bem_converges_to_kirkwood_sphere_r4():
    """The two sites of the 1,280-panel sphere: error ~ A (ratio ~4 per subdivision), Richardson
    extrapolation within 1e-4."""
    pr = gen.sphere_r4_1280()
    exact, _, _ = kw.solvation(pr.sites, 4.0, 1.0, 80.0, 0.125, 0.39)
    vals = [mp.solvation(_problem_on(s, pr.sites, pr.params)).dG_kcal for s in (2, 3, 4)]
    e = np.abs(np.array(vals) - exact)
    assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5
    rich = vals[2] + (vals[2] - vals[1]) / 3.0
    assert abs(rich - exact) < 1e-4 * abs(exact)


def test_oracle_bem_random_multipoles_vs_kirkwood():
    """Random charges, dipoles, traceless quadrupoles and Thole-damped polarizable sites."""
    pr = gen.sphere_random(4.0, 2, 5, 2.2, 1.2, 11)
    exact, mu_ex, _ = kw.solvation(pr.sites, 4.0, 1.0, 80.0, 0.125, 0.39)
    vals = []
    for s in (2, 3):
        r = mp.solvation(_problem_on(s, pr.sites, pr.params), direct_polarization=True)
        vals.append(r.dG_kcal)
    e = np.abs(np.array(vals) - exact)
    assert e[1] < e[0] / 3.0
    rich = vals[1] + (vals[1] - vals[0]) / 3.0
    assert abs(rich - exact) < 2e-3 * abs(exact)
    assert abs(vals[1] - exact) < 1e-2 * abs(exact)


def test_equal_permittivity_no_salt_has_no_reaction():
    """eps1 = eps2, kappa = 0: the medium is homogeneous, so Delta G_solv -> 0 with refinement."""
    pr = gen.sphere_random(4.0, 2, 4, 2.0, 1.2, 12)
    pr.params.eps_out = 1.0
    pr.params.kappa = 0.0
    g = [mp.solvation(_problem_on(s, pr.sites, pr.params), direct_polarization=True).dG_kcal for s in (2, 3)]
    assert abs(g[1]) < abs(g[0]) / 3.0
    pr2 = gen.sphere_random(4.0, 2, 4, 2.0, 1.2, 12)
    ref = abs(mp.solvation(_problem_on(3, pr2.sites, pr2.params), direct_polarization=True).dG_kcal)
    assert abs(g[1]) < 1e-2 * ref


@pytest.mark.parametrize("kind", ["quadrupole", "dipole", "charge"])
def test_single_moment_off_centre_vs_kirkwood(kind):
    """One off-centre site carrying only one kind of moment, so that moment's reaction
    energy is the whole of Delta G: checks each term of Eqs. rhs_multipole and
    energy_multipole_polarizable in isolation (O(A) convergence, Richardson)."""
    rng = np.random.default_rng(21)
    q = np.zeros(1)
    d = np.zeros((1, 3))
    Q = np.zeros((1, 3, 3))
    if kind == "quadrupole":
        A = rng.normal(size=(3, 3))
        A = A + A.T
        Q[0] = A - np.trace(A) / 3 * np.eye(3)
    elif kind == "dipole":
        d[0] = rng.normal(size=3)
    else:
        q[0] = 0.7
    s = gen.Sites(pos=np.array([[0.9, -0.6, 1.1]]), q=q, d=d, Q=Q, alpha=np.zeros(1))
    exact, _, _ = kw.solvation(s, 4.0, 1.0, 80.0, 0.125, 0.39)
    vals = [mp.solvation(_problem_on(sub, s, gen.Params())).dG_kcal for sub in (2, 3)]
    e = np.abs(np.array(vals) - exact)
    assert 3.0 < e[0] / e[1] < 5.0
    rich = vals[1] + (vals[1] - vals[0]) / 3.0
    assert abs(rich - exact) < 3e-3 * abs(exact)


# ---------------------------------------------------------------- Stern layer (a < r < b, no ions)

def _stern_order_n_by_linear_solve(n, eps1, eps2, kappa, a, b):
    """Reaction coefficient B of phi_1 = r^-(n+1)/eps1 + B r^n for one Legendre order, from the
    four interface conditions (continuity of phi and of eps dphi/dr at r = a and at r = b) solved
    as a 4 x 4 linear system in (B, C, D, F), with phi_2 = C r^n + D r^-(n+1) in the layer and
    phi_3 = F k_n(kappa r) outside (scipy's k_n)."""
    kn = special.spherical_kn(n, kappa * b)
    dkn = kappa * special.spherical_kn(n, kappa * b, derivative=True)
    A = np.array([
        [a ** n, -a ** n, -a ** -(n + 1.0), 0.0],
        [eps1 * n * a ** (n - 1.0), -eps2 * n * a ** (n - 1.0), eps2 * (n + 1.0) * a ** -(n + 2.0), 0.0],
        [0.0, b ** n, b ** -(n + 1.0), -kn],
        [0.0, eps2 * n * b ** (n - 1.0), -eps2 * (n + 1.0) * b ** -(n + 2.0), -eps2 * dkn],
    ])
    rhs = np.array([-a ** -(n + 1.0) / eps1, (n + 1.0) * a ** -(n + 2.0), 0.0, 0.0])
    return np.linalg.solve(A, rhs)[0]


def test_stern_coefficients_vs_interface_linear_solve():
    for eps1, eps2, kappa, a, b in ((4.0, 80.0, 0.125, 4.0, 5.0), (1.0, 78.3, 0.4, 3.0, 4.5)):
        f = kw.f_coeffs(12, eps1, eps2, kappa, a, b)
        for n in range(13):
            ref = _stern_order_n_by_linear_solve(n, eps1, eps2, kappa, a, b)
            assert f[n] * a ** -(2.0 * n + 1.0) == pytest.approx(ref, rel=1e-9), n


def test_stern_special_cases():
    # b = a: the layer vanishes; kappa = 0: ions absent, the layer is plain solvent
    for kappa in (0.0, 0.125, 1.0):
        assert np.allclose(kw.f_coeffs(60, 4.0, 80.0, kappa, 4.0, 4.0), kw.f_coeffs(60, 4.0, 80.0, kappa, 4.0),
                           rtol=1e-13, atol=0.0)
    assert np.allclose(kw.f_coeffs(60, 4.0, 80.0, 0.0, 4.0, 5.0), kw.f_coeffs(60, 4.0, 80.0, 0.0, 4.0),
                       rtol=1e-13, atol=0.0)
    # a thicker layer keeps the ions further away: the screening contribution only weakens
    f4, f5, f9 = (kw.f_coeffs(10, 4.0, 80.0, 0.125, 4.0, b) for b in (4.0, 5.0, 9.0))
    f_none = kw.f_coeffs(10, 4.0, 80.0, 0.0, 4.0)
    assert np.all(f4 <= f5) and np.all(f5 <= f9) and np.all(f9 <= f_none + 1e-15)
    with pytest.raises(ValueError):
        kw.f_coeffs(3, 4.0, 80.0, 0.125, 4.0, 3.5)


def test_stern_born_ion():
    for eps1, eps2, kappa, a, b in ((4.0, 80.0, 0.125, 4.0, 5.0), (1.0, 78.3, 0.3, 2.0, 3.4)):
        s = gen.Sites(pos=np.zeros((1, 3)), q=np.array([-0.7]), d=np.zeros((1, 3)), Q=np.zeros((1, 3, 3)),
                      alpha=np.zeros(1))
        got, _, _ = kw.solvation(s, a, eps1, eps2, kappa, 0.39, b=b)
        ref = kw.born_stern(-0.7, a, b, eps1, eps2, kappa)
        assert got == pytest.approx(ref, rel=1e-12)
        assert kw.born_stern(-0.7, a, a, eps1, eps2, kappa) == pytest.approx(kw.born(-0.7, a, eps1, eps2, kappa),
                                                                            rel=1e-13)


def test_paper_production_near_settings_converge():
    """One far node and 19 nodes for near pairs within 1.25 sqrt(A) (Sec. "Comparison with
    Tinker-APBS") still converge at O(A) to the closed form; with 4 far nodes the 19-node near
    rule moves the discrete Delta G by far less than the discretisation error."""
    from oracle import bem
    pr = gen.sphere_r4_1280()
    par = pr.params
    exact, _, _ = kw.solvation(pr.sites, 4.0, par.eps_in, par.eps_out, par.kappa, par.thole_a)

    def dG(sub, k, nf, rule):
        v, f = gen.icosphere(4.0, sub)
        m = bem.build_mesh(v, f, k, nf, near_rule=rule)
        solver = bem.DenseSolver(m, par.eps_in, par.eps_out, par.kappa)
        solver.mesh = m
        return mp.solvation(gen.Problem("sphere", v, f, pr.sites, par), solver=solver,
                            direct_polarization=True).dG_kcal

    vals = [dG(s, 1, 1.25, "gauss19") for s in (2, 3)]
    e = np.abs(np.array(vals) - exact)
    assert 3.0 < e[0] / e[1] < 4.5
    rich = vals[1] + (vals[1] - vals[0]) / 3.0
    assert abs(rich - exact) < 3e-3 * abs(exact)
    g19, gex = dG(3, 4, 2.0, "gauss19"), dG(3, 4, 2.0, "exact")
    assert abs(g19 - gex) < 1e-2 * abs(gex - exact)
