"""Pins for the oracle's multipole algebra, Thole damping, site fields and SCF.

Independent references: central finite differences, harmonicity (Laplace),
reciprocity of interaction energies, the far field of an explicit charge cloud
(which fixes the quadrupole convention of Eq. pot_multipole), Gauss's law for
the Thole smeared charge, and the direct solution of the SCF fixed point.
"""
import numpy as np
import pytest
from scipy import integrate

import gen
from oracle import multipole as mp, bem, panel

FOUR_PI = 4.0 * np.pi


def _fd(fun, R, h=1e-5):
    out = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        out.append((fun(R + e) - fun(R - e)) / (2 * h))
    return np.stack(out, axis=-1)


def test_t_tensors_are_derivatives_and_harmonic():
    rng = np.random.default_rng(1)
    R = rng.normal(size=(6, 3)) * 1.3
    T = mp.t_tensors(R, 4)
    for n in range(4):
        fd = _fd(lambda X: mp.t_tensors(X, 4)[n], R)
        assert np.allclose(fd, T[n + 1], rtol=1e-7, atol=1e-9)
    for n in range(2, 5):
        tr = np.trace(T[n], axis1=1, axis2=2)
        assert np.max(np.abs(tr)) < 1e-12
        # full symmetry under index swaps
        assert np.allclose(T[n], np.swapaxes(T[n], 1, 2))
        assert np.allclose(T[n], np.swapaxes(T[n], 1, -1))


def test_quadrupole_convention_matches_charge_cloud():
    """A cloud of point charges has the far potential of its (q, p, Q) moments with
    Q = sum_c q_c (3 r r - r^2 I), the convention of Eq. pot_multipole."""
    rng = np.random.default_rng(2)
    rc = rng.normal(size=(5, 3)) * 0.05
    qc = rng.normal(size=5)
    q = qc.sum()
    p = (qc[:, None] * rc).sum(0)
    Q = sum(qc[c] * (3 * np.outer(rc[c], rc[c]) - rc[c] @ rc[c] * np.eye(3)) for c in range(5))
    pts = rng.normal(size=(7, 3))
    pts = 3.0 * pts / np.linalg.norm(pts, axis=1, keepdims=True)
    exact = np.array([sum(qc[c] / np.linalg.norm(x - rc[c]) for c in range(5)) for x in pts]) / FOUR_PI
    got = mp.rhs(pts, np.zeros((1, 3)), np.array([q]), p[None], Q[None], 1.0)
    # next term is the octupole: O(|r_c|^3 / R^4)
    assert np.max(np.abs(got - exact)) < 5 * 0.15 ** 3 / 3.0 ** 4 / FOUR_PI * np.abs(qc).sum()
    # the error must be far smaller than the quadrupole term itself
    no_Q = mp.rhs(pts, np.zeros((1, 3)), np.array([q]), p[None], np.zeros((1, 3, 3)), 1.0)
    assert np.max(np.abs(got - exact)) < 0.05 * np.max(np.abs(no_Q - exact))


def test_rhs_literal_equals_tensor_form():
    """Eq. rhs_multipole written literally equals q T0 - p.T1 + Q:T2/6 for traceless Q."""
    rng = np.random.default_rng(3)
    ns = 6
    pos = rng.normal(size=(ns, 3))
    q, d, Q, alpha = gen.random_multipoles(rng, ns)
    pts = rng.normal(size=(9, 3)) * 4 + 8
    got = mp.rhs(pts, pos, q, d, Q, 2.0)
    ref = np.zeros(9)
    for k in range(ns):
        T0, T1, T2 = mp.t_tensors(pts - pos[k], 2)
        ref += q[k] * T0 - T1 @ d[k] + np.einsum("pij,ij->p", T2, Q[k]) / 6.0
    assert np.allclose(got, ref / (FOUR_PI * 2.0), rtol=1e-13, atol=1e-16)


def test_thole_lambda3_is_gauss_law_of_smeared_charge():
    """lambda3(u) = charge enclosed within u of rho = (3a/4pi) exp(-a u^3) (Thole's density)."""
    a = 0.39
    for u in (0.2, 0.7, 1.3, 2.5):
        enc = integrate.quad(lambda s: 4 * np.pi * s * s * 3 * a / (4 * np.pi) * np.exp(-a * s ** 3), 0, u,
                             epsabs=1e-15)[0]
        R = np.array([[u, 0.0, 0.0]])
        l3, _, _ = mp.thole_lambdas(R, np.array([1.0]), np.array([1.0]), a)
        assert abs(l3[0] - enc) < 1e-13


def test_thole_damped_tensors_are_consistent_derivatives():
    """T1d -> T2d -> T3d are gradients of each other (lambda5, lambda7 follow from lambda3)."""
    rng = np.random.default_rng(4)
    al, am, a = 1.3, 0.8, 0.39

    def tensors(X):
        l3, l5, l7 = mp.thole_lambdas(X, np.full(X.shape[0], al), np.full(X.shape[0], am), a)
        return mp.damped_tensors(X, l3, l5, l7)

    R = rng.normal(size=(5, 3)) * 0.9
    T1, T2, T3 = tensors(R)
    assert np.allclose(_fd(lambda X: tensors(X)[0], R), T2, rtol=1e-7, atol=1e-9)
    assert np.allclose(_fd(lambda X: tensors(X)[1], R), T3, rtol=1e-7, atol=1e-9)
    # damping off when either polarizability is zero; vanishes at large separation
    l3, l5, l7 = mp.thole_lambdas(R, np.zeros(5), np.ones(5), a)
    assert np.all(l3 == 1) and np.all(l5 == 1) and np.all(l7 == 1)
    l3, l5, l7 = mp.thole_lambdas(R * 50, np.ones(5), np.ones(5), a)
    assert np.all(1 - l7 < 1e-12)


def _two_sites(rng):
    pos = rng.normal(size=(2, 3)) * 1.5
    q, d, Q, alpha = gen.random_multipoles(rng, 2)
    return gen.Sites(pos=pos, q=q, d=d, Q=Q, alpha=alpha)


def test_interaction_energy_reciprocity_and_field():
    """U = L_1 Phi_2(r_1) = L_2 Phi_1(r_2) for two permanent multipoles; E = -grad Phi."""
    rng = np.random.default_rng(5)
    s = _two_sites(rng)
    z = np.zeros((2, 3))
    P, G, H = mp.mult_potentials(s.pos, s.q, s.d, s.Q, z, s.alpha, s.group, s.body, 1.0, 0.39,
                                 masked=False, same_body_only=False)
    u1 = s.q[0] * P[0] + s.d[0] @ G[0] + np.sum(s.Q[0] * H[0]) / 6
    u2 = s.q[1] * P[1] + s.d[1] @ G[1] + np.sum(s.Q[1] * H[1]) / 6
    assert abs(u1 - u2) < 1e-13 * max(1, abs(u1))

    def pot_at(x):
        sub = gen.Sites(pos=np.vstack([x, s.pos[1]]), q=s.q, d=s.d, Q=s.Q, alpha=s.alpha)
        return mp.mult_potentials(sub.pos, s.q, s.d, s.Q, z, s.alpha, s.group, s.body, 1.0, 0.39,
                                  masked=False, same_body_only=False)

    h = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        gp = (pot_at(s.pos[0] + e)[0][0] - pot_at(s.pos[0] - e)[0][0]) / (2 * h)
        hp = (pot_at(s.pos[0] + e)[1][0] - pot_at(s.pos[0] - e)[1][0]) / (2 * h)
        assert abs(gp - G[0][k]) < 1e-7 * max(1, abs(gp))
        assert np.allclose(hp, H[0][k], rtol=1e-6, atol=1e-8)


def test_reaction_at_sites_potential_and_derivatives():
    """phi_solv = -K_L(phi) + V_L(psi) via the panel K-node sums; grad/Hessian by FD."""
    v, f = gen.icosphere(4.0, 2)
    mesh = bem.build_mesh(v, f, 4, 2.0)
    rng = np.random.default_rng(6)
    phi = rng.normal(size=f.shape[0])
    psi = rng.normal(size=f.shape[0])
    pos = rng.normal(size=(3, 3))
    p0, g0, h0 = mp.reaction_at_sites(mesh, phi, psi, pos)
    n = f.shape[0]
    for l in range(3):
        x = np.repeat(pos[l][None], n, 0)
        vl, kl, _, _ = panel.kpoint_sums(x, mesh.ygauss, mesh.wgauss, mesh.normal, 0.0)
        assert abs(p0[l] - (-kl @ phi + vl @ psi)) < 1e-12 * max(1, abs(p0[l]))
    h = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        pp, gp, _ = mp.reaction_at_sites(mesh, phi, psi, pos + e)
        pm, gm, _ = mp.reaction_at_sites(mesh, phi, psi, pos - e)
        assert np.allclose((pp - pm) / (2 * h), g0[:, k], rtol=1e-7, atol=1e-9)
        assert np.allclose((gp - gm) / (2 * h), h0[:, :, k], rtol=1e-6, atol=1e-8)
    assert np.max(np.abs(np.trace(h0, axis1=1, axis2=2))) < 1e-10 * np.max(np.abs(h0))


def test_sor_reaches_direct_fixed_point():
    """SOR with w = 0.7 converges to the solution of the direct 3Ns system (vacuum and dissolved)."""
    pr = gen.sphere_random(4.0, 2, 6, 2.4, 1.2, 42)
    pr.params.scf_tol = 1e-12
    pr.params.gmres_tol = 1e-12
    r_sor = mp.solvation(pr)
    r_dir = mp.solvation(pr, direct_polarization=True)
    assert np.max(np.abs(r_sor.mu_diss - r_dir.mu_diss)) < 1e-10
    assert np.max(np.abs(r_sor.mu_vac - r_dir.mu_vac)) < 1e-10
    assert abs(r_sor.dG_kcal - r_dir.dG_kcal) < 1e-9 * abs(r_dir.dG_kcal)


def test_kcal_constant():
    # e^2/(4 pi eps0 A) N_A in kcal/mol from the SI-defined constants
    assert abs(mp.COULOMB_KCAL - 332.0637) < 1e-3


def test_polarizability_volume_units():
    """A polarizability volume alpha (A^3) at distance R from a unit charge in vacuum
    carries mu = alpha q / R^2 e*A (Gaussian definition of alpha), i.e. mu = 4 pi alpha E
    in the paper's units where E = q / (4 pi R^2)."""
    s = gen.Sites(pos=np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0]]), q=np.array([1.0, 0.0]),
                  d=np.zeros((2, 3)), Q=np.zeros((2, 3, 3)), alpha=np.array([0.0, 1.7]))
    par = gen.Params(scf_tol=1e-14)
    mu, _ = mp.vacuum_scf(s, par, direct=True)
    assert np.allclose(mu[1], [1.7 / 2.5 ** 2, 0.0, 0.0], rtol=1e-14)
    mu2, _ = mp.vacuum_scf(s, par)
    assert np.allclose(mu2, mu, atol=1e-12)


def test_polarisation_group_mask():
    """Permanent moments of the same polarisation group do not polarise each other
    (Sec. "Calculation of the electric field"): two charges in one group induce nothing,
    in separate groups they do; the energy is unmasked either way."""
    pos = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    q = np.array([1.0, -1.0])
    z3 = np.zeros((2, 3))
    zQ = np.zeros((2, 3, 3))
    alpha = np.array([1.0, 1.0])
    par = gen.Params(scf_tol=1e-14)
    same = gen.Sites(pos=pos, q=q, d=z3, Q=zQ, alpha=alpha, group=np.array([0, 0], dtype=np.int32))
    diff = gen.Sites(pos=pos, q=q, d=z3, Q=zQ, alpha=alpha, group=np.array([0, 1], dtype=np.int32))
    mu_same, _ = mp.vacuum_scf(same, par, direct=True)
    mu_diff, _ = mp.vacuum_scf(diff, par, direct=True)
    assert np.all(mu_same == 0.0)
    assert np.all(np.abs(mu_diff[:, 0]) > 0.05)
    p_same, _, _ = mp.mult_potentials(pos, q, z3, zQ, z3, alpha, same.group, same.body, 1.0, 0.39,
                                      masked=False, same_body_only=False)
    assert np.allclose(p_same, [-1.0 / (FOUR_PI * 2.0), 1.0 / (FOUR_PI * 2.0)], rtol=1e-14)
