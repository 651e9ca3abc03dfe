"""Point multipoles, induced dipoles and the solvation energy (Secs. "Computation of
the right-hand side", "Induced dipole", "Calculation of the solvation energy").

Units: the paper's, i.e. potentials q / (4 pi eps r) with eps the relative
permittivity (vacuum permittivity set to 1), charges in e, lengths in A.
Energies in those units convert to kcal/mol with ``KCAL_PER_UNIT``.
Polarizabilities are AMOEBA polarizability volumes (A^3); in these units the
induced dipole of Eq. (induced_dipole) is mu = 4 pi alpha E.

Multipole tensors: T^(n) = grad^n (1/R) with R = r_field - r_source, so that a
site (q, p, Q) with traceless Q (Eq. pot_multipole) has potential
    Phi = [q T0 - p . T1 + (1/6) Q : T2] / (4 pi eps).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FOUR_PI = 4.0 * np.pi

# e^2 / (4 pi eps0 A) per mole in kcal/mol, from the SI constants
_E = 1.602176634e-19
_EPS0 = 8.8541878128e-12
_NA = 6.02214076e23
COULOMB_KCAL = _E * _E / (FOUR_PI * _EPS0 * 1e-10) * _NA / 4184.0
KCAL_PER_UNIT = FOUR_PI * COULOMB_KCAL

_I3 = np.eye(3)


# ----------------------------------------------------------------------------
# tensors
# ----------------------------------------------------------------------------

def t_tensors(R: np.ndarray, order: int = 4):
    """Cartesian derivatives of 1/|R| up to ``order`` (<= 4) for rows R [M, 3]."""
    r2 = np.sum(R * R, axis=1)
    ir = 1.0 / np.sqrt(r2)
    ir2 = ir * ir
    ir3 = ir * ir2
    ir5 = ir3 * ir2
    out = [ir]
    if order >= 1:
        out.append(-R * ir3[:, None])
    if order >= 2:
        RR = R[:, :, None] * R[:, None, :]
        out.append(3.0 * RR * ir5[:, None, None] - _I3[None] * ir3[:, None, None])
    if order >= 3:
        ir7 = ir5 * ir2
        RRR = RR[:, :, :, None] * R[:, None, None, :]
        Rd = (R[:, :, None, None] * _I3[None, None, :, :]
              + R[:, None, :, None] * _I3[None, :, None, :]
              + R[:, None, None, :] * _I3[None, :, :, None])
        out.append(-15.0 * RRR * ir7[:, None, None, None] + 3.0 * Rd * ir5[:, None, None, None])
    if order >= 4:
        ir9 = ir7 * ir2
        RRRR = RRR[..., None] * R[:, None, None, None, :]
        d = _I3
        RRd = np.zeros_like(RRRR)
        # six placements of one delta among four indices (i j k l)
        RRd += RR[:, :, :, None, None] * d[None, None, None, :, :]      # R_i R_j d_kl
        RRd += RR[:, :, None, :, None] * d[None, None, :, None, :]      # R_i R_k d_jl
        RRd += RR[:, :, None, None, :] * d[None, None, :, :, None]      # R_i R_l d_jk
        RRd += RR[:, None, :, :, None] * d[None, :, None, None, :]      # R_j R_k d_il
        RRd += RR[:, None, :, None, :] * d[None, :, None, :, None]      # R_j R_l d_ik
        RRd += RR[:, None, None, :, :] * d[None, :, :, None, None]      # R_k R_l d_ij
        dd = (d[:, :, None, None] * d[None, None, :, :] + d[:, None, :, None] * d[None, :, None, :]
              + d[:, None, None, :] * d[None, :, :, None])
        out.append(105.0 * RRRR * ir9[:, None, None, None, None]
                   - 15.0 * RRd * ir7[:, None, None, None, None]
                   + 3.0 * dd[None] * ir5[:, None, None, None, None])
    return out


def thole_lambdas(R: np.ndarray, alpha_l: np.ndarray, alpha_m: np.ndarray, a: float):
    """Thole exponential damping factors (lambda3, lambda5, lambda7) per pair.

    The paper damps the induced-dipole field "Thole-like" without a formula;
    the reading is the AMOEBA form: u = r / (alpha_l alpha_m)^(1/6),
    lambda3 = 1 - e^{-a u^3}, lambda5 = 1 - (1 + a u^3) e^{-a u^3},
    lambda7 = 1 - (1 + a u^3 + 3/5 a^2 u^6) e^{-a u^3};  no damping when
    alpha_l alpha_m = 0.
    """
    r = np.sqrt(np.sum(R * R, axis=1))
    aa = alpha_l * alpha_m
    damp = aa > 0.0
    s = np.where(damp, aa, 1.0) ** (1.0 / 6.0)
    u3 = (r / s) ** 3
    au3 = a * u3
    e = np.where(damp, np.exp(-au3), 0.0)
    l3 = 1.0 - e
    l5 = 1.0 - (1.0 + au3) * e
    l7 = 1.0 - (1.0 + au3 + 0.6 * au3 * au3) * e
    return l3, l5, l7


def damped_tensors(R: np.ndarray, l3, l5, l7):
    """Thole-damped T1, T2, T3 (the derivatives of the smeared-charge potential)."""
    r2 = np.sum(R * R, axis=1)
    ir = 1.0 / np.sqrt(r2)
    ir3 = ir ** 3
    ir5 = ir3 * ir * ir
    ir7 = ir5 * ir * ir
    RR = R[:, :, None] * R[:, None, :]
    T1 = -(l3 * ir3)[:, None] * R
    T2 = 3.0 * (l5 * ir5)[:, None, None] * RR - (l3 * ir3)[:, None, None] * _I3[None]
    RRR = RR[:, :, :, None] * R[:, None, None, :]
    Rd = (R[:, :, None, None] * _I3[None, None, :, :] + R[:, None, :, None] * _I3[None, :, None, :]
          + R[:, None, None, :] * _I3[None, :, :, None])
    T3 = -15.0 * (l7 * ir7)[:, None, None, None] * RRR + 3.0 * (l5 * ir5)[:, None, None, None] * Rd
    return T1, T2, T3


# ----------------------------------------------------------------------------
# right-hand side
# ----------------------------------------------------------------------------

def rhs(points: np.ndarray, pos, q, p, Q, eps_in: float, chunk: int = 2048, point_body=None, site_body=None):
    """Eq. (rhs_multipole) at ``points`` [N, 3]:
    1/(4 pi eps1) sum_k [ q_k/R + p_k . R / R^3 + Q_k : R R / (2 R^5) ], R = x - r_k.
    With bodies given, a point sees only the sites of its own body (each cavity's
    interior representation holds its own charges)."""
    n = points.shape[0]
    out = np.zeros(n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        R = points[s:e, None, :] - pos[None, :, :]
        r2 = np.sum(R * R, axis=2)
        r = np.sqrt(r2)
        t = q[None, :] / r
        t = t + np.sum(p[None, :, :] * R, axis=2) / (r2 * r)
        t = t + np.einsum("mkij,mki,mkj->mk", np.broadcast_to(Q[None], (e - s,) + Q.shape), R, R) \
            / (2.0 * r2 * r2 * r)
        if point_body is not None:
            t = np.where(point_body[s:e, None] == site_body[None, :], t, 0.0)
        out[s:e] = np.sum(t, axis=1)
    return out / (FOUR_PI * eps_in)


# ----------------------------------------------------------------------------
# reaction potential and its derivatives at the sites (Eqs. pot_solvent, Efield_solv, ddphi)
# ----------------------------------------------------------------------------

def reaction_at_sites(mesh, phi: np.ndarray, psi: np.ndarray, pos: np.ndarray, chunk: int = 64,
                      site_body=None):
    """phi_solv = -K_L(phi) + V_L(psi) at the sites, with gradient and Hessian.

    Sites are far from every panel, so the panel integrals use the K-node rule:
    node g of panel j carries a charge m = w_g A_j psi_j and a dipole
    d = w_g A_j phi_j n_j, and 4 pi phi_solv = sum_g [ m T0 + d . T1 ](r - y_g).
    With several bodies a site sees only the surface of its own body.
    Returns (phi [Ns], grad [Ns, 3], hess [Ns, 3, 3]).
    """
    y = mesh.ygauss.reshape(-1, 3)
    k = mesh.ygauss.shape[1]
    m = (mesh.wgauss * psi[:, None]).reshape(-1)
    d = ((mesh.wgauss * phi[:, None])[:, :, None] * mesh.normal[:, None, :]).reshape(-1, 3)
    node_body = np.repeat(mesh.body, k)
    ns = pos.shape[0]
    pot = np.zeros(ns)
    grad = np.zeros((ns, 3))
    hess = np.zeros((ns, 3, 3))
    for s in range(0, ns, chunk):
        e = min(ns, s + chunk)
        for l in range(s, e):
            sel = slice(None) if site_body is None else (node_body == site_body[l])
            R = pos[l][None, :] - y[sel]
            T0, T1, T2, T3 = t_tensors(R, 3)
            ml, dl = m[sel], d[sel]
            pot[l] = np.sum(ml * T0) + np.sum(dl * T1)
            grad[l] = ml @ T1 + np.einsum("gi,gik->k", dl, T2)
            hess[l] = np.einsum("g,gkl->kl", ml, T2) + np.einsum("gi,gikl->kl", dl, T3)
    return pot / FOUR_PI, grad / FOUR_PI, hess / FOUR_PI


# ----------------------------------------------------------------------------
# multipole-multipole potentials and fields (Eqs. Efield_mult, second_derivative)
# ----------------------------------------------------------------------------

def _pairs(pos, body):
    ns = pos.shape[0]
    li, mi = np.nonzero(~np.eye(ns, dtype=bool))
    return li, mi


def mult_potentials(pos, q, d, Q, mu, alpha, group, body, eps_in, thole_a,
                    masked: bool, same_body_only: bool, damp_permanent: bool = False):
    """Potential, gradient and Hessian at every site from all OTHER sites.

    Permanent moments (q, d, Q) are undamped; when ``masked`` the permanent
    contribution of a site in the same polarisation group is dropped (the
    field that polarises, Sec. "Calculation of the electric field"); in the
    energy they are unmasked.  Induced dipoles mu are Thole-damped.  With
    ``same_body_only`` sites of other bodies are ignored (dissolved state of a
    multi-body system: bodies talk only through the solvent).
    ``damp_permanent`` (the AMOEBA rule, not the paper's): the gradient of the
    permanent moments is taken with the Thole-damped tensors too (the charge's
    1/r^3 term with lambda3, the dipole's with lambda3 and lambda5, the
    quadrupole's with lambda5 and lambda7); it applies to the polarising field
    only, so it requires ``masked``, and the potential and Hessian stay undamped.
    Returns (phi [Ns], grad [Ns, 3], hess [Ns, 3, 3]).
    """
    if damp_permanent and not masked:
        raise ValueError("damp_permanent applies to the polarising (masked) field only")
    ns = pos.shape[0]
    li, mi = _pairs(pos, body)
    if same_body_only:
        keep = body[li] == body[mi]
        li, mi = li[keep], mi[keep]
    R = pos[li] - pos[mi]
    T0, T1, T2, T3, T4 = t_tensors(R, 4)
    perm = np.ones(li.size)
    if masked:
        perm = (group[li] != group[mi]).astype(np.float64)
    qm, dm, Qm = q[mi], d[mi], Q[mi]
    pot = perm * (qm * T0 - np.sum(dm * T1, axis=1) + np.einsum("pij,pij->p", Qm, T2) / 6.0)
    grad = perm[:, None] * (qm[:, None] * T1 - np.einsum("pi,pik->pk", dm, T2)
                            + np.einsum("pij,pijk->pk", Qm, T3) / 6.0)
    hess = perm[:, None, None] * (qm[:, None, None] * T2 - np.einsum("pi,pikl->pkl", dm, T3)
                                  + np.einsum("pij,pijkl->pkl", Qm, T4) / 6.0)
    l3, l5, l7 = thole_lambdas(R, alpha[li], alpha[mi], thole_a)
    D1, D2, D3 = damped_tensors(R, l3, l5, l7)
    if damp_permanent:
        grad = perm[:, None] * (qm[:, None] * D1 - np.einsum("pi,pik->pk", dm, D2)
                                + np.einsum("pij,pijk->pk", Qm, D3) / 6.0)
    mm = mu[mi]
    pot = pot - np.sum(mm * D1, axis=1)
    grad = grad - np.einsum("pi,pik->pk", mm, D2)
    hess = hess - np.einsum("pi,pikl->pkl", mm, D3)
    P = np.zeros(ns)
    Gd = np.zeros((ns, 3))
    H = np.zeros((ns, 3, 3))
    np.add.at(P, li, pot)
    np.add.at(Gd, li, grad)
    np.add.at(H, li, hess)
    s = 1.0 / (FOUR_PI * eps_in)
    return P * s, Gd * s, H * s


def thole_matrix(pos, alpha, body, eps_in, thole_a, same_body_only: bool):
    """[3Ns, 3Ns] matrix T with E_induced = T mu (damped dipole field of the other sites)."""
    ns = pos.shape[0]
    li, mi = _pairs(pos, body)
    if same_body_only:
        keep = body[li] == body[mi]
        li, mi = li[keep], mi[keep]
    R = pos[li] - pos[mi]
    l3, l5, l7 = thole_lambdas(R, alpha[li], alpha[mi], thole_a)
    _, D2, _ = damped_tensors(R, l3, l5, l7)
    T = np.zeros((ns, 3, ns, 3))
    T[li, :, mi, :] = D2 / (FOUR_PI * eps_in)
    return T.reshape(3 * ns, 3 * ns)


def site_energy(q, d, Q, pot, grad, hess):
    """Eq. (energy_multipole_polarizable): 1/2 sum [q phi + d . grad phi + (1/6) Q : hess phi]."""
    return 0.5 * (np.sum(q * pot) + np.sum(d * grad) + np.einsum("mij,mij->", Q, hess) / 6.0)


# ----------------------------------------------------------------------------
# self-consistent induced dipoles and the solvation energy
# ----------------------------------------------------------------------------

@dataclass
class SolvationResult:
    dG_kcal: float
    G_diss: float
    G_vac: float
    mu_diss: np.ndarray
    mu_vac: np.ndarray
    phi: np.ndarray
    psi: np.ndarray
    react_pot: np.ndarray
    react_grad: np.ndarray
    react_hess: np.ndarray
    scf_iters_diss: int
    scf_iters_vac: int
    rhs: np.ndarray


def _damp_perm(par) -> bool:
    """Whether the permanent moments' polarising field is Thole-damped (an AMOEBA rule the
    paper does not state; off unless the parameters ask for it)."""
    return bool(getattr(par, "damp_permanent", False))


def _rms(x):
    return float(np.sqrt(np.sum(x * x) / max(1, x.shape[0])))


def vacuum_scf(sites, par, direct: bool = False):
    """Induced dipoles in vacuum (homogeneous eps1, no surface) by SOR or a direct solve."""
    ns = sites.n
    four_pi_alpha = FOUR_PI * sites.alpha
    _, gperm, _ = mult_potentials(sites.pos, sites.q, sites.d, sites.Q, np.zeros((ns, 3)), sites.alpha,
                                  sites.group, sites.body, par.eps_in, par.thole_a, masked=True,
                                  same_body_only=False, damp_permanent=_damp_perm(par))
    Eperm = -gperm
    if direct:
        T = thole_matrix(sites.pos, sites.alpha, sites.body, par.eps_in, par.thole_a, False)
        A = np.eye(3 * ns) - np.repeat(four_pi_alpha, 3)[:, None] * T
        mu = np.linalg.solve(A, (four_pi_alpha[:, None] * Eperm).reshape(-1)).reshape(ns, 3)
        return mu, 0
    mu = np.zeros((ns, 3))
    it = 0
    for it in range(1, par.scf_maxit + 1):
        _, g, _ = mult_potentials(sites.pos, np.zeros(ns), np.zeros((ns, 3)), np.zeros((ns, 3, 3)), mu,
                                  sites.alpha, sites.group, sites.body, par.eps_in, par.thole_a,
                                  masked=True, same_body_only=False)
        E = Eperm - g
        new = (1.0 - par.sor_omega) * mu + par.sor_omega * four_pi_alpha[:, None] * E
        delta = _rms(new - mu)
        mu = new
        if delta < par.scf_tol:
            break
    return mu, it


def solvation(problem, solver=None, direct_polarization: bool = False) -> SolvationResult:
    """Delta G_solv = G_diss - G_vac (Eqs. deltaG_aux2, energy_multipole_polarizable).

    Dissolved state, following the self-consistent scheme of Sec.
    "Self-consistent induced field": mu = 0; repeat { solve Eq. (integral_eq)
    with p = d + mu; E = E_solv + E_mult; mu <- (1 - w) mu + w 4 pi alpha E }
    until the RMS change is below ``scf_tol``; then one last solve with the
    converged mu gives phi_solv and its derivatives for the energy.
    With ``direct_polarization`` the fixed point mu = 4 pi alpha E(mu) is solved
    directly as one 3Ns linear system instead.
    """
    from . import bem

    par = problem.params
    sites = problem.sites
    ns = sites.n
    if solver is None:
        mesh = bem.build_mesh(problem.verts, problem.tris, par.gauss_k, par.near_factor,
                              near_rule=getattr(par, "near_rule", "exact"),
                              body=getattr(problem, "panel_body", None))
        solver = bem.DenseSolver(mesh, par.eps_in, par.eps_out, par.kappa)
        solver.mesh = mesh
    mesh = solver.mesh
    n = mesh.n
    four_pi_alpha = FOUR_PI * sites.alpha

    def bem_solve(p):
        b = np.zeros(2 * n)
        b[:n] = rhs(mesh.cen, sites.pos, sites.q, p, sites.Q, par.eps_in, point_body=mesh.body,
                    site_body=sites.body)
        return solver.solve(b), b

    _, gperm, _ = mult_potentials(sites.pos, sites.q, sites.d, sites.Q, np.zeros((ns, 3)), sites.alpha,
                                  sites.group, sites.body, par.eps_in, par.thole_a, masked=True,
                                  same_body_only=True, damp_permanent=_damp_perm(par))
    Eperm = -gperm

    def E_induced(mu):
        _, g, _ = mult_potentials(sites.pos, np.zeros(ns), np.zeros((ns, 3)), np.zeros((ns, 3, 3)), mu,
                                  sites.alpha, sites.group, sites.body, par.eps_in, par.thole_a,
                                  masked=True, same_body_only=True)
        return -g

    if direct_polarization:
        # E_solv is affine in p: E_solv(d + mu) = E_solv(d) + M mu
        x0, _ = bem_solve(sites.d)
        _, g0, _ = reaction_at_sites(mesh, x0[:n], x0[n:], sites.pos, site_body=sites.body)
        M = np.zeros((3 * ns, 3 * ns))
        for m in range(ns):
            for c in range(3):
                p = np.zeros((ns, 3))
                p[m, c] = 1.0
                b = np.zeros(2 * n)
                b[:n] = rhs(mesh.cen, sites.pos, np.zeros(ns), p, np.zeros((ns, 3, 3)), par.eps_in,
                            point_body=mesh.body, site_body=sites.body)
                xx = solver.solve(b)
                _, gg, _ = reaction_at_sites(mesh, xx[:n], xx[n:], sites.pos, site_body=sites.body)
                M[:, 3 * m + c] = -gg.reshape(-1)
        T = thole_matrix(sites.pos, sites.alpha, sites.body, par.eps_in, par.thole_a, True)
        A = np.eye(3 * ns) - np.repeat(four_pi_alpha, 3)[:, None] * (M + T)
        b = (four_pi_alpha[:, None] * (Eperm - g0)).reshape(-1)
        mu = np.linalg.solve(A, b).reshape(ns, 3)
        it = 0
    else:
        mu = np.zeros((ns, 3))
        it = 0
        for it in range(1, par.scf_maxit + 1):
            x, _ = bem_solve(sites.d + mu)
            _, g, _ = reaction_at_sites(mesh, x[:n], x[n:], sites.pos, site_body=sites.body)
            E = -g + Eperm + E_induced(mu)
            new = (1.0 - par.sor_omega) * mu + par.sor_omega * four_pi_alpha[:, None] * E
            delta = _rms(new - mu)
            mu = new
            if delta < par.scf_tol:
                break

    x, b = bem_solve(sites.d + mu)
    rp, rg, rh = reaction_at_sites(mesh, x[:n], x[n:], sites.pos, site_body=sites.body)
    mp, mg, mh = mult_potentials(sites.pos, sites.q, sites.d, sites.Q, mu, sites.alpha, sites.group,
                                 sites.body, par.eps_in, par.thole_a, masked=False, same_body_only=True)
    G_diss = site_energy(sites.q, sites.d, sites.Q, rp + mp, rg + mg, rh + mh)

    mu_v, it_v = vacuum_scf(sites, par, direct=direct_polarization)
    vp, vg, vh = mult_potentials(sites.pos, sites.q, sites.d, sites.Q, mu_v, sites.alpha, sites.group,
                                 sites.body, par.eps_in, par.thole_a, masked=False, same_body_only=False)
    G_vac = site_energy(sites.q, sites.d, sites.Q, vp, vg, vh)
    return SolvationResult(
        dG_kcal=(G_diss - G_vac) * KCAL_PER_UNIT, G_diss=G_diss, G_vac=G_vac, mu_diss=mu, mu_vac=mu_v,
        phi=x[:n], psi=x[n:], react_pot=rp, react_grad=rg, react_hess=rh, scf_iters_diss=it,
        scf_iters_vac=it_v, rhs=b[:n])
