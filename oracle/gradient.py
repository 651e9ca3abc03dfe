"""Derivatives of Delta G_solv with respect to the site parameters, by differences.

The gradient dDelta G_solv / d(r_l, q_l, d_l, Q_l) of the discrete method is, by
definition, the derivative of the oracle's Delta G_solv (``multipole.solvation``)
with the mesh held fixed.  This module evaluates that definition with the
five-point central difference

    f'(x) ~ [8 (f(x + h) - f(x - h)) - (f(x + 2h) - f(x - 2h))] / (12 h),

whose truncation error is h^4 f^(5) / 30, with every Delta G_solv taken at the
exact fixed point of the induced dipoles (``direct_polarization``: one dense
3 Ns solve) and the exact BEM solution (LU factors of the dense system), so no
iteration tolerance enters the differences.  Quadrupoles are symmetric and
traceless (Eq. pot_multipole), so their gradient G_Q is defined on that space:
the symmetric traceless matrix with dDelta G = G_Q : dQ for every symmetric
traceless dQ.  It is assembled from derivatives along Q_aa (alone) and along the
pair (Q_ab, Q_ba) (half the derivative), then projected, G_Q - tr(G_Q) I / 3 (a
trace added to Q is not a quadrupole: the right-hand side of Eq. rhs_multipole
would see it as an extra 1/r^3 term).

Pins (tests): Euler's identity for the moments -- Delta G_solv is a homogeneous
quadratic form in the permanent moments (q, d, Q), induced dipoles included, so
sum_l (q_l dG/dq_l + d_l . dG/dd_l + Q_l : dG/dQ_l) = 2 Delta G_solv; and the
closed-form (Kirkwood) position derivative of one charge in a dielectric sphere.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import bem
from . import multipole as mp


def _dense_solver(problem):
    par = problem.params
    mesh = bem.build_mesh(problem.verts, problem.tris, par.gauss_k, par.near_factor,
                          near_rule=getattr(par, "near_rule", "exact"),
                          body=getattr(problem, "panel_body", None))
    solver = bem.DenseSolver(mesh, par.eps_in, par.eps_out, par.kappa)
    solver.mesh = mesh
    return solver


def _dG(problem, solver, sites):
    """Delta G_solv (paper units) with modified sites."""
    r = mp.solvation(replace(problem, sites=sites), solver=solver, direct_polarization=True)
    return r.G_diss - r.G_vac


def _copy_sites(s):
    return replace(s, pos=s.pos.copy(), q=s.q.copy(), d=s.d.copy(), Q=s.Q.copy())


def five_point(f, h):
    return (8.0 * (f(h) - f(-h)) - (f(2.0 * h) - f(-2.0 * h))) / (12.0 * h)


def solvation_gradient(problem, sites_idx=None, h_pos=1e-3, h_mom=1e-2, solver=None):
    """Gradient of Delta G_solv (paper units, e^2/A) for the sites ``sites_idx``
    (default all): dict with ``pos`` [m, 3], ``q`` [m], ``d`` [m, 3], ``Q`` [m, 3, 3]
    and ``dG`` (the unperturbed value)."""
    solver = solver or _dense_solver(problem)
    base = problem.sites
    idx = np.arange(base.n) if sites_idx is None else np.asarray(sites_idx)
    m = idx.size
    out = {"pos": np.zeros((m, 3)), "q": np.zeros(m), "d": np.zeros((m, 3)), "Q": np.zeros((m, 3, 3)),
           "dG": _dG(problem, solver, base)}

    def along(field, l, comps, h):
        def f(t):
            s = _copy_sites(base)
            arr = getattr(s, field)
            for comp in comps:
                arr[(l,) + comp] += t
            return _dG(problem, solver, s)
        return five_point(f, h)

    for k, l in enumerate(idx):
        out["q"][k] = along("q", l, [()], h_mom)
        for a in range(3):
            out["pos"][k, a] = along("pos", l, [(a,)], h_pos)
            out["d"][k, a] = along("d", l, [(a,)], h_mom)
            out["Q"][k, a, a] = along("Q", l, [(a, a)], h_mom)
            for b in range(a + 1, 3):
                v = 0.5 * along("Q", l, [(a, b), (b, a)], h_mom)
                out["Q"][k, a, b] = out["Q"][k, b, a] = v
        out["Q"][k] -= np.trace(out["Q"][k]) / 3.0 * np.eye(3)
    return out
