"""Pins of the oracle gradient dDelta G_solv / d(r, q, d, Q) (``oracle/gradient.py``).

* Euler: Delta G_solv is a homogeneous quadratic form in the permanent moments
  (the induced dipoles are linear in them), so
  sum_l q_l g_q + d_l . g_d + Q_l : g_Q = 2 Delta G_solv exactly.
* Kirkwood: in a dielectric sphere the exact Delta G_solv of polarizable point
  multipoles is known in closed form (``oracle/kirkwood.py``); its derivatives
  (five-point differences of the closed form) are the continuum gradient.  The
  BEM gradient must approach it at the rate of the method, O(mean panel area):
  about 4x closer per icosphere subdivision.
* A quadratic form has an exact five-point derivative: moment derivatives do
  not depend on the step.
"""
import numpy as np
import pytest

import gen
from oracle import gradient as og
from oracle import kirkwood as kw
from oracle import multipole as mp


def _sphere_problem(subdiv):
    v, f = gen.icosphere(4.0, subdiv)
    Q = np.array([[0.3, 0.1, 0.0], [0.1, -0.1, 0.05], [0.0, 0.05, -0.2]])
    s = gen.Sites(pos=np.array([[0.2, -0.3, 0.1], [1.5, 0.4, -0.2]]), q=np.array([1.0, -0.5]),
                  d=np.array([[0.0, 0.0, 0.5], [0.2, -0.1, 0.0]]), Q=np.stack([Q, -Q]), alpha=np.array([0.0, 1.0]))
    return gen.Problem(f"sphere_sub{subdiv}", v, f, s, gen.Params())


def _kirkwood_gradient(pr):
    """Five-point derivatives of the closed-form Delta G_solv (paper units)."""
    p = pr.params
    base = pr.sites

    def G(s):
        return kw.solvation(s, 4.0, p.eps_in, p.eps_out, p.kappa, p.thole_a)[0] / mp.KCAL_PER_UNIT

    out = {"pos": np.zeros((base.n, 3)), "q": np.zeros(base.n), "d": np.zeros((base.n, 3)),
           "Q": np.zeros((base.n, 3, 3))}

    def along(field, l, comps, h):
        def f(t):
            s = og._copy_sites(base)
            arr = getattr(s, field)
            for c in comps:
                arr[(l,) + c] += t
            return G(s)
        return og.five_point(f, h)

    for l in range(base.n):
        out["q"][l] = along("q", l, [()], 1e-2)
        for a in range(3):
            out["pos"][l, a] = along("pos", l, [(a,)], 1e-3)
            out["d"][l, a] = along("d", l, [(a,)], 1e-2)
            out["Q"][l, a, a] = along("Q", l, [(a, a)], 1e-2)
            for b in range(a + 1, 3):
                out["Q"][l, a, b] = out["Q"][l, b, a] = 0.5 * along("Q", l, [(a, b), (b, a)], 1e-2)
        out["Q"][l] -= np.trace(out["Q"][l]) / 3.0 * np.eye(3)
    return out


def _euler(pr, g):
    s = pr.sites
    return np.sum(s.q * g["q"]) + np.sum(s.d * g["d"]) + np.sum(s.Q * g["Q"])


def test_euler_identity_polarizable_bumpy():
    pr = gen.small_bumpy(2, 6, 8.0, seed_index=105)
    g = og.solvation_gradient(pr)
    assert _euler(pr, g) == pytest.approx(2.0 * g["dG"], rel=1e-10)


def test_moment_derivatives_do_not_depend_on_the_step():
    pr = gen.small_bumpy(2, 3, 8.0, seed_index=106)
    solver = og._dense_solver(pr)
    a = og.solvation_gradient(pr, sites_idx=[1], h_mom=1e-2, solver=solver)
    b = og.solvation_gradient(pr, sites_idx=[1], h_mom=3e-1, solver=solver)
    for k in ("q", "d", "Q"):
        assert np.allclose(a[k], b[k], rtol=1e-9, atol=1e-12 * np.max(np.abs(a[k]))), k


@pytest.mark.slow
def test_gradient_converges_to_kirkwood():
    ref = _kirkwood_gradient(_sphere_problem(2))
    err = {}
    for sub in (2, 3):
        g = og.solvation_gradient(_sphere_problem(sub))
        err[sub] = {k: np.max(np.abs(g[k] - ref[k])) / np.max(np.abs(ref[k])) for k in ("pos", "q", "d", "Q")}
    for k in ("pos", "q", "d", "Q"):
        # O(A): the mean panel area falls 4x per subdivision
        assert err[3][k] < err[2][k] / 3.0, (k, err)
        assert err[3][k] < 0.02, (k, err)
