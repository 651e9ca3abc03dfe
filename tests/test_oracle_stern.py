"""Pins for the three-region (Stern layer) oracle of ``oracle/stern.py``.

The dense two-surface solution must converge at the panel-area rate to the closed-form
sphere with an ion-exclusion layer (``kirkwood`` with b), land on it under Richardson
extrapolation, and stay clear of the closed form without the layer; the normal flux
through both surfaces must obey Gauss's law (-Q/eps1 through the dielectric boundary,
-Q/eps2 through the ion-exclusion surface).  Sec. "Spherical cavity" (R = 4 with a 1 A
Stern layer) sets the geometry.
"""
import numpy as np
import pytest

import gen
from oracle import kirkwood as kw, multipole as mp, stern


def _solve(sites, params, sub, a=4.0, b=5.0):
    v1, f1 = gen.icosphere(a, sub)
    v2, f2 = gen.icosphere(b, sub)
    S = stern.stern_solver(v1, f1, v2, f2, params)
    r = mp.solvation(gen.Problem("stern", v1, f1, sites, params), solver=S, direct_polarization=True)
    return S, r


@pytest.mark.slow
def test_stern_bem_converges_to_closed_form():
    pr = gen.sphere_random(4.0, 2, 5, 2.2, 1.2, 11)
    par = gen.with_params(pr, kappa=1.0, eps_in=4.0).params
    exact, _, _ = kw.solvation(pr.sites, 4.0, par.eps_in, par.eps_out, par.kappa, par.thole_a, b=5.0)
    no_layer, _, _ = kw.solvation(pr.sites, 4.0, par.eps_in, par.eps_out, par.kappa, par.thole_a)
    assert abs(no_layer - exact) > 5e-3 * abs(exact)  # the layer matters at this salt level
    vals = [_solve(pr.sites, par, s)[1].dG_kcal for s in (2, 3)]
    e = np.abs(np.array(vals) - exact)
    assert 3.5 < e[0] / e[1] < 4.5
    rich = vals[1] + (vals[1] - vals[0]) / 3.0
    assert abs(rich - exact) < 1e-3 * abs(exact)
    assert abs(rich - no_layer) > 5e-3 * abs(no_layer)


def test_stern_gauss_law():
    pr = gen.sphere_r4_1280()
    par = pr.params
    S, r = _solve(pr.sites, par, 2)
    x = S.solve_full(r.rhs)
    n1, n2 = S.mesh.n, S.mesh2.n
    psi1 = x[n1:2 * n1]
    psi2 = x[2 * n1 + n2:]
    Q = float(np.sum(pr.sites.q))
    assert psi1 @ S.mesh.area == pytest.approx(-Q / par.eps_in, rel=5e-3)
    assert psi2 @ S.mesh2.area == pytest.approx(-Q / par.eps_out, rel=5e-3)
