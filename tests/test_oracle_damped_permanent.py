"""The oracle's damped permanent field (an AMOEBA rule the paper does not state; §8(f) 4).

Two sites on the x axis, r apart, both polarizable, in vacuum: a permanent charge q (or a
dipole p along x) at the origin and a bare polarizable site at (r, 0, 0).  With the Thole
factors lambda3, lambda5 of the pair the fixed point mu = 4 pi alpha E has the closed form
    mu_l = 4 pi alpha_l (E_perm + k mu_m),   mu_m = 4 pi alpha_m k mu_l,
    k = (3 lambda5 - lambda3) / (4 pi eps r^3)   (damped dipole-dipole coupling along the axis),
where E_perm = lambda3 q / (4 pi eps r^2) for the charge, (3 lambda5 - lambda3) p /
(4 pi eps r^3) for the dipole and (5 lambda7 - 2 lambda5) Q0 / (4 pi eps r^4) for the linear
quadrupole Q0 diag(2, -1, -1) (Q = int rho (3 r r - r^2 I)) when the permanent field is damped,
and the same with lambda = 1 (r^-2, 2 p r^-3, 3 Q0 r^-4) when it is not.  The damping factors come from Thole's exponential smearing (pinned by Gauss's
law in test_oracle_multipole.py); this pins which damped tensor multiplies which moment in the
polarising field, and that the energy terms stay undamped.
"""
import numpy as np
import pytest

from gen.sites import Sites
from oracle import multipole as mp

FOUR_PI = 4.0 * np.pi


class _P:
    eps_in, thole_a, scf_tol, scf_maxit, sor_omega = 2.0, 0.39, 1e-15, 2000, 0.7


def _lams(r, al, am, a):
    au3 = a * r ** 3 / np.sqrt(al * am)
    e = np.exp(-au3)
    return 1.0 - e, 1.0 - (1.0 + au3) * e, 1.0 - (1.0 + au3 + 0.6 * au3 * au3) * e


def _pair(r, al, am, q=0.0, p=0.0, q0=0.0):
    Q = np.zeros((2, 3, 3))
    Q[0] = q0 * np.diag([2.0, -1.0, -1.0])
    return Sites(pos=np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]), q=np.array([q, 0.0]),
                 d=np.array([[p, 0.0, 0.0], [0.0, 0.0, 0.0]]), Q=Q, alpha=np.array([am, al]))


@pytest.mark.parametrize("kind", ["charge", "dipole", "quadrupole"])
@pytest.mark.parametrize("damp", [True, False])
def test_two_site_closed_form(kind, damp):
    par = _P()
    par.damp_permanent = damp
    r, al, am = 1.3, 1.1, 0.6
    q, p, q0 = {"charge": (1.0, 0.0, 0.0), "dipole": (0.0, 0.8, 0.0), "quadrupole": (0.0, 0.0, 0.7)}[kind]
    st = _pair(r, al, am, q=q, p=p, q0=q0)
    l3, l5, l7 = _lams(r, al, am, par.thole_a)
    eps = par.eps_in
    k = (3.0 * l5 - l3) / (FOUR_PI * eps * r ** 3)
    if kind == "charge":
        e_perm = (l3 if damp else 1.0) * q / (FOUR_PI * eps * r ** 2)
    elif kind == "dipole":
        e_perm = ((3.0 * l5 - l3) if damp else 2.0) * p / (FOUR_PI * eps * r ** 3)
    else:
        e_perm = ((5.0 * l7 - 2.0 * l5) if damp else 3.0) * q0 / (FOUR_PI * eps * r ** 4)
    mu_l = FOUR_PI * al * e_perm / (1.0 - (FOUR_PI ** 2) * al * am * k * k)
    mu_m = FOUR_PI * am * k * mu_l
    for direct in (True, False):
        mu, _ = mp.vacuum_scf(st, par, direct=direct)
        assert np.allclose(mu[1], [mu_l, 0.0, 0.0], rtol=1e-11, atol=1e-13), (direct, mu, mu_l)
        assert np.allclose(mu[0], [mu_m, 0.0, 0.0], rtol=1e-11, atol=1e-13), (direct, mu, mu_m)
    # damping matters at this separation (u^3 ~ 2.7): the two readings differ
    assert abs(l3 - 1.0) > 1e-3


def test_no_smearing_limit_and_energy_terms_undamped():
    """a -> infinity: the smeared charge shrinks to a point (every lambda -> 1), so the damped
    permanent field equals the undamped one; at a = 0.39 they differ; the energy-form
    (unmasked) potentials never take the damping."""
    rng = np.random.default_rng(4)
    n = 6
    pos = rng.normal(size=(n, 3)) * 2.0
    q = rng.uniform(-1, 1, n)
    d = rng.normal(0, 0.3, (n, 3))
    Q = rng.normal(0, 0.2, (n, 3, 3))
    Q = Q + Q.transpose(0, 2, 1)
    Q -= np.trace(Q, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3.0
    alpha = rng.uniform(0.5, 1.5, n)
    group = np.arange(n)
    body = np.zeros(n, dtype=np.int32)
    z = np.zeros((n, 3))
    a = mp.mult_potentials(pos, q, d, Q, z, alpha, group, body, 1.0, 1e6, True, False, damp_permanent=True)
    b = mp.mult_potentials(pos, q, d, Q, z, alpha, group, body, 1.0, 1e6, True, False, damp_permanent=False)
    assert np.allclose(a[1], b[1], rtol=1e-9, atol=1e-12)
    c = mp.mult_potentials(pos, q, d, Q, z, alpha, group, body, 1.0, 0.39, True, False, damp_permanent=True)
    assert np.max(np.abs(c[1] - b[1])) > 1e-3 * np.max(np.abs(b[1]))
    with pytest.raises(ValueError):
        mp.mult_potentials(pos, q, d, Q, z, alpha, group, body, 1.0, 0.39, False, False, damp_permanent=True)
