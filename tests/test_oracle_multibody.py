"""Pins of the oracle's several-body solvent (Sec. "Calculation of the binding energy").

In the complex AB each body keeps its own interior (Laplace) representation --
its own sites and its own surface -- while the solvent (Yukawa) rows see every
surface.  The pins:

* two Born ions far apart: the screened interaction in the dissolved state is the
  Debye-Hueckel pair energy q_A q_B e^{k(a_A+a_B)} e^{-k d} / (4 pi eps2 (1+k a_A)(1+k a_B) d),
  up to the cavities' re-scattering of each other's field, of relative order
  (a_A^3 + a_B^3) / d^3;
* in vacuum all sites interact: the pair energy is q_A q_B / (4 pi eps1 d) exactly;
* bodies very far apart decouple: G_diss(AB) = G_diss(A) + G_diss(B);
* the Laplace blocks of AB are block diagonal and equal those of each body alone.
"""
import numpy as np
import pytest

import gen
from oracle import bem
from oracle import multipole as mp


def _ion(radius, subdiv, q):
    v, f = gen.icosphere(radius, subdiv)
    s = gen.Sites(pos=np.zeros((1, 3)), q=np.array([q]), d=np.zeros((1, 3)), Q=np.zeros((1, 3, 3)),
                  alpha=np.zeros(1))
    return gen.Problem(f"ion_r{radius:g}", v, f, s, gen.Params())


def _pair(a, b, d):
    """AB with B's centre at distance d along x (both generated at the origin)."""
    ab = gen.two_body(a, b, gap=0.0)
    off = np.array([d, 0.0, 0.0])
    ab.verts[a.verts.shape[0]:] = b.verts + off
    ab.sites.pos[a.sites.n:] = b.sites.pos + off
    return ab


def _dh_pair(qa, qb, ra, rb, d, p):
    k = p.kappa
    return qa * qb * np.exp(k * (ra + rb)) * np.exp(-k * d) / (
        4.0 * np.pi * p.eps_out * (1.0 + k * ra) * (1.0 + k * rb) * d)


def _binding_parts(a, b, ab):
    ra, rb, rab = mp.solvation(a), mp.solvation(b), mp.solvation(ab)
    return rab.G_diss - ra.G_diss - rb.G_diss, rab.G_vac - ra.G_vac - rb.G_vac


def test_two_born_ions_screened_interaction():
    qa, qb, ra_, rb_ = 1.0, -0.7, 4.0, 3.0
    a, b = _ion(ra_, 2, qa), _ion(rb_, 2, qb)
    dev = []
    for d in (12.0, 16.0, 24.0):
        diss, vac = _binding_parts(a, b, _pair(a, b, d))
        ex = _dh_pair(qa, qb, ra_, rb_, d, a.params)
        rel = abs(diss / ex - 1.0)
        assert rel < (ra_ ** 3 + rb_ ** 3) / d ** 3, (d, diss, ex)
        dev.append(rel)
        # vacuum: the bare Coulomb pair energy, exactly
        assert vac == pytest.approx(qa * qb / (4.0 * np.pi * a.params.eps_in * d), rel=1e-12)
    assert dev[0] > dev[1] > dev[2]


def test_planted_cross_body_laplace_fails_the_pin():
    """A Laplace representation that also integrates over the other body's surface
    (every panel tagged body 0) must miss the screened pair energy by far."""
    qa, qb, d = 1.0, -0.7, 16.0
    a, b = _ion(4.0, 2, qa), _ion(3.0, 2, qb)
    ab = _pair(a, b, d)
    ab.panel_body = np.zeros(ab.n_panels, np.int32)
    diss, _ = _binding_parts(a, b, ab)
    ex = _dh_pair(qa, qb, 4.0, 3.0, d, a.params)
    assert abs(diss / ex - 1.0) > 10.0


def test_far_apart_bodies_decouple():
    a, b, ab = gen.small_triple(gap=200.0)
    ra = mp.solvation(a, direct_polarization=True)
    rb = mp.solvation(b, direct_polarization=True)
    rab = mp.solvation(ab, direct_polarization=True)
    # the Yukawa coupling across 200 A is below e^{-25}
    assert rab.G_diss == pytest.approx(ra.G_diss + rb.G_diss, rel=1e-10)
    na = a.sites.n
    assert np.allclose(rab.mu_diss[:na], ra.mu_diss, rtol=0, atol=1e-10)
    assert np.allclose(rab.mu_diss[na:], rb.mu_diss, rtol=0, atol=1e-10)
    # vacuum: the bodies still interact through the bare Coulomb field
    assert abs(rab.G_vac - ra.G_vac - rb.G_vac) > 1e-6


def test_laplace_blocks_are_per_body():
    a, b, ab = gen.small_triple()
    p = a.params
    ma = bem.build_mesh(a.verts, a.tris, p.gauss_k, p.near_factor)
    mab = bem.build_mesh(ab.verts, ab.tris, p.gauss_k, p.near_factor, body=ab.panel_body)
    VLa, KLa, VYa, KYa = bem.assemble_layers(ma, p.kappa)
    VL, KL, VY, KY = bem.assemble_layers(mab, p.kappa)
    na = a.n_panels
    assert np.array_equal(VL[:na, :na], VLa) and np.array_equal(KL[:na, :na], KLa)
    assert np.array_equal(VY[:na, :na], VYa) and np.array_equal(KY[:na, :na], KYa)
    assert not VL[:na, na:].any() and not KL[na:, :na].any()
    assert np.all(VY[:na, na:] > 0.0) and np.abs(KY[na:, :na]).max() > 0.0
    # the rows skip nothing else: matvec_rows agrees with the dense matrix
    A = bem.system_matrix((VL, KL, VY, KY), p.eps_in, p.eps_out)
    x = np.random.default_rng(5).normal(size=2 * mab.n)
    rows = np.array([0, na - 1, na, mab.n - 1])
    y1, y2 = bem.matvec_rows(mab, x, rows, p.eps_in, p.eps_out, p.kappa)
    y = A @ x
    assert np.allclose(y1, y[rows], rtol=1e-13, atol=1e-13)
    assert np.allclose(y2, y[mab.n + rows], rtol=1e-13, atol=1e-13)
