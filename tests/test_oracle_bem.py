"""Checks of the oracle's dense BEM system (Eq. integral_eq) beyond the sphere pins.

* Row sums of the assembled double layer approach -1/2 (the solid-angle identity
  holds exactly for accurate integrals; only the far K-node rule perturbs it).
* The sampled-row matvec used at large sizes reproduces the dense product.
* The system is second kind and well conditioned.
"""
import numpy as np

import gen
from oracle import bem


def test_double_layer_row_sums_approach_minus_half():
    errs = []
    for sub in (2, 3):
        v, f = gen.icosphere(4.0, sub)
        mesh = bem.build_mesh(v, f, 4, 2.0)
        VL, KL, VY, KY = bem.assemble_layers(mesh, 0.125)
        errs.append(np.max(np.abs(KL.sum(axis=1) + 0.5)))
    # the far rule's error near the threshold shrinks only like the panel size
    assert errs[0] < 5e-4 and errs[1] < errs[0]


def test_matvec_rows_equal_dense_product():
    pr = gen.small_bumpy(2, 4, 6.0)
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    rng = np.random.default_rng(0)
    x = rng.normal(size=2 * mesh.n)
    y = A @ x
    rows = np.array([0, 7, mesh.n - 1])
    y1, y2 = bem.matvec_rows(mesh, x, rows, par.eps_in, par.eps_out, par.kappa)
    assert np.allclose(y1, y[rows], rtol=1e-13, atol=1e-13)
    assert np.allclose(y2, y[mesh.n + rows], rtol=1e-13, atol=1e-13)


def test_system_is_well_conditioned():
    v, f = gen.icosphere(4.0, 2)
    mesh = bem.build_mesh(v, f, 4, 2.0)
    A = bem.system_matrix(bem.assemble_layers(mesh, 0.125), 1.0, 80.0)
    assert np.linalg.cond(A) < 1e3
