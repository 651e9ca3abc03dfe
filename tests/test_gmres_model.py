"""The Arnoldi variant of the CUDA GMRES, modelled in numpy on the oracle's dense BEM matrix.

The device GMRES runs classical Gram-Schmidt twice per step (CGS2) and takes the new
vector's norm from |w'|^2 - sum_k h2_k^2 (Pythagoras, with h2 = V^T w' from the second
pass) instead of a third inner product.  Here both variants run on the dense system of
Eq. (integral_eq) for a 320-panel sphere: their Givens residual estimates, Hessenberg
matrices and solutions must agree to rounding, and the estimates must match the true
residuals, so the shortcut changes no iterate beyond rounding.
"""
import numpy as np

import gen
from oracle import bem, multipole as mp


def _arnoldi_gmres(A, b, m, pythagoras):
    """m GMRES steps from x = 0: Givens residual estimates, Hessenberg matrix, minimiser."""
    n = b.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    beta = np.linalg.norm(b)
    V[0] = b / beta
    g = np.zeros(m + 1)
    g[0] = beta
    cs, sn = np.zeros(m), np.zeros(m)
    est = np.zeros(m)
    for j in range(m):
        w = A @ V[j]
        h1 = V[:j + 1] @ w
        w = w - V[:j + 1].T @ h1
        h2 = V[:j + 1] @ w
        if pythagoras:
            nn = max(w @ w - h2 @ h2, 0.0)     # |w'|^2 - |h2|^2, before the second subtraction
            w = w - V[:j + 1].T @ h2
        else:
            w = w - V[:j + 1].T @ h2
            nn = w @ w
        H[:j + 1, j] = h1 + h2
        H[j + 1, j] = np.sqrt(nn)
        V[j + 1] = w / H[j + 1, j]
        col = H[:, j].copy()
        for k in range(j):
            t = cs[k] * col[k] + sn[k] * col[k + 1]
            col[k + 1] = -sn[k] * col[k] + cs[k] * col[k + 1]
            col[k] = t
        r = np.hypot(col[j], col[j + 1])
        cs[j], sn[j] = col[j] / r, col[j + 1] / r
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        est[j] = abs(g[j + 1])
    y = np.linalg.lstsq(H, beta * np.eye(m + 1)[0], rcond=None)[0]
    return est, H, V[:m].T @ y


def test_pythagorean_norm_matches_cgs2():
    pr = gen.small_bumpy(subdiv=2, n_sites=8)
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    b = np.zeros(2 * mesh.n)
    b[:mesh.n] = mp.rhs(mesh.cen, pr.sites.pos, pr.sites.q, pr.sites.d, pr.sites.Q, par.eps_in)
    m = 40
    e_ref, H_ref, x_ref = _arnoldi_gmres(A, b, m, pythagoras=False)
    e_pyt, H_pyt, x_pyt = _arnoldi_gmres(A, b, m, pythagoras=True)
    assert np.allclose(e_pyt, e_ref, rtol=1e-8, atol=1e-14 * np.linalg.norm(b))
    assert np.allclose(H_pyt, H_ref, rtol=0.0, atol=1e-10 * np.abs(H_ref).max())
    assert np.linalg.norm(x_pyt - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # the estimate is the true residual of the minimiser after m steps
    true = np.linalg.norm(b - A @ x_pyt)
    assert abs(true - e_pyt[-1]) <= 1e-8 * np.linalg.norm(b)
    assert e_pyt[-1] < 1e-6 * np.linalg.norm(b)
