"""Accurate integrals of the four BEM kernels over one flat triangle.

Sec. "The boundary element method": the singular (collocation point on the
panel) and near-singular (panel within the near threshold) integrals are done
semi-analytically.  The reading used here:

* Project the target x onto the panel plane: foot point p, signed height
  h = n . (x - v0) with n the unit outward normal (for the target's own panel
  h = 0 exactly).
* Split the triangle into the three signed sub-triangles (p, v_a, v_b), one
  per edge; the sign is the orientation of (v_a - p) x (v_b - p) along n.
* In polar coordinates (rho, psi) about p, with s = sqrt(rho^2 + h^2), the
  radial integrals of the kernels have closed forms (Eqs. free-space, layers):

      int_0^R  G_L        rho drho = (s - |h|) / 4pi
      int_0^R  G_Y        rho drho = (e^{-k|h|} - e^{-k s}) / (4pi k)
      int_0^R  dG_L/dn_y  rho drho = sgn(h) (1 - |h|/s) / 4pi
      int_0^R  dG_Y/dn_y  rho drho = sgn(h) (e^{-k|h|} - |h| e^{-k s}/s) / 4pi

  with s = s(R), R = rho_max(psi) the distance from p to the edge along psi,
  and dG/dn_y = n . (x - y) (1 + k r) e^{-k r} / (4 pi r^3) the derivative
  in the source normal (for k = 0 the Laplace forms).
* The angular integral runs over each sub-triangle's edge.  With d the
  distance from p to the edge line and t the signed position along the edge
  from the foot of p, rho_max = sqrt(d^2 + t^2); substituting t = d sinh(u)
  gives dpsi = du / cosh(u) and rho_max = d cosh(u), an integrand whose
  complex singularities stay at |Im u| >= pi/2 however close p is to the edge.
  The oracle integrates u with composite Gauss-Legendre (pieces of length
  <= 0.5, 16 nodes each); tests pin this against adaptive quadrature in psi
  and against brute-force 2-D quadrature of the kernels over the triangle.

Every returned value includes the 1/(4 pi) of the Green's functions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np

_GL_N = 16
_GL_X, _GL_W = np.polynomial.legendre.leggauss(_GL_N)
_PIECE = 0.5
FOUR_PI = 4.0 * np.pi


def _cross(a, b):
    out = np.empty(np.broadcast_shapes(a.shape, b.shape))
    out[..., 0] = a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1]
    out[..., 1] = a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2]
    out[..., 2] = a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]
    return out


def radial_closed_forms(rho, h, kappa):
    """The four radial integrals (times 4 pi) from rho = 0 to rho at height h.

    Returns (VL, VY, KL, KY) arrays, written in cancellation-free forms:
    s - |h| = rho^2 / (s + |h|), and e^{-k|h|} - e^{-k s} = -e^{-k|h|} expm1(-k (s - |h|)).
    """
    ah = np.abs(h)
    sh = np.sign(h)
    s = np.sqrt(rho * rho + h * h)
    sm = rho * rho / (s + ah)
    fvl = sm
    fkl = sh * sm / s
    if kappa > 0.0:
        eh = np.exp(-kappa * ah)
        em = -np.expm1(-kappa * sm)          # 1 - e^{-k (s-|h|)}
        fvy = eh * em / kappa
        fky = sh * (eh * sm / s + (ah / s) * eh * em)
    else:
        fvy = fvl.copy()
        fky = fkl.copy()
    return fvl, fvy, fkl, fky


def panel_integrals(x, v0, v1, v2, kappa, self_panel=None):
    """Integrals over triangles (v0, v1, v2) of G_L, dG_L/dn_y, G_Y, dG_Y/dn_y at targets x.

    All arguments are row-aligned arrays [M, 3]; ``self_panel`` [M] bool marks
    pairs whose target is the centroid of the same panel (h forced to 0).
    Returns (VL, KL, VY, KY), each [M], including 1/(4 pi).
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    v0 = np.atleast_2d(v0)
    v1 = np.atleast_2d(v1)
    v2 = np.atleast_2d(v2)
    m = x.shape[0]
    cr = _cross(v1 - v0, v2 - v0)
    n = cr / np.sqrt(np.sum(cr * cr, axis=1))[:, None]
    h = np.sum(n * (x - v0), axis=1)
    if self_panel is not None:
        h = np.where(np.asarray(self_panel, dtype=bool), 0.0, h)
    p = x - h[:, None] * n

    sub_pair, sub_sig, sub_d, sub_ua, sub_ub = [], [], [], [], []
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        ap = a - p
        bp = b - p
        ab = b - a
        L = np.sqrt(np.sum(ab * ab, axis=1))
        u = ab / L[:, None]
        nc = np.sum(n * _cross(ap, bp), axis=1)
        d = np.abs(nc) / L
        ok = d > 1e-14 * L
        ta = np.sum(ap * u, axis=1)
        tb = np.sum(bp * u, axis=1)
        idx = np.nonzero(ok)[0]
        sub_pair.append(idx)
        sub_sig.append(np.sign(nc[idx]))
        sub_d.append(d[idx])
        sub_ua.append(np.arcsinh(ta[idx] / d[idx]))
        sub_ub.append(np.arcsinh(tb[idx] / d[idx]))
    pair = np.concatenate(sub_pair)
    sig = np.concatenate(sub_sig)
    d = np.concatenate(sub_d)
    ua = np.concatenate(sub_ua)
    ub = np.concatenate(sub_ub)

    npc = np.maximum(1, np.ceil((ub - ua) / _PIECE).astype(np.int64))
    rep = np.repeat(np.arange(pair.size), npc)
    k = np.arange(rep.size) - np.repeat(np.cumsum(npc) - npc, npc)
    du = (ub - ua)[rep] / npc[rep]
    u0 = ua[rep] + k * du
    # nodes: [pieces, GL]
    uu = u0[:, None] + 0.5 * du[:, None] * (_GL_X[None, :] + 1.0)
    ww = 0.5 * du[:, None] * _GL_W[None, :]
    ch = np.cosh(uu)
    rho = d[rep][:, None] * ch
    hh = h[pair[rep]][:, None]
    fvl, fvy, fkl, fky = radial_closed_forms(rho, hh, kappa)
    wt = (ww / ch) * sig[rep][:, None]
    out = np.zeros((4, m))
    for r, f in enumerate((fvl, fkl, fvy, fky)):
        contrib = np.sum(wt * f, axis=1)
        out[r] = np.bincount(pair[rep], weights=contrib, minlength=m)
    return out[0] / FOUR_PI, out[1] / FOUR_PI, out[2] / FOUR_PI, out[3] / FOUR_PI


def kpoint_sums(x, ygauss, wgauss, normal, kappa):
    """K-node quadrature of the four kernels, row-aligned.

    x [M, 3] targets; ygauss [M, K, 3] nodes; wgauss [M, K] weights w_g A_j;
    normal [M, 3] source-panel normals.  Coincident node/target pairs (r = 0)
    contribute zero.  Returns (VL, KL, VY, KY), each [M], including 1/(4 pi).
    """
    r = x[:, None, :] - ygauss
    r2 = np.sum(r * r, axis=2)
    zero = r2 == 0.0
    rr = np.sqrt(np.where(zero, 1.0, r2))
    inv = np.where(zero, 0.0, 1.0 / rr)
    nr = np.sum(normal[:, None, :] * r, axis=2)
    e = np.exp(-kappa * rr)
    vl = np.sum(wgauss * inv, axis=1)
    kl = np.sum(wgauss * nr * inv ** 3, axis=1)
    vy = np.sum(wgauss * e * inv, axis=1)
    ky = np.sum(wgauss * nr * (1.0 + kappa * rr) * e * inv ** 3, axis=1)
    return vl / FOUR_PI, kl / FOUR_PI, vy / FOUR_PI, ky / FOUR_PI
