"""Stern (ion-exclusion) layer: three regions bounded by two closed surfaces, dense FP64.

The sphere test of Sec. "Spherical cavity" puts a 1 A layer free of ions between the
solute's dielectric boundary Gamma_1 and the surface Gamma_2 where the salt begins.
The paper does not write out the boundary integral equations of that case; this
module states the reading used here, built from Green's representation in each region
exactly as Eq. (integral_eq) is for one surface:

  region 1 (inside Gamma_1):   Laplace, permittivity eps1, the sites;
  region 2 (between the two):  Laplace, permittivity eps2, no ions;
  region 3 (outside Gamma_2):  Yukawa (kappa), permittivity eps2.

Unknowns, piecewise constant and collocated at panel centroids: phi_1 and
psi_1 = dphi/dn seen from region 1 on Gamma_1, phi_2 and psi_2 = dphi/dn on Gamma_2
(the same on both sides of Gamma_2: eps2 on both).  Normals point out of the enclosed
volume on both surfaces, so region 2 sees -n_1 on Gamma_1, where its normal derivative
is -(eps1/eps2) psi_1 (continuity of eps dphi/dn).  Rows:

  Gamma_1, region 1:  phi_1/2 + K11 phi_1 - V11 psi_1                                = RHS
  Gamma_1, region 2:  phi_1/2 - K11 phi_1 + (eps1/eps2) V11 psi_1 + K12 phi_2 - V12 psi_2 = 0
  Gamma_2, region 2:  phi_2/2 + K22 phi_2 - V22 psi_2 - K21 phi_1 + (eps1/eps2) V21 psi_1 = 0
  Gamma_2, region 3:  phi_2/2 - KY22 phi_2 + VY22 psi_2                              = 0

with Kij, Vij the Laplace double and single layers for targets on Gamma_i and source
panels on Gamma_j (KY, VY: Yukawa).  The reaction field at the sites is region 1's
representation over Gamma_1 alone, as without a layer.  With kappa = 0 region 3 is plain
solvent and the solution equals the one-surface solution on Gamma_1.

Parity pins (tests/test_oracle_stern.py): convergence to the closed-form sphere with a
Stern layer (``kirkwood.f_coeffs`` with b), the kappa = 0 reduction to the one-surface
system, and Gauss's law for the total normal flux through Gamma_2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import bem, panel


def cross_layers(tgt: bem.Mesh, src: bem.Mesh, kappa: float, near_factor: float, row_chunk: int = 256):
    """Dense [Nt, Ns] VL, KL, VY, KY for targets at the centroids of ``tgt`` and the panels
    of ``src`` (two different surfaces): the K-node rule, replaced by the accurate panel
    integrals where |x_i - c_j|^2 < near_factor^2 A_i, A_i the area of the element holding
    the collocation point (Sec. "The boundary element method"), as on one surface."""
    from scipy.spatial import cKDTree

    nt, ns = tgt.n, src.n
    out = [np.empty((nt, ns)) for _ in range(4)]
    for s in range(0, nt, row_chunk):
        e = min(nt, s + row_chunk)
        m = e - s
        x = np.repeat(tgt.cen[s:e], ns, axis=0)
        yg = np.tile(src.ygauss, (m, 1, 1))
        wg = np.tile(src.wgauss, (m, 1))
        nr = np.tile(src.normal, (m, 1))
        for o, v in zip(out, panel.kpoint_sums(x, yg, wg, nr, kappa)):
            o[s:e] = v.reshape(m, ns)
    thr = (near_factor * near_factor) * tgt.area
    radius = float(np.sqrt(thr.max())) * (1.0 + 1e-6) + 1e-12
    cand = cKDTree(src.cen).query_ball_point(tgt.cen, radius)
    ci = np.repeat(np.arange(nt), [len(c) for c in cand])
    cj = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if nt else np.zeros(0, np.int64)
    d = tgt.cen[ci] - src.cen[cj]
    keep = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] < thr[ci]
    ci, cj = ci[keep], cj[keep]
    if ci.size:
        t = src.tris[cj]
        ex = panel.panel_integrals(tgt.cen[ci], src.verts[t[:, 0]], src.verts[t[:, 1]], src.verts[t[:, 2]], kappa)
        for o, v in zip(out, ex):
            o[ci, cj] = v
    return tuple(out)


def system_matrix(mesh1: bem.Mesh, mesh2: bem.Mesh, eps_in: float, eps_out: float, kappa: float,
                  near_factor: float):
    """The (2 N1 + 2 N2) square matrix of the four rows above, acting on
    [phi_1; psi_1; phi_2; psi_2]."""
    n1, n2 = mesh1.n, mesh2.n
    VL11, KL11, _, _ = bem.assemble_layers(mesh1, kappa)
    VL22, KL22, VY22, KY22 = bem.assemble_layers(mesh2, kappa)
    VL12, KL12, _, _ = cross_layers(mesh1, mesh2, kappa, near_factor)
    VL21, KL21, _, _ = cross_layers(mesh2, mesh1, kappa, near_factor)
    r = eps_in / eps_out
    I1, I2 = np.eye(n1), np.eye(n2)
    A = np.zeros((2 * n1 + 2 * n2, 2 * n1 + 2 * n2))
    p1, s1, p2, s2 = (slice(0, n1), slice(n1, 2 * n1), slice(2 * n1, 2 * n1 + n2),
                      slice(2 * n1 + n2, 2 * n1 + 2 * n2))
    # Gamma_1, region 1
    A[p1, p1] = 0.5 * I1 + KL11
    A[p1, s1] = -VL11
    # Gamma_1, region 2
    A[s1, p1] = 0.5 * I1 - KL11
    A[s1, s1] = r * VL11
    A[s1, p2] = KL12
    A[s1, s2] = -VL12
    # Gamma_2, region 2
    A[p2, p1] = -KL21
    A[p2, s1] = r * VL21
    A[p2, p2] = 0.5 * I2 + KL22
    A[p2, s2] = -VL22
    # Gamma_2, region 3
    A[s2, p2] = 0.5 * I2 - KY22
    A[s2, s2] = VY22
    return A


class SternSolver:
    """LU factors of the three-region system.  ``solve(b)`` takes the one-surface layout
    b = [RHS on Gamma_1; 0] of ``bem.DenseSolver`` and returns [phi_1; psi_1], so the
    induced-dipole iteration and the energy of ``multipole.solvation`` run unchanged on
    Gamma_1; ``solve_full`` returns all four unknowns."""

    def __init__(self, mesh1: bem.Mesh, mesh2: bem.Mesh, eps_in, eps_out, kappa, near_factor):
        self.mesh = mesh1
        self.mesh2 = mesh2
        self.A = system_matrix(mesh1, mesh2, eps_in, eps_out, kappa, near_factor)
        self.lu = scipy.linalg.lu_factor(self.A)

    def solve_full(self, rhs1):
        b = np.zeros(self.A.shape[0])
        b[:self.mesh.n] = rhs1
        return scipy.linalg.lu_solve(self.lu, b)

    def solve(self, b):
        n1 = self.mesh.n
        return self.solve_full(b[:n1])[:2 * n1]


def stern_solver(verts1, tris1, verts2, tris2, params) -> SternSolver:
    """Dielectric boundary (verts1, tris1) inside the ion-exclusion surface (verts2, tris2)."""
    m1 = bem.build_mesh(verts1, tris1, params.gauss_k, params.near_factor)
    m2 = bem.build_mesh(verts2, tris2, params.gauss_k, params.near_factor)
    return SternSolver(m1, m2, params.eps_in, params.eps_out, params.kappa, params.near_factor)
