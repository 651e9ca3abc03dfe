"""Dense FP64 boundary-element system of Eq. (integral_eq) and its solution.

Unknowns: piecewise-constant phi_j and psi_j = dphi_1/dn on each panel j,
collocated at the panel centroids x_i.  Rows, for each target i:

    phi_i / 2 + sum_j K_L[i, j] phi_j - sum_j V_L[i, j] psi_j          = RHS_i
    phi_i / 2 - sum_j K_Y[i, j] phi_j + (eps1 / eps2) sum_j V_Y[i, j] psi_j = 0

with V = int_Tj G dS and K = int_Tj dG/dn_y dS (Eq. layers; n_y the outward
normal of the source panel).  Entries use the panel integrals of ``panel.py``
when the pair is near (``geometry.near_pairs``) and the K-node Gauss rule
otherwise (Sec. "The boundary element method").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

from . import geometry, panel


@dataclass
class Mesh:
    verts: np.ndarray
    tris: np.ndarray
    cen: np.ndarray
    normal: np.ndarray
    area: np.ndarray
    ygauss: np.ndarray     # [N, K, 3]
    wgauss: np.ndarray     # [N, K]
    near_ptr: np.ndarray
    near_cols: np.ndarray
    body: np.ndarray       # [N] body of each panel (several closed surfaces in one solvent)
    near_rule: str = "exact"   # near non-self pairs: "exact" panel integrals or "gauss19" nodes

    @property
    def n(self):
        return int(self.tris.shape[0])

    def same_body(self, rows, cols):
        return self.body[rows] == self.body[cols]


def build_mesh(verts, tris, gauss_k=4, near_factor=2.0, body=None, near_rule="exact") -> Mesh:
    """Panels, Gauss nodes and near pairs.  With several bodies (closed surfaces
    enclosing separate solute cavities, Sec. "Calculation of the binding energy"),
    ``body`` gives each panel's body.  ``near_rule="gauss19"`` integrates near pairs
    other than the self panel with the 19-node rule, as the paper's production runs do
    (Sec. "Comparison with Tinker-APBS"); the self panel stays semi-analytical."""
    if near_rule not in ("exact", "gauss19"):
        raise ValueError("near_rule must be 'exact' or 'gauss19'")
    cen, normal, area = geometry.panel_geometry(verts, tris)
    y, w = geometry.gauss_points(verts, tris, gauss_k)
    ptr, cols = geometry.near_pairs(cen, area, near_factor)
    b = np.zeros(tris.shape[0], dtype=np.int32) if body is None else np.asarray(body, dtype=np.int32)
    return Mesh(verts, tris, cen, normal, area, y, w, ptr, cols, b, near_rule)


def near_values(mesh: Mesh, rows, cols, kappa: float):
    """Near-pair integrals (VL, KL, VY, KY) for targets at the centroids ``rows`` and source
    panels ``cols``: semi-analytical, or the 19-node rule off the self panel under
    ``near_rule="gauss19"``."""
    t = mesh.tris[cols]
    self_p = rows == cols
    out = panel.panel_integrals(mesh.cen[rows], mesh.verts[t[:, 0]], mesh.verts[t[:, 1]],
                                mesh.verts[t[:, 2]], kappa, self_panel=self_p)
    if mesh.near_rule == "gauss19":
        off = ~self_p
        y, w = geometry.gauss_points(mesh.verts, mesh.tris[cols[off]], 19)
        kp = panel.kpoint_sums(mesh.cen[rows[off]], y, w, mesh.normal[cols[off]], kappa)
        for o, v in zip(out, kp):
            o[off] = v
    return out


def near_rows_cols(mesh: Mesh):
    rows = np.repeat(np.arange(mesh.n), np.diff(mesh.near_ptr))
    return rows, mesh.near_cols.astype(np.int64)


def near_exact(mesh: Mesh, kappa: float):
    """Near-pair integrals (``near_values``) for every near pair, in CSR order: (VL, KL, VY, KY)."""
    rows, cols = near_rows_cols(mesh)
    return near_values(mesh, rows, cols, kappa)


def near_kpoint(mesh: Mesh, kappa: float):
    """K-node Gauss sums for every near pair, in CSR order: (VL, KL, VY, KY)."""
    rows, cols = near_rows_cols(mesh)
    return panel.kpoint_sums(mesh.cen[rows], mesh.ygauss[cols], mesh.wgauss[cols],
                             mesh.normal[cols], kappa)


def near_correction(mesh: Mesh, kappa: float):
    """Accurate minus K-node value of each near pair (what a Gauss-node matvec must add)."""
    ex = near_exact(mesh, kappa)
    kp = near_kpoint(mesh, kappa)
    vl, kl, vy, ky = (e - k for e, k in zip(ex, kp))
    rows, cols = near_rows_cols(mesh)
    same = mesh.same_body(rows, cols)   # the Laplace layers do not couple bodies
    return np.where(same, vl, 0.0), np.where(same, kl, 0.0), vy, ky


def assemble_layers(mesh: Mesh, kappa: float, row_chunk: int = 256):
    """Dense [N, N] matrices VL, KL, VY, KY (far: K-node rule, near: accurate integrals)."""
    n = mesh.n
    VL = np.empty((n, n))
    KL = np.empty((n, n))
    VY = np.empty((n, n))
    KY = np.empty((n, n))
    for s in range(0, n, row_chunk):
        e = min(n, s + row_chunk)
        m = e - s
        x = np.repeat(mesh.cen[s:e], n, axis=0)
        yg = np.tile(mesh.ygauss, (m, 1, 1))
        wg = np.tile(mesh.wgauss, (m, 1))
        nr = np.tile(mesh.normal, (m, 1))
        vl, kl, vy, ky = panel.kpoint_sums(x, yg, wg, nr, kappa)
        VL[s:e] = vl.reshape(m, n)
        KL[s:e] = kl.reshape(m, n)
        VY[s:e] = vy.reshape(m, n)
        KY[s:e] = ky.reshape(m, n)
    rows, cols = near_rows_cols(mesh)
    vl, kl, vy, ky = near_exact(mesh, kappa)
    VL[rows, cols] = vl
    KL[rows, cols] = kl
    VY[rows, cols] = vy
    KY[rows, cols] = ky
    # Several bodies: the interior (Laplace) representation of a body integrates over
    # its own surface only; the solvent (Yukawa) one over every surface.
    cross = mesh.body[:, None] != mesh.body[None, :]
    VL[cross] = 0.0
    KL[cross] = 0.0
    return VL, KL, VY, KY


def system_matrix(layers, eps_in: float, eps_out: float):
    """The 2N x 2N matrix of Eq. (integral_eq) acting on x = [phi; psi]."""
    VL, KL, VY, KY = layers
    n = VL.shape[0]
    I = np.eye(n)
    A = np.empty((2 * n, 2 * n))
    A[:n, :n] = 0.5 * I + KL
    A[:n, n:] = -VL
    A[n:, :n] = 0.5 * I - KY
    A[n:, n:] = (eps_in / eps_out) * VY
    return A


class DenseSolver:
    """LU factors of the system matrix; ``solve(b)`` returns the exact discrete solution."""

    def __init__(self, mesh: Mesh, eps_in, eps_out, kappa):
        self.layers = assemble_layers(mesh, kappa)
        self.A = system_matrix(self.layers, eps_in, eps_out)
        self.lu = scipy.linalg.lu_factor(self.A)

    def solve(self, b):
        return scipy.linalg.lu_solve(self.lu, b)

    def matvec(self, x):
        return self.A @ x


def matvec_rows(mesh: Mesh, x: np.ndarray, rows: np.ndarray, eps_in, eps_out, kappa):
    """Rows ``rows`` of both blocks of A x without forming A (for large meshes).

    Returns (y1[rows], y2[rows]) where y1 is the Laplace row and y2 the Yukawa row.
    """
    n = mesh.n
    phi = x[:n]
    psi = x[n:]
    y1 = np.empty(rows.size)
    y2 = np.empty(rows.size)
    for t, i in enumerate(rows):
        xi = np.repeat(mesh.cen[i][None], n, axis=0)
        vl, kl, vy, ky = panel.kpoint_sums(xi, mesh.ygauss, mesh.wgauss, mesh.normal, kappa)
        cols = mesh.near_cols[mesh.near_ptr[i]:mesh.near_ptr[i + 1]].astype(np.int64)
        ex = near_values(mesh, np.full(cols.size, i, dtype=np.int64), cols, kappa)
        vl[cols], kl[cols], vy[cols], ky[cols] = ex
        other = mesh.body != mesh.body[i]
        vl[other] = 0.0
        kl[other] = 0.0
        y1[t] = 0.5 * phi[i] + kl @ phi - vl @ psi
        y2[t] = 0.5 * phi[i] - ky @ phi + (eps_in / eps_out) * (vy @ psi)
    return y1, y2
