"""Plain, slow FP64 CPU oracle for the boundary-integral Poisson-Boltzmann method
with polarizable multipoles (Cooper, arXiv:1810.03698).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path; the two meet only in
the seeded input generators of ``gen/``.

Modules
-------
geometry   panel centroids, normals, areas, Gauss rules, near-pair criterion
panel      semi-analytical single/double-layer integrals over one flat triangle
bem        dense BEM matrix (Eq. integral_eq), LU solve, sampled matvec rows
multipole  multipole tensors, RHS (Eq. rhs_multipole), fields at sites, Thole
           damping, SCF (SOR) and its direct counterpart, energy (Eq.
           energy_multipole_polarizable), solvation energy; several bodies in one
           solvent (Sec. "Calculation of the binding energy")
kirkwood   closed-form reaction field of a dielectric sphere in salt water, with or
           without a Stern (ion-exclusion) layer
gradient   dDelta G_solv / d(site positions, q, d, Q): five-point differences of
           the solvation energy at the exact induced-dipole fixed point
stern      Stern (ion-exclusion) layer: three regions bounded by two surfaces, the
           four Green's-representation rows solved densely (Sec. "Spherical cavity")

Parity pins (see tests/test_oracle_*.py): every function is checked against
something other than itself -- closed forms (Born, Kirkwood, solid angles),
Gauss's law, brute-force quadrature, finite differences, exact identities, the
screened two-ion energy of two bodies, Euler's identity of the gradient.
Parity unpinned: none of the functions here.  The paper's own printed sphere value
(-65.1131 kcal/mol, with a Stern layer) is not reproduced: the orientations and units
of its multipoles are not stated.
"""

__all__ = ["geometry", "panel", "bem", "multipole", "kirkwood", "gradient", "stern"]
