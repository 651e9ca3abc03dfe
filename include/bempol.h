/*
 * bempol.h -- C ABI of a GB300 (sm_103a) boundary-integral Poisson-Boltzmann solver
 * with polarizable point multipoles (Cooper, "A boundary-integral approach for the
 * Poisson-Boltzmann equation with polarizable force fields", arXiv:1810.03698).
 *
 * Model (Sec. "The boundary integral formulation", Eqs. pde, green_identity,
 * layers, free-space, integral_eq): solute region Omega_1 (permittivity eps_in,
 * point multipoles), solvent Omega_2 (eps_out, inverse Debye length kappa), interface
 * Gamma given as a closed triangle mesh.  Unknowns are phi and psi = dphi_1/dn on
 * Gamma, piecewise constant per flat panel, collocated at the panel centroids
 * (Sec. "The boundary element method"):
 *
 *   phi_i/2 + K_L[phi]_i - V_L[psi]_i                    = RHS_i   (Eq. rhs_multipole)
 *   phi_i/2 - K_Y[phi]_i + (eps_in/eps_out) V_Y[psi]_i   = 0
 *
 * with G_L = 1/(4 pi r), G_Y = e^{-kappa r}/(4 pi r), V = int G, K = int dG/dn_y
 * (n the outward normal of the source panel).  Far-away panels use a K-node
 * Gauss rule; panels within near_factor*sqrt(A_i) of collocation point i use
 * FP64 semi-analytical integrals.
 *
 * Units: angstrom, elementary charge; potentials q/(4 pi eps r) (vacuum
 * permittivity 1); polarizabilities are polarizability volumes (A^3), so an
 * induced dipole is mu = 4 pi alpha E in these units (Eq. induced_dipole);
 * energies are reported in kcal/mol (1 e^2/A in these units = 4 pi * 332.0637).
 *
 * Conventions common to every entry point
 *  - Every function returns a bempol_status; on error the context keeps a
 *    message readable with bempol_last_error().  Nothing aborts the process.
 *  - Pointers marked "host or device" are read or written according to the
 *    `where` argument (BEMPOL_HOST or BEMPOL_DEVICE).  Device pointers belong to
 *    the current CUDA context of the device given to bempol_create.
 *  - Pointers marked "device" must be device memory; "host" must be host memory.
 *  - The caller owns every buffer it passes; the library owns its internal
 *    geometry, tree, near-field tables and solver workspaces (allocated by
 *    bempol_set_mesh / bempol_set_sites / first solve, freed by bempol_destroy).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute entry
 *    points enqueue their work on that stream; solver entry points also
 *    synchronise it to read convergence scalars.
 *  - Panel-indexed arrays at the ABI are in the caller's triangle order
 *    (the library reorders internally and maps back).
 *  - Double-precision is used at the ABI throughout.
 *
 * Several bodies and several systems (Sec. "Calculation of the binding energy":
 * a complex AB is two solute cavities in one solvent).  A context may hold
 * several independent systems, each with one or more bodies (closed surfaces).
 * Within a system the Laplace layers, the right-hand side and the reaction field
 * at a site involve only the site's or panel's own body; the Yukawa layers couple
 * every panel of the system; different systems never interact.  The entry points
 * without "_systems" in their name treat everything as one body of one system.
 */
#ifndef BEMPOL_H
#define BEMPOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bempol_ctx bempol_ctx;

typedef enum {
  BEMPOL_OK = 0,
  BEMPOL_ERR_ARG = 1,             /* bad argument (NULL, size, enum, parameter range) */
  BEMPOL_ERR_MESH = 2,            /* mesh fails validation (index range, degenerate or inverted panel, not closed) */
  BEMPOL_ERR_SITES = 3,           /* sites fail validation (outside or within the near radius of a panel, alpha < 0, Q not symmetric traceless) */
  BEMPOL_ERR_NOT_CONVERGED = 4,   /* GMRES or SCF hit its iteration limit; results hold the last iterate */
  BEMPOL_ERR_CUDA = 5,            /* a CUDA runtime call failed (message has the CUDA error string) */
  BEMPOL_ERR_TIMEOUT = 6,         /* a bounded device-side wait expired */
  BEMPOL_ERR_OOM = 7,             /* device allocation failed */
  BEMPOL_ERR_STATE = 8            /* call out of order (e.g. solve before set_mesh) */
} bempol_status;

enum { BEMPOL_HOST = 0, BEMPOL_DEVICE = 1 };

/* Matrix-vector product / operator forms. */
enum {
  BEMPOL_OP_FP64_DIRECT = 0,   /* every Gauss-node pair in FP64, FP64 sums */
  BEMPOL_OP_FP32_DIRECT = 1,   /* every pair in FP32, FP32 tile sums, FP64 per-target sums */
  BEMPOL_OP_FP32_TREE = 2,     /* treecode (Taylor far field, theta, order) in FP32, FP64 per-target sums */
  BEMPOL_OP_FP64_TREE = 3      /* treecode in FP64 */
};

typedef struct {
  double eps_in, eps_out;      /* relative permittivities of solute and solvent */
  double kappa;                /* inverse Debye length, 1/A (>= 0) */
  int gauss_k;                 /* Gauss nodes per far panel: 1, 3 or 4 */
  double near_factor;          /* near-singular threshold: |x_i - c_j| < near_factor*sqrt(A_i) */
  double theta;                /* treecode multipole acceptance: cell accepted if R_cell / dist < theta */
  int order;                   /* treecode Taylor order P (1..6) */
  int leaf;                    /* treecode maximum panels per leaf */
  double gmres_tol;            /* stop when ||b - A x||_2 / ||b||_2 < gmres_tol */
  int gmres_restart;           /* Krylov basis size before a restart */
  int gmres_maxit;             /* total GMRES iterations per solve */
  double scf_tol;              /* SCF stop: sqrt(sum_i |mu_new - mu_old|^2 / Ns) < scf_tol (e*A) */
  double sor_omega;            /* SOR coefficient (paper: 0.7) */
  int scf_maxit;
  int op;                      /* operator used inside GMRES: BEMPOL_OP_* */
  int residual_op;             /* operator for the outer FP64 residual of iterative refinement
                                  (BEMPOL_OP_*; equal to `op` = plain GMRES, no refinement) */
  double inner_tol;            /* relative tolerance of each inner solve under refinement */
  int refine_maxit;            /* maximum refinement (outer) steps */
  double thole_a;              /* Thole damping parameter (AMOEBA: 0.39) */
  int refine_scope;            /* which BEM solves of bempol_solve* are refined when residual_op != op:
                                  BEMPOL_REFINE_EVERY or BEMPOL_REFINE_FINAL (see below) */
  int thole_perm;              /* 1: Thole-damp the permanent moments' polarising field too (AMOEBA's
                                  rule; the paper damps only the induced dipoles): the 1/r^3 terms
                                  take lambda3, the 1/r^5 lambda5, the 1/r^7 lambda7.  The energy's
                                  permanent terms stay undamped.  bempol_gradient does not support
                                  it (BEMPOL_ERR_ARG).  0 (default): the paper's rule. */
  int near_rule;               /* accurate value of a near pair other than the self panel:
                                  BEMPOL_NEAR_SEMI_ANALYTICAL (default) or BEMPOL_NEAR_GAUSS19, the
                                  fully symmetric 19-node rule of degree 9 (Dunavant 1985), which
                                  the paper's production runs apply within 1.25 sqrt(A) (Sec.
                                  "Comparison with Tinker-APBS").  The self panel stays
                                  semi-analytical.  Fixed once a mesh is set. */
} bempol_params;

enum { BEMPOL_NEAR_SEMI_ANALYTICAL = 0, BEMPOL_NEAR_GAUSS19 = 19 };

/* Scope of the FP64 iterative refinement inside bempol_solve* (residual_op != op).
 *  BEMPOL_REFINE_EVERY: every BEM solve of both induced-dipole iterations is refined, and the
 *    right-hand sides, reaction fields and multipole fields use residual_op's precision.
 *  BEMPOL_REFINE_FINAL: the solves inside the induced-dipole iteration run plain GMRES with
 *    `op` (warm-started) to max(gmres_tol, 1e-6) when op is an FP32 form (the residual such an
 *    operator reaches) or to gmres_tol otherwise, with site-side sums in op's precision; only
 *    the last solve, whose phi and psi give the energy, is refined against residual_op (to
 *    gmres_tol), and its right-hand side, reaction field and energy-form multipole fields use
 *    residual_op's precision.  The adjoint (bempol_gradient) then runs its transposed solves
 *    with `op` alone. */
enum { BEMPOL_REFINE_EVERY = 0, BEMPOL_REFINE_FINAL = 1 };

typedef struct {
  /* scalars, always written (host memory inside this struct) */
  double dG_solv_kcal;         /* G_diss - G_vac in kcal/mol (Eqs. deltaG_aux2, energy_multipole_polarizable) */
  double G_diss, G_vac;        /* the two energies in the paper's units (e^2/A, vacuum permittivity 1) */
  int scf_iters_diss, scf_iters_vac;
  int gmres_iters_total;       /* GMRES iterations summed over all solves */
  int matvecs_total;           /* operator applications (inner + residual) */
  int n_solves;                /* BEM solves performed */
  double last_rel_residual;    /* ||b - A x|| / ||b|| of the final BEM solve (with residual_op) */
  double t_setup_ms, t_scf_ms, t_total_ms;   /* wall time of the phases, measured on the stream */
  /* optional outputs (NULL to skip), in the caller's order; host or device per `where` */
  double* phi;                 /* [N]   potential on the panels */
  double* dphidn;              /* [N]   dphi_1/dn on the panels */
  double* site_reaction;       /* [Ns*10] per site: phi_solv, grad phi_solv (3), Hessian xx,xy,xz,yy,yz,zz */
  double* mu_diss;             /* [Ns*3] induced dipoles, dissolved state */
  double* mu_vac;              /* [Ns*3] induced dipoles, vacuum state */
  int where;                   /* BEMPOL_HOST or BEMPOL_DEVICE for the optional outputs */
  int residual_matvecs;        /* of matvecs_total, the products with residual_op (refinement residuals) */
} bempol_result;

/* Per-system result of bempol_solve_systems (host memory). */
typedef struct {
  double dG_solv_kcal;         /* this system's G_diss - G_vac in kcal/mol */
  double G_diss, G_vac;        /* paper units as in bempol_result */
  int scf_iters_diss, scf_iters_vac;
  int gmres_iters;             /* GMRES iterations this system took, summed over its solves */
  int n_solves;                /* BEM solves that included this system */
  double last_rel_residual;    /* relative residual of its final solve */
  int converged;               /* 1 if its SCFs and every solve converged */
  int64_t n_panels, n_sites;
} bempol_system_result;

/* Fill `p` with the defaults: eps 1/80, kappa 0.125, K=4, near 2.0, theta 0.5,
 * P=5, leaf 256, GMRES 1e-8/100/500, SCF 1e-8/omega 0.7/200, op FP64 direct,
 * residual FP64 direct, inner_tol 1e-3, refine 20, Thole 0.39, refine_scope EVERY,
 * thole_perm 0, near_rule semi-analytical. */
void bempol_default_params(bempol_params* p);

/* Create a context on CUDA device `device`.  Validates `p` (ranges above);
 * BEMPOL_ERR_ARG on a bad value, BEMPOL_ERR_CUDA if the device cannot be used.
 * *out is NULL on failure. */
bempol_status bempol_create(const bempol_params* p, int device, bempol_ctx** out);

/* Replace the parameters of an existing context (same validation as create).
 * Geometry-dependent tables are rebuilt on the next call that needs them when
 * gauss_k, near_factor, kappa or leaf change. */
bempol_status bempol_set_params(bempol_ctx* c, const bempol_params* p);

/* Release everything the context owns.  NULL is a no-op. */
void bempol_destroy(bempol_ctx* c);

/* Message of the last error on this context ("" when none); owned by the context. */
const char* bempol_last_error(const bempol_ctx* c);

/* Set the surface (Sec. "The boundary element method": flat triangles).
 *   verts [nv*3] float64 (x,y,z per vertex), host or device per `where`
 *   tris  [nt*3] int32, counter-clockwise seen from the solvent side (so
 *         (v1-v0)x(v2-v0) is the outward normal n of Eq. pde), host or device
 * Validates index range, zero-area panels and closedness (every edge shared by
 * exactly two panels with opposite orientation), then builds on `stream`: panel
 * centroids/normals/areas, Gauss nodes, the Morton-ordered panel permutation and
 * treecode cells, the near-pair list and its FP64 semi-analytical corrections
 * (exact minus K-node value for each near pair).  Synchronises `stream`.
 * Errors: BEMPOL_ERR_ARG, BEMPOL_ERR_MESH, BEMPOL_ERR_OOM, BEMPOL_ERR_CUDA. */
bempol_status bempol_set_mesh(bempol_ctx* c, int64_t nv, const double* verts, int64_t nt,
                              const int32_t* tris, int where, void* stream);

/* Set the point multipoles (Eqs. pot_multipole, induced_dipole).
 *   pos   [ns*3] A;  q [ns] e;  d [ns*3] permanent dipoles e*A;
 *   Q     [ns*9] e*A^2, row-major 3x3, symmetric and traceless in the paper's
 *         convention Q = int rho (3 r r - r^2 I) (a trace below 1e-9 |Q| is
 *         removed, a larger one or asymmetry is rejected);
 *   alpha [ns] polarizability volumes A^3 (>= 0);
 *   group [ns] int32 polarisation group (NULL = every site its own group).
 * All host or device per `where`.  Validation: every site strictly inside the
 * surface and farther than near_factor*sqrt(A_j) from every panel centroid j
 * (BEMPOL_ERR_SITES).  Requires bempol_set_mesh first, and a single-body mesh
 * (BEMPOL_ERR_STATE; see bempol_set_sites_systems) or a Stern-layer mesh
 * (bempol_set_mesh_stern; the sites then lie inside both surfaces). */
bempol_status bempol_set_sites(bempol_ctx* c, int64_t ns, const double* pos, const double* q,
                               const double* d, const double* Q, const double* alpha,
                               const int32_t* group, int where, void* stream);

/* Set several bodies and systems at once.  As bempol_set_mesh, plus
 *   panel_system [nt] int32 system of each triangle: ids 0..S-1, each present
 *                (NULL = all 0);
 *   panel_body   [nt] int32 body of each triangle within its system, any ids >= 0
 *                (NULL = all 0);
 * host or device per `where`.  Every (system, body) must be a closed surface of
 * its own (no edge shared between bodies: BEMPOL_ERR_MESH).  Limits: at most
 * 1,023 (system, body) pairs and 16,777,215 triangles (BEMPOL_ERR_ARG).  Panels
 * are reordered by system, body and Morton code; the octree is a forest with one
 * root per body, and near-field pairs and treecode interaction lists never cross
 * systems. */
bempol_status bempol_set_mesh_systems(bempol_ctx* c, int64_t nv, const double* verts, int64_t nt,
                                      const int32_t* tris, const int32_t* panel_system,
                                      const int32_t* panel_body, int where, void* stream);

/* Stern (ion-exclusion) layer, Sec. "Spherical cavity": the dielectric boundary Gamma_1
 * (verts1 [nv1*3], tris1 [nt1*3]) strictly inside the surface Gamma_2 (verts2, tris2) where
 * the ions begin; three regions: Laplace with eps_in inside Gamma_1, Laplace with eps_out
 * and no ions between, Yukawa (kappa) with eps_out outside Gamma_2.  Unknowns phi and
 * psi = dphi/dn on both surfaces (psi on Gamma_1 as seen from the solute), laid out as for
 * one surface over the panels of both: caller order is Gamma_1's triangles, then Gamma_2's.
 * Rows, with r = eps_in/eps_out and Kij, Vij the Laplace layers at Gamma_i from Gamma_j:
 *   Gamma_1: phi1/2 + K11 phi1 - V11 psi1 = RHS;
 *            phi1/2 - K11 phi1 + r V11 psi1 + K12 phi2 - V12 psi2 = 0;
 *   Gamma_2: phi2/2 + K22 phi2 - V22 psi2 - K21 phi1 + r V21 psi1 = 0;
 *            phi2/2 - KY22 phi2 + VY22 psi2 = 0.
 * The reaction field at the sites is Gamma_1's.  Host arrays only (`where` must be
 * BEMPOL_HOST).  Each surface must be closed and Gamma_1 must lie inside Gamma_2
 * (BEMPOL_ERR_MESH).  Such a context takes the direct operator forms only (a treecode
 * form is BEMPOL_ERR_ARG), its sites are set with bempol_set_sites (all inside Gamma_1),
 * and bempol_gradient does not cover it (BEMPOL_ERR_ARG). */
bempol_status bempol_set_mesh_stern(bempol_ctx* c, int64_t nv1, const double* verts1, int64_t nt1,
                                    const int32_t* tris1, int64_t nv2, const double* verts2, int64_t nt2,
                                    const int32_t* tris2, int where, void* stream);

/* Sites of a context set with bempol_set_mesh_systems.  As bempol_set_sites, plus
 *   site_system, site_body [ns] int32 (NULL = all 0), host or device per `where`.
 * Sites must be ordered by system, then by body (in the order the bodies' ids
 * sort), and each site's (system, body) must have a surface (BEMPOL_ERR_SITES
 * otherwise).  Validation also rejects a site inside another body of its system.
 * Polarisation groups are global ids (a group should not span bodies). */
bempol_status bempol_set_sites_systems(bempol_ctx* c, int64_t ns, const double* pos, const double* q,
                                       const double* d, const double* Q, const double* alpha,
                                       const int32_t* group, const int32_t* site_system,
                                       const int32_t* site_body, int where, void* stream);

/* Number of systems and of bodies ((system, body) pairs) of the current mesh. */
bempol_status bempol_systems(const bempol_ctx* c, int64_t* n_systems, int64_t* n_bodies);

/* Solvation free energy Delta G_solv = G_diss - G_vac (Sec. "Calculation of the
 * solvation energy") with the self-consistent induced dipoles of Sec.
 * "Self-consistent induced field": vacuum SCF; then mu = 0, repeat { solve the
 * BEM system with RHS from p = d + mu (GMRES with params.op, warm-started, FP64
 * Krylov basis, optional FP64 iterative refinement with params.residual_op);
 * E = E_solv + E_mult; mu <- (1-omega) mu + omega 4 pi alpha E } until the RMS
 * change < scf_tol; one more solve with the converged mu; energy of Eq.
 * energy_multipole_polarizable.  Fills `out` (scalars always, arrays if non-NULL).
 * Returns BEMPOL_ERR_NOT_CONVERGED (with `out` filled) if GMRES or the SCF hit
 * their limits.  Synchronises `stream`. */
bempol_status bempol_solve(bempol_ctx* c, void* stream, bempol_result* out);

/* bempol_solve for every system of the context at once (Sec. "Calculation of the
 * binding energy": Delta G_solv of A, B and AB gives Delta Delta G_bind =
 * Delta G_solv,AB - Delta G_solv,A - Delta G_solv,B).  The systems share every
 * kernel launch: one matrix-vector product serves all of them, while each system
 * runs its own GMRES (own Krylov basis, Hessenberg matrix and stopping test) and
 * its own vacuum and dissolved SCF (own RMS test); a converged system stops
 * updating while the others continue.  In the dissolved state a site feels the
 * reaction field of its own body's surface and the multipoles of its own body; in
 * vacuum it feels every site of its system.
 *   per [n_per] host array (NULL to skip), n_per >= number of systems.
 * `out` receives the sums over systems (dG_solv_kcal, G_diss, G_vac), the largest
 * SCF iteration counts and residual, the totals of GMRES iterations (lockstep
 * iterations, each counted once), operator applications and solves, and the
 * optional arrays for every panel and site.  BEMPOL_ERR_NOT_CONVERGED if any
 * system did not converge (results filled). */
bempol_status bempol_solve_systems(bempol_ctx* c, void* stream, bempol_result* out, bempol_system_result* per,
                                   int64_t n_per);

/* Adjoint gradient (not part of the paper's method: its derivatives with respect
 * to the site parameters, for force fields and fitting).  Uses the state of the
 * last bempol_solve / bempol_solve_systems on this context (mesh, sites and
 * parameters unchanged since; BEMPOL_ERR_STATE otherwise).  The energy of Eq.
 * energy_multipole_polarizable is not stationary in the induced dipoles, so the
 * gradient is the full discrete adjoint: one transposed BEM system A^T lambda = c
 * per step of a transposed induced-dipole relaxation (same omega, scf_tol and
 * scf_maxit; GMRES with params.op / residual_op applied as transposed products),
 * the same without BEM for the vacuum state, then per-site fields and,
 * for positions, their derivatives (dual numbers, no differencing).
 * Outputs (device float64, caller's site order, NULL to skip):
 *   grad_q [ns]   dDelta G_solv/dq_l,   grad_d [ns*3] dDelta G_solv/dd_l,
 *   grad_Q [ns*9] dDelta G_solv/dQ_l as the symmetric traceless 3x3 matrix G with
 *                 dDelta G = sum_l G_l : dQ_l for symmetric traceless dQ_l,
 *   grad_pos [ns*3] dDelta G_solv/dr_l with the mesh held fixed (the surface does
 *                 not follow the sites).
 * Units: `units` = BEMPOL_UNITS_PAPER gives paper units (e^2/A per e, per e*A, per
 * e*A^2, per A); BEMPOL_UNITS_KCAL gives kcal/mol per the same (the paper units times
 * 4 pi 332.0637133, as dG_solv_kcal).  With several systems each site's gradient is that
 * of its own system's Delta G_solv.  info (host, may be NULL) receives iteration
 * counts and the event time.  BEMPOL_ERR_NOT_CONVERGED if a limit was hit (outputs
 * written).  Synchronises `stream`. */
typedef struct {
  int scf_iters_diss, scf_iters_vac;  /* transposed relaxation steps */
  int gmres_iters_total;              /* GMRES iterations of the transposed solves */
  int n_solves;                       /* transposed BEM solves */
  int converged;
  double t_ms;
} bempol_gradient_info;

enum { BEMPOL_UNITS_PAPER = 0, BEMPOL_UNITS_KCAL = 1 };

bempol_status bempol_gradient(bempol_ctx* c, void* stream, double* grad_q, double* grad_d, double* grad_Q,
                              double* grad_pos, bempol_gradient_info* info, int units);

/* y = A x for the operator form `op` (BEMPOL_OP_*), one matrix-vector product of
 * Eq. integral_eq.  x, y: device float64 [2N] = [phi; psi] in the caller's panel
 * order (y may not alias x).  Enqueued on `stream`, no synchronisation. */
bempol_status bempol_matvec(bempol_ctx* c, const double* x, double* y, int op, void* stream);

/* y = A^T x, the transpose of the operator of bempol_matvec (used by the adjoint;
 * the paper has no counterpart): charges x_phi (Laplace) and x_psi (Yukawa) at the
 * collocation points evaluated at every panel's Gauss nodes, plus the near
 * corrections by columns.  BEMPOL_OP_FP32_TREE uses the same octree and lists
 * with charge moments of order 4 whatever params.order (the nodes' potential
 * gradient takes coefficients to order 5); BEMPOL_OP_FP64_TREE is applied as
 * BEMPOL_OP_FP64_DIRECT.
 * x, y: device float64 [2N] in the caller's order (y may not alias x).  Enqueued
 * on `stream`, no synchronisation. */
bempol_status bempol_matvec_transposed(bempol_ctx* c, const double* x, double* y, int op, void* stream);

/* Right-hand side of Eq. rhs_multipole at every collocation point, with the
 * sites' q and Q and the total dipoles p (device float64 [ns*3]; NULL = the
 * permanent d).  b: device float64 [N] (caller order).  `op` selects FP64
 * (BEMPOL_OP_FP64_*) or FP32-pair/FP64-sum arithmetic.  Enqueued on `stream`. */
bempol_status bempol_rhs(bempol_ctx* c, const double* p, double* b, int op, void* stream);

/* Reaction potential, field gradient and Hessian at the sites from a surface
 * solution x = [phi; psi] (device float64 [2N], caller order) (Eqs. pot_solvent,
 * Efield_solv, ddphi): out [ns*10] device float64, per site phi_solv,
 * dphi/dx,dy,dz, then d2phi xx,xy,xz,yy,yz,zz.  K-node quadrature over every
 * panel of the site's own body (sites are validated to be far from the surface).
 * Enqueued on `stream`. */
bempol_status bempol_site_reaction(bempol_ctx* c, const double* x, double* out, int op, void* stream);

/* Same result as bempol_site_reaction, for callers that cannot allow a device
 * allocation during the call (the paper has no counterpart: this is a property
 * of the library, not of the method).  bempol_site_reaction may cudaMalloc its
 * partial-sum buffer when it grows; this variant calls no cudaMalloc, cudaFree or
 * other allocating routine.  Use it where another runtime owns the device memory
 * pool, or in loops that cannot take an allocation's implicit synchronisation.
 *   x   device float64 [2N] (caller order), out device float64 [ns*10] as above.
 * Limit: at most 26,214 sites (its partial sums live in one fixed 2 MiB
 * file-scope device array that every GPU loading the library keeps until
 * process exit); more sites give BEMPOL_ERR_ARG.  The array is shared by every
 * call on every context: calls that overlap on the GPU race.  Each call writes
 * every scratch entry it reads, so nothing carries over between calls.  The
 * first call on a device looks up the array's device address (one-time set-up,
 * cached for the process); that lookup may make the CUDA driver load this
 * library's device code, which allocates inside the driver, so make the first
 * call early (before any stream capture and before the allocation-free phase).
 * After a cudaDeviceReset neither contexts nor the cached address are valid.
 * Other errors as bempol_site_reaction.  Enqueued on `stream`. */
bempol_status bempol_site_reaction_noalloc(bempol_ctx* c, const double* x, double* out, int op, void* stream);

/* Multipole-multipole potentials at the sites (Eqs. Efield_mult,
 * second_derivative) with induced dipoles mu (device float64 [ns*3], NULL = 0):
 *   mode 0 (polarising field): permanent moments of the same polarisation group
 *          are masked, induced dipoles Thole-damped; out [ns*3] = E (field).
 *   mode 1 (energy): permanent moments unmasked, induced dipoles damped;
 *          out [ns*10] = phi, grad phi (3), Hessian (6) as in bempol_site_reaction.
 *   Modes 0 and 1 sum over the sites of each site's own body (dissolved state);
 *   modes 2 and 3 are modes 0 and 1 summed over every site of its system (vacuum).
 * FP64.  Enqueued on `stream`. */
bempol_status bempol_multipole_field(bempol_ctx* c, const double* mu, int mode, double* out, void* stream);

/* Autotuner of the treecode (not a step of the paper's method): for the current mesh,
 * times the FP32 treecode product (CUDA events, mean of 3 after a warm-up) for every
 * leaf in {128, 192, 256, 384}, theta in {0.4, 0.5, 0.6} and order in {4, 5, 6}, measures
 * its error ||y - y_ref|| / ||y_ref|| against the FP32 direct product y_ref on a fixed
 * pseudo-random vector, and keeps in the context's parameters the fastest candidate
 * whose error is <= target_err (the tree is rebuilt for it).  `out` (host, may be
 * NULL) receives the choice, its time and error and the number of candidates.
 * BEMPOL_ERR_NOT_CONVERGED (parameters unchanged) if no candidate reaches the target.
 * Synchronises `stream`. */
typedef struct {
  int leaf;
  double theta;
  int order;
  double matvec_ms;   /* FP32 treecode product time of the choice */
  double rel_err;     /* its error against the FP32 direct product */
  int candidates;
} bempol_tune_result;

bempol_status bempol_autotune(bempol_ctx* c, double target_err, bempol_tune_result* out, void* stream);

/* Sizes of the library's tables: number of panels, Gauss nodes per panel,
 * sites, near pairs, treecode cells and leaves (any pointer may be NULL). */
bempol_status bempol_sizes(const bempol_ctx* c, int64_t* n_panels, int32_t* gauss_k, int64_t* n_sites,
                           int64_t* n_near, int64_t* n_cells, int64_t* n_leaves);

/* Kernel accounting (not part of the method; for measurement).  When enabled,
 * the pair kernels (direct or treecode near field), the treecode far-field
 * kernels, whole treecode products and the right-hand sides, reaction fields and
 * multipole fields of bempol_solve* are bracketed by CUDA events on their launch
 * stream; bempol_stats_read synchronises the device and reports the summed event
 * times.  In a treecode product the near-field kernel runs concurrently with the
 * moment, M2M and far-field kernels (these on a side stream of the context), so
 * pair_ms and far_ms then overlap and tree_ms (fork to join on the caller's stream)
 * is the product's own duration.  Products with the FP64 treecode are counted apart
 * (tree64_*), so the pair/far/tree counters describe the FP32 treecode alone. */
typedef struct {
  int64_t kernel_launches;     /* kernels this library launched (all contexts) since the last reset */
  int64_t pair_launches;       /* launches of the pair kernel */
  double pair_ms;              /* summed CUDA-event time of those launches (0 unless enabled) */
  int64_t far_launches;        /* launches of the treecode far-field kernel */
  double far_ms;
  int64_t pair_interactions;   /* (target, Gauss node) pairs evaluated by the pair kernels */
  int64_t far_evaluations;     /* (target, cell) Taylor evaluations of the far-field kernel */
  int64_t tree_products;       /* treecode products (forward or transposed) */
  double tree_ms;              /* summed CUDA-event time of those products, fork to join */
  int64_t rhs_calls;           /* right-hand sides evaluated inside bempol_solve* */
  double rhs_ms;
  int64_t reaction_calls;      /* reaction fields at the sites inside the induced-dipole iteration */
  double reaction_ms;
  int64_t site_field_calls;    /* multipole fields at the sites inside the induced-dipole iterations */
  double site_field_ms;
  /* host wall-clock of the last bempol_set_mesh*, by phase (the stream is synchronised at each
     phase boundary while timing is enabled): closedness check, panel geometry and Morton
     order, block tables, octree and interaction lists, near table and its integrals */
  double mesh_validate_ms, mesh_geometry_ms, mesh_blocks_ms, mesh_tree_ms, mesh_near_ms;
  /* FP64 treecode products (BEMPOL_OP_FP64_TREE, e.g. the refinement residuals), fork to
     join; the pair, far and tree counters above cover the FP32 treecode only */
  int64_t tree64_products;
  double tree64_ms;
} bempol_stats;

/* Arithmetic-pipe throughput of a device (measurement support, not part of the
 * method): the treecode and direct pair kernels are bound by the FP32 FMA pipe and
 * the special-function unit (rsqrt, 2^x), the FP64 direct form by the FP64 FMA
 * pipe, so these are the peaks their roofline fractions divide by.  Each rate comes
 * from a kernel of independent dependency chains of one PTX instruction
 * (fma.rn.f32, fma.rn.f64, rsqrt.approx.ftz.f32, ex2.approx.ftz.f32) over SMs x 8
 * blocks x 256 threads, timed with CUDA events on the legacy default stream (best
 * of `reps` after one warm-up launch).  `iters` sets the FP32 chain length (the
 * FP64 chains run iters/8 + 1 steps, the MUFU chains iters/4 + 1); 65,536 gives
 * launches of a few milliseconds.  FMA counts as two flops.  The rates hold at
 * the SM clock of the run, which the attribute below does not report (it is the
 * device's nominal maximum): sample the clock alongside.  Synchronises the device's
 * default stream.  BEMPOL_ERR_ARG / BEMPOL_ERR_CUDA. */
typedef struct {
  double fp32_fma_tflops;      /* FP32 FMA throughput, TFLOP/s */
  double fp64_fma_tflops;      /* FP64 FMA throughput, TFLOP/s */
  double mufu_rsqrt_gops;      /* rsqrt.approx.f32 per second / 1e9 */
  double mufu_ex2_gops;        /* ex2.approx.f32 per second / 1e9 */
  double ms_fp32, ms_fp64, ms_rsqrt, ms_ex2;   /* best launch time of each kernel */
  int sm_count;
  double clock_mhz_attr;       /* cudaDevAttrClockRate (maximum SM clock) */
} bempol_peaks;

bempol_status bempol_measure_peaks(int device, int iters, int reps, bempol_peaks* out);

/* The 19-node triangle rule used by near_rule = BEMPOL_NEAR_GAUSS19 (Sec. "Comparison with
 * Tinker-APBS": 19 Gauss nodes for near pairs): the fully symmetric rule of degree 9, solved
 * on the host from its moment equations.  Writes 19 x 4 doubles to host memory `nodes`
 * (caller-owned): barycentric coordinates l1, l2, l3 and the weight (weights sum to 1;
 * node 0 is the centroid).  Host only: needs no device or context.
 * BEMPOL_ERR_ARG (NULL) / BEMPOL_ERR_NOT_CONVERGED (the solve failed). */
bempol_status bempol_near_rule19(double* nodes);

/* The table from which the treecode forms each cell's far-field coefficients at Taylor
 * order `order` (1..6; Sec. "The treecode algorithm", Cartesian Taylor expansion of the
 * Laplace and Yukawa kernels about the cell centre).  With a cell's moments X_k in the
 * order k = (a, b, n - a - b) for n = 0..P, a = n..0, b = n - a..0, its coefficient of
 * entry q is  B_q = sum_{u = ptr[q]}^{ptr[q+1]-1} coef[u] * X_{moment[u]},  and the far
 * potential of the cell at Delta = x - c is  sum_m g_m(|Delta|) sum_e Delta^e B_{(m, e)}
 * with g_m = (1/r d/dr)^m G.  Entries run over the monomial exponents e = (a, b, c) in
 * the order a, then b, then c ascending, |e| <= P, and within one e over m = |e| ..
 * floor((P + |e|) / 2).  Call with NULL arrays to get *n_entries (NB) and *n_terms, then
 * with caller-owned host arrays ptr [NB + 1], moment [n_terms] and coef [n_terms].  Host
 * only: needs no device or context.  BEMPOL_ERR_ARG: order outside 1..6 or a NULL count. */
bempol_status bempol_far_coefficients(int order, int64_t* n_entries, int64_t* n_terms, int32_t* ptr,
                                      int32_t* moment, double* coef);

/* Target sharding over several GPUs (Sec. "The treecode algorithm": the source-target
 * and box-target interactions of different targets are independent).  Each GPU holds
 * the whole mesh, sites and sources in its own context and computes only the rows of
 * its rank: a contiguous range of the library's internal (Morton) panel order, cut at
 * target-batch boundaries so that the treecode work (near pairs plus weighted far
 * terms) is balanced.  After every treecode product the rows are exchanged through a
 * caller-supplied all-gather, and everything else (GMRES with its Arnoldi process,
 * induced dipoles, energies) runs redundantly on every rank with identical results.
 *
 * bempol_shard_rows: host only (no device work).  Split n_units consecutive units
 * with costs cost[n_units] (NULL = 1 each, every cost >= 0) into `world` contiguous
 * ranges of nearly equal cost: bounds[world+1] (host int64) with bounds[0] = 0,
 * bounds[world] = n_units, nondecreasing; range r = [bounds[r], bounds[r+1]).  Cut r
 * is the unit boundary whose cost prefix is nearest to r/world of the total (ties to
 * the earlier one; a zero total gives equal unit counts).  BEMPOL_ERR_ARG on NULL
 * bounds, n_units < 0, world < 1 or a negative cost. */
bempol_status bempol_shard_rows(int64_t n_units, const double* cost, int world, int64_t* bounds);

/* Exchange callback: called by the library on its host thread after this rank's rows
 * of a product are in the exchange buffer; it must fill every other rank's rows (of
 * both halves, phi rows [0, N) and psi rows [N, 2N), internal order) with theirs, with
 * the copies ordered on `stream` (e.g. an NCCL all-gather), and return.  bounds
 * [world+1] (host, valid during the call) are the row bounds of every rank.  The
 * callback must not call into the same context. */
typedef void (*bempol_exchange_fn)(void* user, const int64_t* bounds, int world, void* stream);

/* Make this context rank `rank` of `world` for every treecode product (forward,
 * BEMPOL_OP_FP32_TREE and BEMPOL_OP_FP64_TREE; direct forms and the transposed
 * product compute every row).  exchange_buf: caller-owned device float64 [2N], kept
 * until the sharding is replaced or the context destroyed; each product copies its
 * result there (internal order), calls fn(user, stream) and copies it back.
 * world = 1 (fn and exchange_buf may be NULL) turns sharding off.  Rebuilt with the
 * tree (bempol_set_mesh, theta or leaf changes).  Requires a mesh (BEMPOL_ERR_STATE);
 * BEMPOL_ERR_ARG on a bad rank/world or NULL fn/buffer with world > 1. */
bempol_status bempol_set_shard(bempol_ctx* c, int rank, int world, double* exchange_buf, bempol_exchange_fn fn,
                               void* user);

/* Row bounds of the current sharding in internal panel order (host int64 [world+1];
 * bounds[world] = N).  Builds the tree if needed.  BEMPOL_ERR_STATE without a mesh. */
bempol_status bempol_shard_bounds(bempol_ctx* c, int64_t* bounds);

/* Turn event timing on (1) or off (0).  Counting is always on. */
bempol_status bempol_stats_enable(bempol_ctx* c, int enable);

/* Read the counters (host struct); reset = 1 zeroes them afterwards. */
bempol_status bempol_stats_read(bempol_ctx* c, bempol_stats* out, int reset);

/* Copy out the geometry and the near-field table, in the caller's order (host
 * pointers, any may be NULL): centroid [N*3], normal [N*3], area [N];
 * near_ptr [N+1] int64 (CSR rows), near_col [n_near] int32 (ascending per row),
 * near_corr [n_near*4] float64 per pair (V_L, K_L, V_Y, K_Y) of
 * (semi-analytical - K-node) integrals including 1/(4 pi).  Synchronises. */
bempol_status bempol_get_geometry(bempol_ctx* c, double* centroid, double* normal, double* area,
                                  int64_t* near_ptr, int32_t* near_col, double* near_corr);

#ifdef __cplusplus
}
#endif

#endif /* BEMPOL_H */
