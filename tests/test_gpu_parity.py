"""GPU parity: every C-ABI entry point against the FP64 oracle, element by element.

Bars (derived in the design notes from the arithmetic of each path):
  * integer/index work (near-pair lists): bit-exact;
  * geometry formed with separately rounded FP64 operations: bit-exact;
  * FP64 kernels: relative 1e-12 of the largest entry (rounding-order only);
  * FP32-pair kernels (FP32 tiles, FP64 sums): relative 2e-5 of the largest entry;
  * Delta G_solv of the FP64 direct solve: 1e-10 relative.
Cases span several 128-target tiles with a ragged tail (1,280 and 5,120 panels,
40 and 2 sites) plus the K = 1 / 3 Gauss rules and kappa = 0.
"""
import numpy as np
import pytest

import gen
from oracle import bem, geometry, multipole as mp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_1810_03698_gb300 as mod
    return mod


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


CASES = {
    "sphere1280": lambda: gen.sphere_r4_1280(),
    "bumpy1280": lambda: gen.small_bumpy(3, 40, 8.0),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, bp):
    pr = CASES[request.param]()
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    s = bp.problem_solver(pr)
    return pr, mesh, s


def test_geometry_bit_exact(case):
    pr, mesh, s = case
    g = s.geometry()
    assert np.array_equal(g["centroid"], mesh.cen)
    assert np.array_equal(g["area"], mesh.area)
    assert np.array_equal(g["normal"], mesh.normal)
    assert np.array_equal(g["near_ptr"], mesh.near_ptr)
    assert np.array_equal(g["near_col"], mesh.near_cols)


def test_near_corrections(case):
    pr, mesh, s = case
    g = s.geometry()
    ref = np.stack(bem.near_correction(mesh, pr.params.kappa), axis=1)
    # corrections are differences of O(1/(4 pi) sqrt(A)) integrals; compare per kernel
    for k in range(4):
        assert _relmax(g["near_corr"][:, k], ref[:, k]) < 1e-12, k


@pytest.fixture(scope="module")
def dense(case):
    pr, mesh, s = case
    par = pr.params
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    return A


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_matvec(case, dense, op, tol):
    pr, mesh, s = case
    rng = np.random.default_rng(5)
    x = rng.normal(size=2 * mesh.n)
    y = torch.zeros(2 * mesh.n, dtype=torch.float64, device="cuda")
    s.matvec(_dev(x), y, op=op)
    torch.cuda.synchronize()
    ref = dense @ x
    assert _relmax(y.cpu().numpy(), ref) < tol


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-13), ("fp32_direct", 2e-5)])
def test_rhs(case, op, tol):
    pr, mesh, s = case
    st = pr.sites
    rng = np.random.default_rng(6)
    p = st.d + rng.normal(size=st.d.shape) * 0.1
    b = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    s.rhs(b, p=_dev(p), op=op)
    torch.cuda.synchronize()
    ref = mp.rhs(mesh.cen, st.pos, st.q, p, st.Q, pr.params.eps_in)
    assert _relmax(b.cpu().numpy(), ref) < tol


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_site_reaction(case, op, tol):
    pr, mesh, s = case
    rng = np.random.default_rng(7)
    x = rng.normal(size=2 * mesh.n)
    out = torch.zeros(pr.sites.n * 10, dtype=torch.float64, device="cuda")
    s.site_reaction(_dev(x), out, op=op)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 10)
    pot, grad, hess = mp.reaction_at_sites(mesh, x[:mesh.n], x[mesh.n:], pr.sites.pos)
    iu = np.triu_indices(3)
    assert _relmax(o[:, 0], pot) < tol
    assert _relmax(o[:, 1:4], grad) < tol
    assert _relmax(o[:, 4:], hess[:, iu[0], iu[1]]) < tol


def test_multipole_field(case):
    pr, mesh, s = case
    st = pr.sites
    rng = np.random.default_rng(8)
    mu = rng.normal(size=(st.n, 3)) * 0.2
    E = torch.zeros(st.n * 3, dtype=torch.float64, device="cuda")
    s.multipole_field(E, mu=_dev(mu), mode=0)
    F = torch.zeros(st.n * 10, dtype=torch.float64, device="cuda")
    s.multipole_field(F, mu=_dev(mu), mode=1)
    torch.cuda.synchronize()
    par = pr.params
    _, g, _ = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                 par.thole_a, masked=True, same_body_only=True)
    assert _relmax(E.cpu().numpy().reshape(-1, 3), -g) < 1e-12
    P, G, H = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                 par.thole_a, masked=False, same_body_only=True)
    f = F.cpu().numpy().reshape(-1, 10)
    iu = np.triu_indices(3)
    assert _relmax(f[:, 0], P) < 1e-12
    assert _relmax(f[:, 1:4], G) < 1e-12
    assert _relmax(f[:, 4:], H[:, iu[0], iu[1]]) < 1e-12


def _tight(pr):
    return gen.with_params(pr, gmres_tol=1e-13, scf_tol=1e-12, scf_maxit=400)


@pytest.mark.parametrize("name", list(CASES))
def test_solvation_fp64_direct_matches_oracle(bp, name):
    pr = _tight(CASES[name]())
    ref = mp.solvation(pr, direct_polarization=True)
    s = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    out = s.solve(outputs=True)
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-10 * abs(ref.dG_kcal)
    assert abs(out["G_vac"] - (ref.G_vac)) < 1e-10 * abs(ref.G_vac)
    assert _relmax(out["mu_diss"].reshape(-1, 3), ref.mu_diss) < 1e-9
    assert _relmax(out["mu_vac"].reshape(-1, 3), ref.mu_vac) < 1e-9
    assert _relmax(out["phi"], ref.phi) < 1e-9
    assert _relmax(out["dphidn"], ref.psi) < 1e-9


def test_sor_iterations_match_oracle_sor(bp):
    """Same SCF recursion (mu = 0, SOR w = 0.7, RMS test) gives the same iteration counts."""
    pr = gen.with_params(gen.sphere_r4_1280(), gmres_tol=1e-13)
    ref = mp.solvation(pr)
    s = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    out = s.solve()
    assert out["scf_iters_vac"] == ref.scf_iters_vac
    assert abs(out["scf_iters_diss"] - ref.scf_iters_diss) <= 1
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-9 * abs(ref.dG_kcal)


def test_fp32_direct_with_fp64_refinement(bp):
    """FP32 pair kernels inside GMRES, FP64 residual and site kernels: FP64-level result."""
    pr = _tight(gen.sphere_r4_1280())
    ref = mp.solvation(pr, direct_polarization=True)
    s = bp.problem_solver(pr, op="fp32_direct", residual_op="fp64_direct", inner_tol=1e-4)
    out = s.solve()
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-10 * abs(ref.dG_kcal)


def test_fp32_direct_plain(bp):
    pr = gen.with_params(gen.sphere_r4_1280(), gmres_tol=1e-7, scf_tol=1e-8)
    ref = mp.solvation(pr, direct_polarization=True)
    s = bp.problem_solver(pr, op="fp32_direct", residual_op="fp32_direct")
    out = s.solve()
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-5 * abs(ref.dG_kcal)


@pytest.mark.parametrize("k,kappa", [(1, 0.125), (3, 0.0), (4, 0.0)])
def test_other_rules_and_no_salt(bp, k, kappa):
    pr = gen.small_bumpy(2, 12, 6.0)
    pr = gen.with_params(pr, gauss_k=k, kappa=kappa, gmres_tol=1e-13, scf_tol=1e-12)
    ref = mp.solvation(pr, direct_polarization=True)
    s = bp.problem_solver(pr)
    out = s.solve()
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-10 * abs(ref.dG_kcal)


def test_reruns_are_bit_identical(bp):
    pr = gen.small_bumpy(3, 20, 8.0)
    s = bp.problem_solver(pr, op="fp32_direct", residual_op="fp64_direct")
    a = s.solve(outputs=True)
    b = s.solve(outputs=True)
    assert a["dG_solv_kcal"] == b["dG_solv_kcal"]
    assert np.array_equal(a["phi"], b["phi"])
