"""GPU parity of the adjoint: the transposed operator and the moment gradient.

* A^T u against the oracle's dense matrix transposed (FP64 rounding-order bar
  1e-12, FP32 pairs 2e-5 of the largest entry), one and two bodies.
* dDelta G_solv/d(q, d, Q, r) of the adjoint against the oracle's derivative
  (five-point differences at the exact fixed point: exact for the quadratic moment
  dependencies up to rounding; for positions the h^4 truncation at h = 1e-3 A and
  the rounding of the differences are below 1e-10 relative), with GMRES and SCF
  run to 1e-12: bar 1e-8 of the largest entry.  Euler's identity sum_l m_l . g_l = 2 Delta G_solv on the GPU
  result alone.  The FP32 operator with FP64 refinement: bar 1e-6.
"""
import numpy as np
import pytest

import gen
from oracle import bem
from oracle import gradient as og

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


PROBLEMS = {
    "bumpy320": lambda: gen.small_bumpy(2, 6, 8.0, seed_index=105),
    "complex640": lambda: gen.small_triple(seed_index=421, subdiv=2, radius=7.0, n_sites=6, gap=1.0)[2],
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def prob(request):
    pr = PROBLEMS[request.param]()
    return request.param, gen.with_params(pr, gmres_tol=1e-12, scf_tol=1e-12, scf_maxit=400)


@pytest.mark.parametrize("op,bar", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_transposed_matvec(bp, prob, op, bar):
    _, pr = prob
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor, body=pr.panel_body)
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    s = bp.problem_solver(pr)
    u = np.random.default_rng(31).normal(size=2 * mesh.n)
    y = torch.zeros(2 * mesh.n, dtype=torch.float64, device="cuda")
    s.matvec_transposed(_dev(u), y, op=op)
    assert _relmax(y.cpu().numpy(), A.T @ u) < bar


def _sample(pr):
    n = pr.sites.n
    return np.array(sorted({0, n // 2, n - 1}))


@pytest.mark.parametrize("theta,bar", [(1e-3, 2e-5), (0.5, 5e-4)])
def test_transposed_tree(bp, theta, bar):
    """FP32 treecode A^T u (order 4): theta -> 0 reduces it to the FP32 direct sum; at
    theta = 0.5 it is within the forward treecode's bar of the dense A^T u."""
    pr = gen.small_bumpy(3, 8, 8.0, seed_index=108)
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    s = bp.problem_solver(pr, leaf=32, theta=theta, order=5)
    u = np.random.default_rng(32).normal(size=2 * mesh.n)
    y = torch.zeros(2 * mesh.n, dtype=torch.float64, device="cuda")
    s.matvec_transposed(_dev(u), y, op="fp32_tree")
    assert s.sizes()["n_leaves"] > 8
    assert _relmax(y.cpu().numpy(), A.T @ u) < bar


@pytest.fixture(scope="module")
def oracle_grad(prob):
    """Oracle derivatives for three sites (first, middle, last: both bodies of the complex)."""
    name, pr = prob
    return og.solvation_gradient(pr, sites_idx=_sample(pr))


def test_moment_gradient_fp64(bp, prob, oracle_grad):
    _, pr = prob
    s = bp.problem_solver(pr)
    r = s.solve()
    assert r["G_diss"] - r["G_vac"] == pytest.approx(oracle_grad["dG"], rel=1e-10)
    g = s.gradient()
    assert g["info"]["converged"] == 1
    idx = _sample(pr)
    for k in ("q", "d", "Q", "pos"):
        assert _relmax(g[k][idx], oracle_grad[k]) < 1e-8, k
    st = pr.sites
    euler = np.sum(st.q * g["q"]) + np.sum(st.d * g["d"]) + np.sum(st.Q * g["Q"])
    assert euler == pytest.approx(2.0 * (r["G_diss"] - r["G_vac"]), rel=1e-9)


def test_moment_gradient_fp32_refined(bp, prob, oracle_grad):
    _, pr = prob
    s = bp.problem_solver(pr, op="fp32_direct", residual_op="fp64_direct")
    s.solve()
    g = s.gradient()
    idx = _sample(pr)
    for k in ("q", "d", "Q", "pos"):
        assert _relmax(g[k][idx], oracle_grad[k]) < 1e-6, k


def test_moment_gradient_tree(bp, prob, oracle_grad):
    """FP32 treecode forward and transposed solves with FP64 direct refinement."""
    _, pr = prob
    s = bp.problem_solver(pr, op="fp32_tree", residual_op="fp64_direct", leaf=32, theta=0.5, order=5)
    s.solve()
    g = s.gradient()
    idx = _sample(pr)
    for k in ("q", "d", "Q", "pos"):
        assert _relmax(g[k][idx], oracle_grad[k]) < 1e-6, k


def test_autograd_function(bp, prob, oracle_grad):
    """torch.autograd through solvation_energy: backward = the adjoint gradient in kcal/mol."""
    _, pr = prob
    if pr.panel_body is not None:
        pytest.skip("single-body problems only (the helper sets sites without bodies)")
    s = bp.problem_solver(pr)
    st = pr.sites
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").requires_grad_(True)
    pos, q, d, Q = dev(st.pos), dev(st.q), dev(st.d), dev(st.Q)
    alpha = torch.as_tensor(st.alpha, dtype=torch.float64, device="cuda")
    group = torch.as_tensor(st.group, dtype=torch.int32, device="cuda")
    G = bp.solvation_energy(s, pos, q, d, Q, alpha, group)
    G.backward()
    assert G.item() == pytest.approx(oracle_grad["dG"] * bp.KCAL_PER_UNIT, rel=1e-10)
    idx = _sample(pr)
    for k, t in (("pos", pos), ("q", q), ("d", d), ("Q", Q)):
        got = t.grad.cpu().numpy()[idx] / bp.KCAL_PER_UNIT
        assert _relmax(got, oracle_grad[k]) < 1e-8, k


def test_gradient_needs_a_solve(bp):
    pr = gen.small_bumpy(2, 3, 8.0, seed_index=107)
    s = bp.problem_solver(pr)
    with pytest.raises(bp.BempolError) as e:
        s.gradient()
    assert e.value.status == 8


@pytest.mark.parametrize("op,bar", [("fp64_direct", 1e-12), ("fp32_tree", 2e-4)])
def test_adjoint_identity_fullsize(bp, op, bar):
    """<y, A x> = <A^T y, x> on the 20,480-panel sphere with 100 sites: to rounding for
    the direct form; for the treecode the two products are separate approximations, each
    within the treecode's error."""
    pr = gen.sphere_r10_20480()
    s = bp.problem_solver(pr, theta=0.5, order=5)
    n = pr.n_panels
    g = np.random.default_rng(34)
    x = _dev(g.normal(size=2 * n))
    y = _dev(g.normal(size=2 * n))
    ax = torch.zeros_like(x)
    aty = torch.zeros_like(x)
    s.matvec(x, ax, op=op)
    s.matvec_transposed(y, aty, op=op)
    lhs = float(torch.dot(y, ax))
    rhs = float(torch.dot(aty, x))
    scale = float(torch.linalg.norm(y) * torch.linalg.norm(ax))
    assert abs(lhs - rhs) <= bar * scale


def test_gradient_units_kcal(bp):
    """units="kcal" is the paper-unit gradient times 4 pi 332.0637 (the library scales)."""
    pr = gen.sphere_r4_1280()
    s = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    s.solve()
    a = s.gradient()
    b = s.gradient(units="kcal")
    for k in ("q", "d", "Q", "pos"):
        assert np.allclose(b[k], a[k] * bp.KCAL_PER_UNIT, rtol=1e-12, atol=0.0), k
    s.close()
