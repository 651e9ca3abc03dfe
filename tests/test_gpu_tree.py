"""Treecode parity (Sec. "The treecode algorithm") against the FP64 oracle.

The treecode approximates the discrete operator, so the checks are the ones
the approximation fixes: the error against the oracle's dense product falls
with the Taylor order P and with theta, theta -> 0 reproduces the direct sum,
and Delta G_solv stays within 1e-4 relative of the oracle at theta = 0.5, P = 5.
Meshes of 1,280 and 5,120 panels with small leaves give trees of several levels.
"""
import numpy as np
import pytest

import gen
from oracle import bem, multipole as mp

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


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def mid(bp):
    pr = gen.small_bumpy(4, 30, 10.0, seed_index=104)
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    s = bp.problem_solver(pr, leaf=64)
    rng = np.random.default_rng(11)
    x_rand = rng.normal(size=2 * mesh.n)
    c = mesh.cen / np.linalg.norm(mesh.cen, axis=1).max()
    x_smooth = np.concatenate([np.sin(2 * c[:, 0]) + c[:, 1] * c[:, 2], np.cos(3 * c[:, 2]) - c[:, 0]])
    return pr, mesh, A, s, {"random": x_rand, "smooth": x_smooth}


def _apply(s, x, op):
    y = torch.zeros(x.size, dtype=torch.float64, device="cuda")
    s.matvec(torch.tensor(x, device="cuda"), y, op=op)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("kind", ["random", "smooth"])
def test_error_falls_with_order(mid, kind):
    pr, mesh, A, s, xs = mid
    x = xs[kind]
    ref = A @ x
    errs = []
    for P in (1, 3, 5):
        s.set_params(order=P, theta=0.5)
        errs.append(_relmax(_apply(s, x, "fp64_tree"), ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-4
    s.set_params(order=5)
    e32 = _relmax(_apply(s, x, "fp32_tree"), ref)
    assert e32 < 2e-4


def test_error_falls_with_theta(mid):
    pr, mesh, A, s, xs = mid
    x = xs["smooth"]
    ref = A @ x
    errs = []
    for th in (0.8, 0.5, 0.3):
        s.set_params(order=4, theta=th)
        errs.append(_relmax(_apply(s, x, "fp64_tree"), ref))
    assert errs[0] > errs[1] > errs[2]


def test_small_theta_is_the_direct_sum(mid):
    pr, mesh, A, s, xs = mid
    x = xs["random"]
    ref = A @ x
    s.set_params(order=3, theta=1e-3)
    assert _relmax(_apply(s, x, "fp64_tree"), ref) < 1e-12
    assert s.sizes()["n_leaves"] > 8
    assert _relmax(_apply(s, x, "fp32_tree"), ref) < 2e-5
    s.set_params(theta=0.5, order=5)


@pytest.mark.parametrize("leaf", [16, 48])
def test_tree_solvation_within_1e4(bp, leaf):
    pr = gen.with_params(gen.small_bumpy(3, 40, 8.0), gmres_tol=1e-7, scf_tol=1e-7)
    ref = mp.solvation(pr, direct_polarization=True)
    for op in ("fp32_tree", "fp64_tree"):
        s = bp.problem_solver(pr, op=op, residual_op=op, theta=0.5, order=5, leaf=leaf)
        out = s.solve()
        assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-4 * abs(ref.dG_kcal), op


def test_fp32_tree_with_fp64_tree_refinement(bp):
    pr = gen.with_params(gen.small_bumpy(3, 40, 8.0), gmres_tol=1e-10, scf_tol=1e-10)
    s32 = bp.problem_solver(pr, op="fp32_tree", residual_op="fp64_tree", inner_tol=1e-3, leaf=32)
    s64 = bp.problem_solver(pr, op="fp64_tree", residual_op="fp64_tree", leaf=32)
    a = s32.solve()
    b = s64.solve()
    # refinement converges to the FP64 tree operator's solution
    assert abs(a["dG_solv_kcal"] - b["dG_solv_kcal"]) < 1e-8 * abs(b["dG_solv_kcal"])


@pytest.mark.parametrize("op,res_op,leaf", [("fp32_tree", "fp64_tree", 32), ("fp32_direct", "fp64_direct", 256)])
def test_refine_final_solve_only(bp, op, res_op, leaf):
    """refine_scope "final": the induced-dipole iteration solves with the FP32 form alone
    (to max(gmres_tol, 1e-6)), and only the last solve, which gives the energy, is refined
    against the FP64 form to gmres_tol.  Delta G matches the oracle within the treecode
    bar and the fully refined form within the SCF's own accuracy."""
    pr = gen.with_params(gen.small_bumpy(3, 40, 8.0), gmres_tol=1e-9, scf_tol=1e-7)
    ref = mp.solvation(pr, direct_polarization=True)
    fin = bp.problem_solver(pr, op=op, residual_op=res_op, refine_scope="final", leaf=leaf).solve()
    every = bp.problem_solver(pr, op=op, residual_op=res_op, refine_scope="every", leaf=leaf).solve()
    assert fin["residual_matvecs"] >= 1 and fin["last_rel_residual"] < 1e-9
    assert every["residual_matvecs"] > fin["residual_matvecs"]
    assert abs(fin["dG_solv_kcal"] - ref.dG_kcal) < 1e-4 * abs(ref.dG_kcal)
    assert abs(fin["dG_solv_kcal"] - every["dG_solv_kcal"]) < 1e-5 * abs(every["dG_solv_kcal"])
    if op == "fp32_direct":   # the direct forms approximate nothing: FP64-level agreement
        assert abs(every["dG_solv_kcal"] - ref.dG_kcal) < 1e-7 * abs(ref.dG_kcal)


def test_autotune_meets_its_target(bp):
    """The autotuner's choice reproduces the direct product within the target."""
    pr = gen.small_bumpy(4, 10, 8.0, seed_index=109)
    s = bp.problem_solver(pr)
    r = s.autotune(target_err=1e-4)
    assert r["candidates"] == 36 and 0 <= r["rel_err"] <= 1e-4
    assert (s.params.leaf, s.params.theta, s.params.order) == (r["leaf"], r["theta"], r["order"])
    n = pr.n_panels
    x = torch.as_tensor(np.random.default_rng(33).normal(size=2 * n), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    yd = torch.zeros_like(x)
    s.matvec(x, y, op="fp32_tree")
    s.matvec(x, yd, op="fp64_direct")
    err = float(torch.linalg.norm(y - yd) / torch.linalg.norm(yd))
    assert err < 1e-4 + 1e-5   # the target plus the FP32 direct product's own rounding
