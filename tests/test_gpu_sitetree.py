"""Reaction potential, field and Hessian at the sites by the treecode (Eqs. pot_solvent,
Efield_solv, ddphi through Sec. "The treecode algorithm"), against the oracle's direct
K-node sums (oracle.multipole.reaction_at_sites).

* theta -> 0 opens every cell: the treecode is the direct sum (FP64 1e-12, FP32 pairs
  2e-5 of the largest entry of each output);
* at theta = 0.5 (the sites accept cells at theta / 2: the field and Hessian are
  derivatives of the truncated expansion) the error falls with the Taylor order and at
  order 5 the potential, field and Hessian are each within 1e-4 of their largest entry;
* several bodies: a site sees only its own body's surface;
* the solvation energy with the treecode reaction field (FP32 treecode, FP64-treecode
  refinement of the final solve) within 1e-4 of the oracle's.
"""
import numpy as np
import pytest

import gen
from oracle import bem
from oracle import multipole as mp

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


@pytest.fixture(scope="module", params=[(3, 40), (4, 40)], ids=["1280p", "5120p"])
def case(request, bp):
    sub, ns = request.param
    pr = gen.small_bumpy(sub, ns, 8.0)
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    x = np.random.default_rng(17).normal(size=2 * mesh.n)
    pot, grad, hess = mp.reaction_at_sites(mesh, x[:mesh.n], x[mesh.n:], pr.sites.pos)
    iu = np.triu_indices(3)
    return pr, x, (pot, grad, hess[:, iu[0], iu[1]])


def _site_tree(bp, pr, x, op, **kw):
    s = bp.problem_solver(pr, leaf=kw.pop("leaf", 64), **kw)
    out = torch.zeros(pr.sites.n * 10, dtype=torch.float64, device="cuda")
    s.site_reaction(torch.as_tensor(x, device="cuda"), out, op=op)
    torch.cuda.synchronize()
    s.close()
    o = out.cpu().numpy().reshape(-1, 10)
    return o[:, 0], o[:, 1:4], o[:, 4:]


def _errs(got, ref):
    return [_relmax(g, r) for g, r in zip(got, ref)]


def test_small_theta_is_the_direct_sum(bp, case):
    pr, x, ref = case
    assert max(_errs(_site_tree(bp, pr, x, "fp64_tree", theta=1e-3, order=3), ref)) < 1e-12
    assert max(_errs(_site_tree(bp, pr, x, "fp32_tree", theta=1e-3, order=3), ref)) < 2e-5


def test_error_falls_with_order_and_meets_the_bar(bp, case):
    pr, x, ref = case
    e = [max(_errs(_site_tree(bp, pr, x, "fp64_tree", theta=0.5, order=p), ref)) for p in (2, 4, 6)]
    assert e[0] > e[1] > e[2], e
    bars = (1e-4, 1e-4, 1e-4)
    for op in ("fp64_tree", "fp32_tree"):
        e5 = _errs(_site_tree(bp, pr, x, op, theta=0.5, order=5), ref)
        assert all(e < b for e, b in zip(e5, bars)), (op, e5)


def test_two_bodies_see_their_own_surface(bp):
    a, b, ab = gen.small_triple()
    par = ab.params
    mesh = bem.build_mesh(ab.verts, ab.tris, par.gauss_k, par.near_factor, body=ab.panel_body)
    x = np.random.default_rng(23).normal(size=2 * mesh.n)
    st = ab.sites
    order = np.argsort(st.body, kind="stable")
    pot, grad, hess = mp.reaction_at_sites(mesh, x[:mesh.n], x[mesh.n:], st.pos[order], site_body=st.body[order])
    iu = np.triu_indices(3)
    s = bp.problem_solver(ab, leaf=32, theta=1e-3, order=3)
    out = torch.zeros(st.n * 10, dtype=torch.float64, device="cuda")
    s.site_reaction(torch.as_tensor(x, device="cuda"), out, op="fp64_tree")
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 10)
    assert _relmax(o[:, 0], pot) < 1e-12
    assert _relmax(o[:, 1:4], grad) < 1e-12
    assert _relmax(o[:, 4:], hess[:, iu[0], iu[1]]) < 1e-12


def test_solvation_with_tree_site_fields(bp):
    pr = gen.with_params(gen.small_bumpy(3, 40, 8.0), gmres_tol=1e-8, scf_tol=1e-8)
    ref = mp.solvation(pr, direct_polarization=True)
    out = bp.problem_solver(pr, op="fp32_tree", residual_op="fp64_tree", refine_scope="final", leaf=32,
                            theta=0.5, order=5).solve()
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-4 * abs(ref.dG_kcal)
