"""The Stern (ion-exclusion) layer on the GPU (bempol_set_mesh_stern; Sec. "Spherical
cavity": R = 4 A dielectric boundary inside a 5 A ion-exclusion surface) against the
three-region oracle ``oracle/stern.py``, itself pinned to the closed-form sphere with a
layer and to Gauss's law (test_oracle_stern.py).

  * FP64 direct: Delta G_solv at 1e-10 relative, phi and psi on both surfaces at 1e-9 of
    their largest entry;
  * FP32 direct refined against FP64 direct: Delta G at 1e-10; plain FP32 direct at 1e-5;
  * the layer changes Delta G at this salt level (kappa = 1/A) by far more than the bars;
  * refusals: a treecode operator form and the adjoint gradient (BEMPOL_ERR_ARG), the
    surfaces swapped (BEMPOL_ERR_MESH).
"""
import numpy as np
import pytest

import gen
from oracle import multipole as mp, stern

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
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def _case(sub=3, kappa=1.0):
    pr = gen.sphere_random(4.0, sub, 5, 2.2, 1.2, 11)
    pr = gen.with_params(pr, kappa=kappa, eps_in=4.0, gmres_tol=1e-13, scf_tol=1e-12, scf_maxit=400)
    v2, f2 = gen.icosphere(5.0, sub)
    return pr, v2, f2


def _solver(bp, pr, v2, f2, **kw):
    from paper_1810_03698_gb300 import _param_kw
    s = bp.Solver(device=0, **_param_kw(pr.params, kw))
    s.set_mesh_stern(pr.verts, pr.tris, v2, f2)
    st = pr.sites
    s.set_sites(np.ascontiguousarray(st.pos), np.ascontiguousarray(st.q), np.ascontiguousarray(st.d),
                np.ascontiguousarray(st.Q.reshape(-1, 9)), np.ascontiguousarray(st.alpha),
                np.ascontiguousarray(st.group, dtype=np.int32))
    return s


@pytest.fixture(scope="module")
def oracle_ref():
    pr, v2, f2 = _case()
    S = stern.stern_solver(pr.verts, pr.tris, v2, f2, pr.params)
    r = mp.solvation(pr, solver=S, direct_polarization=True)
    return pr, v2, f2, S, r


def test_fp64_direct_matches_oracle(bp, oracle_ref):
    pr, v2, f2, S, r = oracle_ref
    s = _solver(bp, pr, v2, f2, op="fp64_direct", residual_op="fp64_direct")
    out = s.solve(outputs=True)
    s.close()
    assert abs(out["dG_solv_kcal"] - r.dG_kcal) < 1e-10 * abs(r.dG_kcal), (out["dG_solv_kcal"], r.dG_kcal)
    x = S.solve_full(r.rhs)
    n1, n2 = S.mesh.n, S.mesh2.n
    phi = np.concatenate([x[:n1], x[2 * n1:2 * n1 + n2]])
    psi = np.concatenate([x[n1:2 * n1], x[2 * n1 + n2:]])
    assert _relmax(out["phi"], phi) < 1e-9
    assert _relmax(out["dphidn"], psi) < 1e-9
    # without the layer (one surface at R = 4) Delta G moves by far more than the bar
    s1 = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    one = s1.solve()["dG_solv_kcal"]
    s1.close()
    assert abs(one - r.dG_kcal) > 1e-3 * abs(r.dG_kcal)


def test_fp32_direct_forms(bp, oracle_ref):
    pr, v2, f2, S, r = oracle_ref
    s = _solver(bp, pr, v2, f2, op="fp32_direct", residual_op="fp64_direct")
    got = s.solve()["dG_solv_kcal"]
    s.close()
    assert abs(got - r.dG_kcal) < 1e-10 * abs(r.dG_kcal)
    pl = gen.with_params(pr, gmres_tol=1e-6, scf_tol=1e-6)
    s = _solver(bp, pl, v2, f2, op="fp32_direct", residual_op="fp32_direct")
    got = s.solve()["dG_solv_kcal"]
    s.close()
    assert abs(got - r.dG_kcal) < 1e-5 * abs(r.dG_kcal)


def test_refusals(bp):
    pr, v2, f2 = _case(sub=2)
    s = _solver(bp, pr, v2, f2, op="fp32_tree", residual_op="fp64_tree")
    with pytest.raises(bp.BempolError) as ei:
        s.solve()
    assert bp.STATUS[ei.value.status] == "ERR_ARG"
    s.set_params(op="fp64_direct", residual_op="fp64_direct")
    s.solve()
    with pytest.raises(bp.BempolError) as ei:
        s.gradient()
    assert bp.STATUS[ei.value.status] == "ERR_ARG"
    s.close()
    s = bp.Solver(device=0)
    with pytest.raises(bp.BempolError) as ei:
        s.set_mesh_stern(v2, f2, pr.verts, pr.tris)  # the outer surface given as the inner one
    assert bp.STATUS[ei.value.status] == "ERR_MESH"
    s.close()
