"""Delta G_solv of the benchmarked form (FP32 treecode, theta 0.5, order 5, leaf 256,
with the final solve refined against the FP64 treecode) at the benchmark sizes.

20,480-panel sphere (R = 10 A, 100 random multipole sites): the GPU's FP64 direct form
(pinned to the oracle at 1e-10 on the small cases) gives the reference value, and both
forms are checked against Kirkwood's closed form for the sphere through the O(A)
convergence of the discretisation (Sec. "Spherical cavity": the error shrinks with the
panel area, so a quarter per subdivision).  81,920-panel bumpy surface (2,000 sites):
the refined FP32 form against the FP64 treecode form on the same inputs.

Tolerances of config 3 (GMRES 1e-6, SCF 1e-6 e*A) on both sizes; the refined form must
agree with its FP64 reference within 1e-4 relative (the treecode bar), and the measured
gaps are far smaller.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import gen
from gen.surfaces import icosphere

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
TREE = dict(theta=0.5, order=5, leaf=256)


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_1810_03698_gb300 as mod
    return mod


def _digest(sites):
    h = hashlib.sha256()
    for a in (sites.pos, sites.q, sites.d, sites.Q, sites.alpha):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def _solve(bp, pr, **kw):
    s = bp.problem_solver(pr, **kw)
    out = s.solve()
    s.close()
    return out


def test_sphere_20480_refined_tree_vs_fp64_direct_and_kirkwood(bp):
    gold = json.load(open(os.path.join(HERE, "golden", "kirkwood_sphere_r10_100sites.json")))
    pr = gen.with_params(gen.sphere_r10_20480(), gmres_tol=1e-6, scf_tol=1e-6)
    assert _digest(pr.sites) == gold["sites_sha256"]
    exact = gold["dG_kcal"]
    v4, f4 = icosphere(10.0, 4)
    pr4 = gen.Problem("sphere_r10_sub4", v4, f4, pr.sites, pr.params)
    d4 = _solve(bp, pr4, op="fp64_direct", residual_op="fp64_direct")["dG_solv_kcal"]
    d5 = _solve(bp, pr, op="fp64_direct", residual_op="fp64_direct")["dG_solv_kcal"]
    t5o = _solve(bp, pr, op="fp32_tree", residual_op="fp64_tree", refine_scope="final", **TREE)
    t5 = t5o["dG_solv_kcal"]
    assert t5o["residual_matvecs"] >= 1
    # (a) the refined treecode form against the FP64 direct form at the same inputs
    assert abs(t5 - d5) < 1e-4 * abs(d5), (t5, d5)
    # (b) both converge to the closed form at O(A): the error falls ~4x from subdivision 4
    # to 5, Richardson's extrapolation removes it, and each form is within that error
    e4, e5 = abs(d4 - exact), abs(d5 - exact)
    assert 3.0 < e4 / e5 < 5.0, (e4, e5)
    rich = d5 + (d5 - d4) / 3.0
    assert abs(rich - exact) < 0.1 * e5, (rich, exact)
    assert abs(t5 - exact) < 1.05 * e5, (t5, exact, e5)


def test_bumpy_81920_refined_tree_vs_fp64_tree(bp):
    pr = gen.bumpy_r14_81920()
    ref = _solve(bp, pr, op="fp64_tree", residual_op="fp64_tree", **TREE)
    got = _solve(bp, pr, op="fp32_tree", residual_op="fp64_tree", refine_scope="final", **TREE)
    plain = _solve(bp, pr, op="fp32_tree", residual_op="fp32_tree", **TREE)
    g, r = got["dG_solv_kcal"], ref["dG_solv_kcal"]
    assert got["residual_matvecs"] >= 1 and got["last_rel_residual"] < 1e-6
    assert abs(g - r) < 1e-5 * abs(r), (g, r)
    assert abs(plain["dG_solv_kcal"] - r) < 1e-5 * abs(r)
