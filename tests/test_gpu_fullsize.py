"""Parity at the benchmark sizes (20,480 and 81,920 panels) on sampled outputs.

The oracle cannot form the dense operator at these sizes, so it computes sampled
rows of the matrix-vector product (every Gauss node of every panel plus the
accurate near integrals), sampled right-hand-side entries and the reaction field
at sampled sites, one by one, and the GPU results are compared on those.
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


@pytest.fixture(scope="module", params=[("sphere_r10_20480", 2), ("bumpy_r14_81920", 3)], ids=lambda p: p[0])
def big(request, bp):
    name, seed = request.param
    pr = gen.WORKLOADS[name]()
    par = pr.params
    mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
    s = bp.problem_solver(pr, leaf=256, theta=0.5, order=5)
    rng = np.random.default_rng(100 + seed)
    rows = np.sort(rng.choice(mesh.n, size=24, replace=False))
    x = rng.normal(size=2 * mesh.n)
    y1, y2 = bem.matvec_rows(mesh, x, rows, par.eps_in, par.eps_out, par.kappa)
    ref = np.concatenate([y1, y2])
    return pr, mesh, s, rows, x, ref


def _rows(s, x, rows, op, n):
    y = torch.zeros(x.size, dtype=torch.float64, device="cuda")
    s.matvec(torch.tensor(x, device="cuda"), y, op=op)
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    return np.concatenate([y[rows], y[n + rows]])


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 5e-5), ("fp32_tree", 5e-4),
                                    ("fp64_tree", 5e-4)])
def test_matvec_rows(big, op, tol):
    pr, mesh, s, rows, x, ref = big
    got = _rows(s, x, rows, op, mesh.n)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-13), ("fp32_direct", 2e-5)])
def test_rhs_rows(big, op, tol):
    pr, mesh, s, rows, x, ref = big
    st = pr.sites
    b = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    s.rhs(b, op=op)
    torch.cuda.synchronize()
    want = mp.rhs(mesh.cen[rows], st.pos, st.q, st.d, st.Q, pr.params.eps_in)
    got = b.cpu().numpy()[rows]
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < tol


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 5e-5)])
def test_site_reaction_sampled(big, op, tol):
    pr, mesh, s, rows, x, ref = big
    out = torch.zeros(pr.sites.n * 10, dtype=torch.float64, device="cuda")
    s.site_reaction(torch.tensor(x, device="cuda"), out, op=op)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 10)
    pick = np.random.default_rng(5).choice(pr.sites.n, size=6, replace=False)
    pot, grad, hess = mp.reaction_at_sites(mesh, x[:mesh.n], x[mesh.n:], pr.sites.pos[pick])
    iu = np.triu_indices(3)
    got = o[pick]
    for a, b in ((got[:, 0], pot), (got[:, 1:4], grad), (got[:, 4:], hess[:, iu[0], iu[1]])):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < tol


def test_near_table_matches_oracle(big):
    pr, mesh, s, rows, x, ref = big
    g = s.geometry()
    assert np.array_equal(g["near_ptr"], mesh.near_ptr)
    assert np.array_equal(g["near_col"], mesh.near_cols)
