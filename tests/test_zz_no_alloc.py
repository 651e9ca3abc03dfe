"""bempol_site_reaction_noalloc against bempol_site_reaction, through the C ABI.

The no-allocation variant keeps its partial sums in a fixed device array instead
of a buffer the context allocates, for callers that cannot allow a device
allocation during the call (another runtime owns the device memory pool, or the
loop cannot take cudaMalloc's implicit synchronisation).  It must give the same
reaction potential, field and Hessian at the sites as the allocating entry point,
call after call: the shared array keeps the previous call's contents, which must
not leak into the next, also when the calls alternate between contexts with
different site counts (and so different numbers of partial-sum splits).  Once the
device code is loaded, repeated calls must leave the device's free memory
unchanged.  This file is named to be collected last.
"""
import numpy as np
import pytest

import gen

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


def _compare(s, bp, ns, n, op, tol, rng):
    x = torch.tensor(rng.normal(size=2 * n), dtype=torch.float64, device="cuda")
    ref = torch.zeros(ns * 10, dtype=torch.float64, device="cuda")
    got = torch.full((ns * 10,), float("nan"), dtype=torch.float64, device="cuda")
    s.site_reaction(x, ref, op=op)
    s.site_reaction_noalloc(x, got, op=op)
    torch.cuda.synchronize()
    r = ref.cpu().numpy().reshape(ns, 10)
    g = got.cpu().numpy().reshape(ns, 10)
    assert np.all(np.isfinite(g))
    for a, b in ((g[:, 0], r[:, 0]), (g[:, 1:4], r[:, 1:4]), (g[:, 4:], r[:, 4:])):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < tol


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_noalloc_matches_site_reaction_twice(bp, op, tol):
    pr = gen.small_bumpy(3, 40, 8.0)
    s = bp.problem_solver(pr)
    rng = np.random.default_rng(3)
    for call in range(2):
        _compare(s, bp, pr.sites.n, pr.n_panels, op, tol, rng)
    s.close()


def test_noalloc_alternating_contexts_and_no_allocation(bp):
    """Two contexts of different size (40 sites on 5,120 panels, 12 sites on 1,280)
    call in turn, so the number of partial-sum splits and the part of the array in
    use change from call to call; then repeated calls leave free memory unchanged."""
    rng = np.random.default_rng(5)
    pa = gen.small_bumpy(4, 40, 8.0)
    pb = gen.small_bumpy(3, 12, 8.0)
    sa = bp.problem_solver(pa)
    sb = bp.problem_solver(pb)
    for _ in range(2):
        _compare(sa, bp, pa.sites.n, pa.n_panels, "fp64_direct", 1e-12, rng)
        _compare(sb, bp, pb.sites.n, pb.n_panels, "fp64_direct", 1e-12, rng)
    x = torch.tensor(rng.normal(size=2 * pa.n_panels), dtype=torch.float64, device="cuda")
    out = torch.zeros(pa.sites.n * 10, dtype=torch.float64, device="cuda")
    sa.site_reaction_noalloc(x, out, op="fp32_direct")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        sa.site_reaction_noalloc(x, out, op="fp32_direct")
        sa.site_reaction_noalloc(x, out, op="fp64_direct")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    sa.close()
    sb.close()
