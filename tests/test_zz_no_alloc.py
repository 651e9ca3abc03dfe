"""bempol_site_reaction_noalloc against bempol_site_reaction, through the C ABI.

The no-allocation variant keeps its partial sums in a fixed device array instead
of a buffer the context allocates, for callers that cannot allow a device
allocation during the call.  It must give the same reaction potential, field and
Hessian at the sites as the allocating entry point, call after call (the shared
array keeps the previous call's contents, which must not leak into the next).
This file is named to be collected last.
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


@pytest.mark.parametrize("op,tol", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_noalloc_matches_site_reaction_twice(bp, op, tol):
    pr = gen.small_bumpy(3, 40, 8.0)
    s = bp.problem_solver(pr)
    n = pr.n_panels
    ns = pr.sites.n
    rng = np.random.default_rng(3)
    for call in range(2):
        x = torch.tensor(rng.normal(size=2 * n), dtype=torch.float64, device="cuda")
        ref = torch.zeros(ns * 10, dtype=torch.float64, device="cuda")
        got = torch.full((ns * 10,), float("nan"), dtype=torch.float64, device="cuda")
        s.site_reaction(x, ref, op=op)
        s.site_reaction_noalloc(x, got, op=op)
        torch.cuda.synchronize()
        r = ref.cpu().numpy().reshape(ns, 10)
        g = got.cpu().numpy().reshape(ns, 10)
        assert np.all(np.isfinite(g)), call
        for a, b in ((g[:, 0], r[:, 0]), (g[:, 1:4], r[:, 1:4]), (g[:, 4:], r[:, 4:])):
            assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < tol, call
    s.close()
