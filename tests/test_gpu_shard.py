"""The library's sharded treecode product (bempol_set_shard) on one GPU.

Ranks are simulated by contexts on the same mesh, driven one after another from the
host (no kernel waits on another): rank 0's exchange callback runs the product of
every other rank's context and copies that rank's rows into rank 0's buffer.  The
result must equal the unsharded product bit for bit (each row's sums do not depend on
which rank computes them), for the FP32 and FP64 treecodes; the ranks' row ranges
must be contiguous, cover every panel, and balance the treecode work.
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


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_product_equals_unsharded(bp, world):
    pr = gen.small_bumpy(4, 20, 8.0)
    n = pr.n_panels
    ref = bp.problem_solver(pr, leaf=64)
    ranks = [bp.problem_solver(pr, leaf=64) for _ in range(world)]
    x = torch.as_tensor(np.random.default_rng(21).normal(size=2 * n), dtype=torch.float64, device="cuda")
    op_now = {"op": "fp32_tree"}
    calls = []

    def exchange0(buf, bounds):
        calls.append(1)
        for k in range(1, world):
            tmp = torch.empty_like(x)
            ranks[k].matvec(x, tmp, op=op_now["op"])       # rank k's product: its rows land in its buffer
            other = ranks[k]._shard[0]
            a, e = bounds[k], bounds[k + 1]
            buf[a:e] = other[a:e]
            buf[n + a:n + e] = other[n + a:n + e]

    for k in range(1, world):
        ranks[k].set_shard(k, world, lambda buf, bounds: None)
    ranks[0].set_shard(0, world, exchange0)
    bounds = ranks[0].shard_bounds()
    assert len(bounds) == world + 1 and bounds[0] == 0 and bounds[-1] == n
    assert all(bounds[k] < bounds[k + 1] for k in range(world))
    assert all(r.shard_bounds() == bounds for r in ranks)
    for op in ("fp32_tree", "fp64_tree"):
        op_now["op"] = op
        y = torch.empty_like(x)
        yr = torch.empty_like(x)
        ranks[0].matvec(x, y, op=op)
        ref.matvec(x, yr, op=op)
        torch.cuda.synchronize()
        assert torch.equal(y, yr), op
    assert len(calls) == 2
    # the direct forms are not sharded: no exchange
    y = torch.empty_like(x)
    ranks[0].matvec(x, y, op="fp64_direct")
    torch.cuda.synchronize()
    assert len(calls) == 2
    # per-rank work balanced: near pairs and far terms of each rank's product
    work = []
    for r in ranks:
        r.stats(reset=True)
        r.matvec(x, torch.empty_like(x), op="fp32_tree")
        st = r.stats(reset=True)
        work.append(st["pair_interactions"] + 68.0 * st["far_evaluations"])
    assert max(work) < 1.5 * (sum(work) / world), work
    ranks[0].set_shard(0, 1)
    y = torch.empty_like(x)
    ranks[0].matvec(x, y, op="fp32_tree")
    ref.matvec(x, yr, op="fp32_tree")
    torch.cuda.synchronize()
    assert torch.equal(y, yr)
