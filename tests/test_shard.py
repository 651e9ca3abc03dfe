"""Target sharding of the matrix-vector product over ranks, on the CPU (no GPU).

The library splits the target rows into contiguous ranges of nearly equal cost
(bempol_shard_rows) and every rank computes its own rows; one all-gather per product
(``allgather_rows``, the binding's torch.distributed exchange) gives every rank the
whole vector.  Here the per-rank product is the FP64 oracle's row evaluation
(``oracle.bem.matvec_rows``): after the gather each rank must hold exactly (bit for
bit) the single-rank product, because every row is computed independently of the
split.  Ranks are spawned processes on the gloo backend.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bp():
    from conftest import build_library
    build_library()
    import paper_1810_03698_gb300 as mod
    return mod


def test_shard_rows_partition(bp):
    rng = np.random.default_rng(11)
    for n, world in ((0, 2), (5, 1), (10, 3), (997, 4), (64, 7)):
        cost = rng.uniform(0.0, 3.0, size=n)
        for c in (None, cost):
            b = bp.shard_rows(n, world, c)
            assert len(b) == world + 1 and b[0] == 0 and b[-1] == n
            assert all(b[k] <= b[k + 1] for k in range(world))
            if c is not None and n:
                total, cmax = c.sum(), c.max()
                for k in range(world):   # nearest-prefix cuts: each range within one unit of its share
                    assert abs(c[b[k]:b[k + 1]].sum() - total / world) <= cmax + 1e-12
    assert bp.shard_rows(10, 3, [1] * 9 + [10]) == [0, 6, 9, 10]
    assert bp.shard_rows(4, 3, [0, 0, 0, 0]) == [0, 1, 2, 4]
    with pytest.raises(Exception):
        bp.shard_rows(3, 2, [1.0, -1.0, 1.0])
    with pytest.raises(Exception):
        bp.shard_rows(3, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import gen
        import paper_1810_03698_gb300 as bp
        from oracle import bem
        pr = gen.small_bumpy(2, 6, 6.0, seed_index=131)
        par = pr.params
        mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor)
        n = mesh.n
        x = np.random.default_rng(5).normal(size=2 * n)
        cost = np.diff(mesh.near_ptr).astype(np.float64) + 1.0   # uneven per-row work
        bounds = bp.shard_rows(n, world, cost)
        rows = np.arange(bounds[rank], bounds[rank + 1])
        buf = torch.full((2 * n,), float("nan"), dtype=torch.float64)
        if rows.size:
            y1, y2 = bem.matvec_rows(mesh, x, rows, par.eps_in, par.eps_out, par.kappa)
            buf[bounds[rank]:bounds[rank + 1]] = torch.from_numpy(y1)
            buf[n + bounds[rank]:n + bounds[rank + 1]] = torch.from_numpy(y2)
        bp.allgather_rows(buf, bounds, rank, world)
        y1, y2 = bem.matvec_rows(mesh, x, np.arange(n), par.eps_in, par.eps_out, par.kappa)
        full = np.concatenate([y1, y2])
        q.put((rank, bool(np.array_equal(buf.numpy(), full)), bounds))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_the_single_rank_product(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(o[1] for o in out), out
    assert all(o[2] == out[0][2] for o in out)      # every rank cut the rows the same way
    assert len({o[2][k + 1] - o[2][k] for o in out[:1] for k in range(world)}) >= 1
