"""The N > 1 path of bench.py on the CPU: two gloo ranks (spawned processes) run the
timing reduction (max over ranks, units = steps x ranks) and the reference arm's
rank gating (rank 0 alone prints); no GPU and no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 300.0][rank]
    total = bench.job_time_ms(local, dist, "cpu")
    q.put((rank, total, bench.seconds_per_unit(total, 5, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; 2 ranks x 5 problems in 0.3 s
    assert [o[1] for o in out] == [300.0, 300.0]
    assert out[0][2] == pytest.approx(0.3 / 10)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        gpus, steps, warmup = 2, 1, 0
    bench.run_reference(A(), rank=1)
    assert capsys.readouterr().out == ""
