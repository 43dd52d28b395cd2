"""The N > 1 path of bench.py on CPU: two gloo ranks, max-over-ranks timing and the whole-job rate
(independent replicas, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [0.5, 1.25][rank]
    slowest = bench.reduce_max(local_seconds, dist, "cpu")
    rate = bench.job_rate(world, 128 ** 3, 50, slowest)
    q.put((rank, slowest, rate, bench.rank_info()))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_job_rate():
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
    for rank, slowest, rate, info in out:
        assert slowest == 1.25
        assert rate == pytest.approx(2 * 128 ** 3 * 50 / 1.25 / 1e6)
        assert info[0] == rank and info[1] == 2


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_rate(1, 1000, 10, 2.0) == pytest.approx(1000 * 10 / 2.0 / 1e6)
