"""The multi-rank path of bench.py on CPU: world-size-2 gloo ranks aggregate the job's
rate as units of all ranks over the slowest rank's time (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [0.5, 2.0][rank]  # rank 1 is the slowest
    rate = bench.whole_job_rate(100, seconds, world, dist, "cpu")
    mx = bench.reduce_max(seconds, dist, "cpu")
    q.put((rank, rate, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, mx in res:
        assert mx == 2.0
        assert rate == pytest.approx(2 * 100 / 2.0)  # both ranks' units over the slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.whole_job_rate(10, 0.5, 1) == pytest.approx(20.0)
    assert bench.reduce_max(3.0) == 3.0
