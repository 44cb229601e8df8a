"""Host logic of the multi-process bench (one replica per GPU, chains sharded, no
data-path collective): two gloo ranks on the CPU check the max-over-ranks timing
and the whole-job throughput that rank 0 reports."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env()[:2] == (rank, world)
    ms_local = [4.0, 6.5][rank]
    dist.barrier()
    ms, value = bench.reduce_timing(ms_local, 256, world, dist, torch.device("cpu"))
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_timing_is_max_and_value_is_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value in res:
        assert ms == pytest.approx(6.5)
        assert value == pytest.approx(2 * 256 / 6.5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.reduce_timing(5.0, 256, 1, None)
    assert ms == 5.0 and value == pytest.approx(256 / 5e-3)
