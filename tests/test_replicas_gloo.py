"""Host logic of multi-GPU runs on CPU: ``bench.py --gpus N`` runs independent
replicas (the operator has no exchange step on resident blocks); the timing
is the max over ranks and the throughput sums every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world),
                       "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    t = bench.reduce_max(10.0 + rank, w)
    bench.barrier(w)
    out[rank] = t
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_reduce_max_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {r: 10.0 + world - 1 for r in range(world)}


def test_aggregate_is_sum_over_max_time():
    assert bench.aggregate([100, 100], [1.0, 2.0]) == 100.0
    assert bench.aggregate([5], [0.5]) == 10.0


def test_single_rank_helpers_need_no_process_group():
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
