"""Host logic of the multi-GPU bench path on CPU: two gloo ranks, each timing its own
independent run; the job time is the max over ranks and the job's units add up."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    r, lr, w = bench.dist_env()
    ms = 10.0 + 7.0 * rank
    out[rank] = (r, w, bench.max_over_ranks(ms, w), bench.job_units(1024, 700, 5, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_time_and_units():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (0, 2, 17.0, 1024 * 700 * 5 * 2)
    assert out[1] == (1, 2, 17.0, 1024 * 700 * 5 * 2)


def test_single_rank_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
