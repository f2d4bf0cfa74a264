"""Multi-GPU runs are independent replicas (no collective on the data path):
the bench's aggregation takes the slowest rank's time and the sum of all
ranks' iterations.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, it = bench.aggregate_ranks(total_s=1.0 + rank, iters=100 * (rank + 1), world=world, device="cpu")
    out[rank] = (t, it)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_max_time_sum_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == (2.0, 300) and out[1] == (2.0, 300)


def test_single_rank_is_identity():
    import bench

    assert bench.aggregate_ranks(1.5, 42, 1) == (1.5, 42)
