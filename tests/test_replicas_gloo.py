"""Multi-GPU runs are replicas (no exchange step in the method's scope): the
benchmark's host logic takes the slowest rank's time and the summed work.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.reduce_over_ranks(10.0 * (rank + 1), 1000.0 + rank, dist, "cpu")
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_reduction_over_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
            assert p.exitcode == 0
        assert out[0] == out[1] == (20.0, 2001.0)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(3.0, 7.0) == (3.0, 7.0)
