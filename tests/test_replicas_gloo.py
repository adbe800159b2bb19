"""The N > 1 benchmark path: replica sources and the max-over-ranks aggregation, as world_size-2
gloo processes on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1005_0542_gb300.replicas import replica_source, whole_job_rate


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    src = replica_source((1024, 16), rank, 2048)
    rate, t = whole_job_rate(1.0 + rank, 8, world, dist=dist)
    out[rank] = (src, rate, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_world_size_two():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == (1024, 16) and out[1][0] == (1088, 16)   # distinct replica sources
    for r in range(2):
        assert out[r][2] == pytest.approx(2.0)                    # slowest rank's time
        assert out[r][1] == pytest.approx(2 * 8 / 2.0)            # all ranks' units / max time
