"""Replica aggregation of bench.py on CPU: two gloo ranks, each timing its own
replica; the whole-job value is all ranks' units over the slowest rank's time."""
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
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2105_02127_gb300 import replicas
    r, w, lr = replicas.world()
    assert (r, w, lr) == (rank, world, rank)
    replicas.barrier()
    secs = 1.0 + rank  # rank 1 is the slow one
    units = 1000.0 * (rank + 1)
    out[rank] = (replicas.max_over_ranks(secs), replicas.job_throughput(units, secs))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(100)
        assert p.exitcode == 0
    for r in range(2):
        mx, thr = out[r]
        assert mx == 2.0
        assert thr == pytest.approx(3000.0 / 2.0)
