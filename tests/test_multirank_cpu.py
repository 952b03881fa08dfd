"""The multi-rank logic of bench.py on two CPU processes (gloo).

Ensembles of droplet boxes are independent, so N GPUs run N replicas with no
data-path collective; the only cross-rank steps are the barrier and the
max-over-ranks of the timed region.  This checks that reduction, the
whole-job rate, and that every rank draws its own gradient history.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2112_09972_gb300 import workloads

    local = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(local)
    hist = workloads.C2_THROUGHPUT.gradient_history(16, box_id=rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, hist.tolist())
    dist.barrier()
    out[rank] = (t, bench.job_rate(1000, 10, world, t), np.array(gathered[0]), np.array(gathered[1]))
    dist.destroy_process_group()


def test_two_rank_reduction_and_rate():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        t, rate, h0, h1 = res[r]
        assert t == 2.0  # max over ranks
        assert rate == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)
        assert not np.allclose(h0, h1)  # each rank drives its own box
