"""The bench's multi-GPU path on CPU: two gloo ranks.  Environments are
independent, so ranks run their own batches with distinct seeds and no
collective on the data path; the only collectives are the max-over-ranks of
the timed region and the whole-job value."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2306_07552_b300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.WORKLOADS["apartments4096"]
    ms_local = [100.0, 250.0][rank]          # rank 1 is the slow one
    value, ms = bench.job_value(dist, w.n_envs, 50, ms_local)
    q.put((rank, value, ms, bench.rank_seeds(w, rank)))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    w = I.WORKLOADS["apartments4096"]
    for rank, value, ms, seeds in out:
        assert ms == 250.0                            # max over ranks
        assert value == pytest.approx(2 * w.n_envs * 50 / 0.250)   # whole job
    assert out[0][3] != out[1][3]                     # independent streams
