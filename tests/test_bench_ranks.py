"""Host logic of the multi-GPU benchmark path, run as two gloo ranks on the CPU.

With N ranks each rank runs its own link on its own GPU (weak scaling, no data-path collective);
the only collectives are a barrier and the maximum of the timed seconds, and the reported value is
the units of all ranks over the slowest rank's time.  These tests run that logic with the gloo
backend, ranks as child processes, rendezvous on 127.0.0.1.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    seconds = [1.5, 2.0][rank]              # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(seconds, w)
    value = bench.whole_job_rate(1000.0, w, t)
    dist.destroy_process_group()
    q.put((r, lr, w, t, value))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, lr, w, t, value) in enumerate(out):
        assert (r, lr, w) == (rank, rank, 2)
        assert t == pytest.approx(2.0)                 # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
