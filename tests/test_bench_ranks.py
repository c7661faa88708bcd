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


def _partition_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2205_00237_gb300 import inputs as I
    from paper_2205_00237_gb300.partition import rank_links
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = I.batch_links(4096, seed=0)                      # the batched workload's links
    work = [P * T for _, P, T in spec]
    mine = rank_links(work, rank, world)
    # every rank reports its links; rank 0 checks the split
    sizes = [None] * world
    dist.all_gather_object(sizes, mine)
    dist.destroy_process_group()
    q.put((rank, sizes, sum(work[i] for i in mine), sum(work), max(work)))


def test_batch_links_are_split_once_over_two_gloo_ranks():
    """Every link of the 4096-link batch lands on exactly one of two ranks (computed independently by
    each rank), and each rank's path-steps stay within the largest link of half the total."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, parts0, load0, total, biggest), (_, parts1, load1, _, _) = out
    assert parts0 == parts1                                  # both ranks computed the same split
    flat = sorted(parts0[0] + parts0[1])
    assert flat == list(range(4096))                         # each link exactly once
    assert load0 + load1 == total
    for load in (load0, load1):
        assert abs(load - total / 2) <= biggest


def test_partition_balances_uneven_links():
    sys.path.insert(0, ROOT)
    from paper_2205_00237_gb300.partition import partition_links
    work = [100, 1, 1, 1, 50, 50, 7, 3]
    parts = partition_links(work, 3)
    assert sorted(sum(parts, [])) == list(range(len(work)))
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(work)
    assert partition_links(work, 1) == [list(range(len(work)))]
