"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2)
take the max of their timed regions and report the whole-job rate, and the
reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [120.0, 150.0][rank]                 # each rank's total ms over its timed steps
    mx = bench.max_over_ranks(mine, world)
    rate = bench.whole_job_rate(world, 10, mx)
    printed = ""
    if rank == 1:                               # the reference arm: ranks other than 0 do no work
        import contextlib
        import io
        import types
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(types.SimpleNamespace(steps=1, warmup=0, gpus=2), rank, world)
        printed = buf.getvalue()
    dist.barrier()
    q.put((rank, mx, rate, printed))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_report_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, printed in out:
        assert mx == 150.0                     # the slowest rank decides
        assert rate == pytest.approx(2 * 10 / 0.150)
        assert printed == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 4, 100.0) == pytest.approx(40.0)


def test_lpt_partition_of_the_ragged_batch():
    """The ragged batch's instances shared out over ranks (bench --workload c3a
    under torchrun): every instance on exactly one rank, the same partition on
    every rank, and no rank above the mean load by more than the largest
    instance (the LPT bound)."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    sizes = W.ragged_sizes(512)
    costs = [4.0 * n * n for n in sizes]
    for world in (1, 2, 3, 4, 8):
        parts = bench.lpt_partition(costs, world)
        assert parts == bench.lpt_partition(costs, world)
        flat = sorted(i for part in parts for i in part)
        assert flat == list(range(len(sizes)))
        loads = [sum(costs[i] for i in part) for part in parts]
        assert max(loads) <= sum(costs) / world + max(costs)
        assert all(len(part) > 0 for part in parts)
