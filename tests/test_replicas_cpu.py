"""The multi-GPU path (independent replicas, timing collectives only) run as
two gloo ranks on the CPU: every rank gets its own data seed, and both ranks
report the slowest rank's time and the job-wide throughput."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1705_07497_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.rank_info()
        replicas.barrier(w)
        secs = 1.0 + r  # rank 1 is the slower one
        slowest = replicas.max_over_ranks(secs, w)
        out.put((r, w, local, replicas.rank_seed(1000, r), slowest, replicas.job_throughput(w, 5, slowest)))
        replicas.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(world))
    assert [x[0] for x in res] == [0, 1]
    assert all(x[1] == 2 and x[2] == x[0] for x in res)
    assert [x[3] for x in res] == [1000, 1001]  # distinct data per rank
    assert all(x[4] == 2.0 for x in res)  # both see the slowest rank's time
    assert all(abs(x[5] - 2 * 5 / 2.0) < 1e-12 for x in res)


def test_single_process_needs_no_process_group():
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    replicas.barrier(1)
    assert replicas.job_throughput(1, 4, 2.0) == 2.0
