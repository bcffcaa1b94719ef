"""The replica path of bench.py with two ranks on CPU (gloo): the reported time is the slowest rank's and
the throughput counts every rank's bytes; the barrier and the reduction run on every rank."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    tdist.barrier()
    ms = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
    got = bench.max_over_ranks(ms, "cpu")
    out.put((rank, got, bench.whole_job_gbs(1 << 30, world, got[0])))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, gbs in res:
        assert got == [11.0, 20.0, 10.0]
        assert gbs == pytest.approx(2 * (1 << 30) / 11.0e-3 / 1e9)
