"""Replicated runs (one process per GPU): the bench's whole-job figures are the
slowest rank's time and the work summed over ranks.  Checked with two gloo
ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.reduce_over_ranks(10.0 + 5.0 * rank, 100 + rank, "cpu")
    msf, workf = bench.reduce_over_ranks(3.0 - rank, 0.5 * (rank + 1), "cpu")
    bench.rank_barrier()
    out.put((rank, ms, work, msf, workf))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, work, msf, workf in res:
        assert ms == 15.0 and work == 201 and isinstance(work, int)  # max time, summed int work
        assert msf == 3.0 and workf == 1.5                          # float work summed too


def test_reduce_without_process_group_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 3) == (7.5, 3)
