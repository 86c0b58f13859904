"""The replica form of the benchmark for N > 1 ranks (no data-path
collective): the ranks meet only at the barriers around a timed region and
in the maximum of their times, and the whole-job value is ranks x units over
the slowest rank's time.  Run here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.replica_barrier()
        slowest = bench.replica_max(times[rank], "cpu")
        bench.replica_barrier()
        out.put((rank, slowest, bench.replica_throughput(20, slowest, world)))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [3.5, 4.25]   # ms of the two ranks' timed regions
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 4.25
        assert value == pytest.approx(2 * 20 / 4.25e-3)


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(20, 4.0, 1) == pytest.approx(5000.0)
