"""The N-GPU form of bench.py runs independent replicas; its only exchange
is the timing: max over ranks of the timed region, sum of the units.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    try:
        ms, units = bench.replica_totals([1500.0, 2500.0][rank], [304, 300][rank])
        out.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_replica_totals_take_the_slowest_rank_and_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2500.0, 604.0), (1, 2500.0, 604.0)]


def test_replica_totals_without_a_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.replica_totals(12.5, 7) == (12.5, 7.0)
