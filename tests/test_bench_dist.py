"""bench.py's whole-job aggregation over ranks, with world size 2 on gloo
(CPU): units add up, time is the slowest rank's."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(world, "gloo")
    elapsed = [2.0, 3.0][rank]
    units = [10.0, 20.0][rank]
    value, t = bench.aggregate(d, elapsed, units)
    d.barrier()
    d.close()
    q.put((rank, value, t))


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in out:
        assert t == 3.0
        assert value == pytest.approx(30.0 / 3.0)


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(1, "gloo")
    assert bench.aggregate(d, 2.0, 10.0) == (5.0, 2.0)
