"""The N > 1 path of bench.py runs independent replicas (weak scaling); only
the timing crosses ranks: units are summed and the time is the maximum over
ranks.  Checked with two gloo ranks on CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank)
    bench.barrier()
    out[rank] = (units, secs)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (pytest.approx(3000.0), pytest.approx(1.5))


def test_single_process_aggregation_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(42.0, 2.0) == (42.0, 2.0)
