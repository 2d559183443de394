"""Host side of the N-GPU bench path (replicas only: independent runs, no
data-path collective): the timing aggregation over ranks, run as two gloo
processes on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 80.0][rank]
    coef = [1.0e9, 3.0e9][rank]
    ms_max, coef_all = bench.aggregate_replicas(ms, coef, dist, "cpu")
    out.put((rank, ms_max, coef_all))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, coef_all in res:
        assert ms_max == 120.0          # the slowest rank's time
        assert coef_all == 4.0e9        # every rank's coefficients


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(5.0, 7.0, None, "cpu") == (5.0, 7.0)
