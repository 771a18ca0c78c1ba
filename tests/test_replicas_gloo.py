"""The multi-GPU mode is independent replicas: each rank runs the whole
workload and ranks only meet at the barriers around the timed region.  This
checks the whole-job aggregation bench.py uses (slowest rank's time, sum of
every rank's particle-steps) with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench
    dist = bench.init_dist(world, "gloo")
    bench.barrier(world)
    t, u = bench.combine(1.0 + rank, 1000 * (rank + 1), world)
    q.put((rank, t, u))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, u in res:
        assert t == 2.0          # max over ranks
        assert u == 3000.0       # sum of units


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine(0.5, 123, 1) == (0.5, 123)


def test_scan_split_balances_work():
    # the 256-run scan split over 2, 4 and 8 ranks: every run exactly once,
    # and the busiest rank within the greedy bound (mean + largest run)
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    runs = W.batch_scan(256)
    costs = [bench.run_cost(*r) for r in runs]
    for world in (2, 4, 8):
        share = bench.balance_runs(runs, world)
        assert sorted(i for s in share for i in s) == list(range(len(runs)))
        loads = [sum(costs[i] for i in s) for s in share]
        assert max(loads) <= sum(costs) / world + max(costs)
        assert max(loads) / min(loads) < 1.1
