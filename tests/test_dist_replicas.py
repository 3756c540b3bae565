"""The multi-rank path of bench.py on CPU (gloo, world size 2).

The operation has no exchange step, so N GPUs run N independent replicas; the
only cross-rank logic is the barrier and the reduction of the timing (max over
ranks) and of the work (sum over ranks).  Those run here as two gloo ranks.
"""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ws, r, local = bench.dist_env()
    dist = bench.init_dist(ws)
    bench.barrier(dist)
    t_max = bench.max_over_ranks(dist, 10.0 + rank)       # per-rank times 10, 11
    total = bench.sum_over_ranks(dist, 1000.0 * (rank + 1))  # per-rank work 1000, 2000
    q.put((rank, ws, local, t_max, total))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, local, t_max, total in results:
        assert ws == 2 and local == rank
        assert t_max == 11.0      # the slowest rank sets the time
        assert total == 3000.0    # whole-job work is the sum


def test_single_process_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    ws, rank, local = bench.dist_env()
    assert (ws, rank, local) == (1, 0, 0)
    assert bench.init_dist(ws) is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0
