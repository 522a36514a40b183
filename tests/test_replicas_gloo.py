"""The N > 1 path of bench.py (replicas, one independent problem per rank) on CPU:
two gloo ranks aggregate their times and iteration counts as the contract says
(max over ranks of the times, sum of the iterations) and keep every rank's own
iterations and times."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = bench.aggregate_replicas(dist, 1.0 + rank, 10.0 - rank, 100 + rank, torch.device("cpu"))
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_replicas_aggregate_on_gloo():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        s, m, it, per_rank = res[r]
        assert s == 2.0 and m == 10.0 and it == 201
        # every rank's own record, in rank order, on every rank
        assert [p["rank"] for p in per_rank] == [0, 1]
        assert [p["iters"] for p in per_rank] == [100, 101]
        assert [p["solve_s"] for p in per_rank] == [1.0, 2.0]
        assert [p["step_ms"] for p in per_rank] == [10.0, 9.0]
