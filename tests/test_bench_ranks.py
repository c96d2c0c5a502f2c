"""The multi-rank path of bench.py (replicas: one decomposition per rank) on CPU:
two gloo ranks check the barrier, the maximum over ranks and the whole-job rate."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ranks = bench.Ranks(dist, "cpu")
    ranks.barrier()
    local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
    ms = ranks.max(local_ms)
    rate = bench.replica_rate(20, ms, world)
    out.put((rank, ms, rate))
    ranks.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    # 2 ranks x 20 sweeps over the slowest rank's 20 ms
    assert res[0][2] == pytest.approx(2 * 20 / 0.020)


def test_single_process_is_a_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(None, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5
    assert bench.replica_rate(10, 5.0, 1) == pytest.approx(2000.0)
