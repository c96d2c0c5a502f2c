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


def test_reference_arm_line_on_cpu():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys; the 64^3 workload keeps it to seconds."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "c1", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
