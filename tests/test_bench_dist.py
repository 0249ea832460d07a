"""bench.py's multi-GPU path, on the CPU: two gloo ranks.

Cells are independent, so with N GPUs every rank solves its own seeded batch
and no data crosses ranks; the only collectives are the ones that aggregate
the measurement (the slowest rank's time, every rank's cells).  These tests
run that host logic as two processes over gloo on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, world, dist = bench.dist_setup(2)
    seconds, cells = [2.0, 3.0][r], [100, 300][r]
    rate = bench.whole_job_rate(dist, seconds, cells)
    slowest = bench.max_over_ranks(dist, seconds)
    total = bench.sum_over_ranks(dist, cells)
    _, T, _, Y, _ = bench.workload(64, r)
    q.put((r, world, rate, slowest, total, float(T.sum()), float(Y.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_aggregate_and_shard():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, rate, slowest, total, tsum, _) in enumerate(res):
        assert rank == r and world == 2
        assert slowest == 3.0 and total == 400.0
        assert np.isclose(rate, 400.0 / 3.0)        # all cells over the slowest rank's time
    assert res[0][5] != res[1][5]                     # each rank its own batch


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(None, 2.0, 100) == 50.0
    assert bench.max_over_ranks(None, 1.5) == 1.5


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line():
    # rank 0 of the reference arm: the oracle on a bounded sample, one JSON line
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--cells", "4096", "--max-iters", "200"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cell-solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
