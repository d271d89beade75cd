"""The multi-GPU path of bench.py shards the work into independent tables, one
per rank, with no data-path collective; only the timing is reduced (max over
ranks).  Checked here with two gloo ranks on CPU: the reduction, the whole-job
throughput, and that each rank draws its own keys for its own table."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench as B
    from paper_2510_15095_gb300 import workload as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms = B.max_over_ranks(torch, dist, ms_local, world, torch.device("cpu"))
    keys, _ = W.take_keys(B.shard_seed(rank), 0, 4096)
    gathered = [None] * world
    dist.all_gather_object(gathered, keys.tolist())
    if rank == 0:
        out.put({"ms": ms, "gops": B.job_gops(1000, 4, world, ms), "shards": gathered})
    dist.destroy_process_group()


def test_two_rank_timing_and_disjoint_shards():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["ms"] == 15.0                       # the slowest rank's time
    assert abs(res["gops"] - 1000 * 4 * 2 / 15e-3 / 1e9) < 1e-12
    a, b = (np.array(x, np.uint32) for x in res["shards"])
    # shards come from different seeds: independent tables, no exchange needed
    assert a.size == b.size == 4096 and not np.array_equal(a, b)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench as B
    assert B.max_over_ranks(torch, None, 3.5, 1, torch.device("cpu")) == 3.5
    assert B.job_gops(2_000_000, 5, 1, 10.0) == pytest.approx(1.0)
    assert B.shard_seed(0) != B.shard_seed(1)
