"""Autotuner: workload classes and the JSON cache (CPU), and a tuning run on
the GPU whose candidates must all give identical per-op results."""
import json

import pytest

from paper_2510_15095_gb300 import autotune as A


def test_workload_key_bands():
    assert A.workload_key(1 << 26, 95, (2, 1, 1), False) == "cap26-load95-mix5:2:2-fixed"
    assert A.workload_key((1 << 26) + 5, 94.2, (4, 4, 2), True) == "cap26-load95-mix4:4:2-resizable"
    assert A.workload_key(1000, 52, (1, 0, 0), False).startswith("cap10-load50-mix10:0:0")
    assert A.workload_key(1 << 22, 90, (2, 1, 1), True, True) == "cap22-load90-mix5:2:2-resizable-multi"


def test_candidates_cover_space():
    c = list(A.candidates({"a": [1, 2], "b": [3, 4, 5]}))
    assert len(c) == 6 and {"a": 2, "b": 5} in c


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "t.json")
    assert A.load_cache(p) == {}
    A.save_cache({"k": {"config": {"max_evictions": 8}}}, p)
    assert A.load_cache(p)["k"]["config"]["max_evictions"] == 8
    assert json.load(open(p))


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = str(tmp_path / "tune.json")
    # every block shape, the persisting L2 window on and off, and two bucket
    # widths must give the same per-op results (tune() checks it)
    space = {"max_evictions": [16], "placement": [0], "bucket_slots": [16, 32],
             "block_threads": [128, 256, 512], "l2_persist": [0, 1]}
    cfg = A.tune(1 << 18, 95, (2, 1, 1), False, cache_path=p, space=space)
    assert set(cfg) == set(space)
    cache = A.load_cache(p)
    (entry,) = cache.values()
    assert len(entry["candidates"]) == 12 and entry["gops"] > 0
    # a second call is served from the cache
    assert A.tune(1 << 18, 95, (2, 1, 1), False, cache_path=p, space=space) == cfg
    rcfg = A.tune(1 << 18, 90, (4, 4, 2), True, cache_path=p,
                  space={"resize_batch": [256, 1024], "max_evictions": [16], "placement": [0]})
    assert rcfg["resize_batch"] in (256, 1024)
    # tables served in multi-table batches: both widths, both resize batch
    # sizes, identical per-op results (tune() checks it)
    mcfg = A.tune(1 << 16, 90, (2, 1, 1), True, cache_path=p, multi=True, reps=1,
                  space={"bucket_slots": [16, 32], "resize_batch": [256, 1024],
                         "max_evictions": [16], "placement": [0]})
    assert mcfg["bucket_slots"] in (16, 32)
    assert any(k.endswith("-multi") for k in A.load_cache(p))
