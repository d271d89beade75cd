"""Serving loop: each request's result is the same alone and in the mix.

A trace of requests with Poisson arrivals is served by continuous batching
(multi-table asynchronous batches, two in flight).  The same requests are then
replayed one at a time through hive_execute on fresh tables, in arrival order,
and every per-op status and find value must match bit for bit; a per-table
oracle dictionary checks the results too.  The HBM-budget admission rejects
requests that can never fit and serves the rest correctly.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive, serving, workload
    hive.load_library()
    return hive, serving, workload


def _tables(H, W, n_tables, preload, init_slots, max_slots):
    tabs = []
    for t in range(n_tables):
        tb = H.HiveTable(init_slots, max_slots=max_slots, resizable=True, resize_batch=256)
        k, v = W.preload_t(torch, 1000 + t, preload, "cuda")
        tb.insert(k, v)
        tabs.append(tb)
    return tabs


def _oracle_check(H, W, reqs, n_tables, preload):
    dicts = []
    for t in range(n_tables):
        d = oracle.Dict()
        k, v = W.preload_t(torch, 1000 + t, preload, "cpu")
        d.insert(k.numpy().view(np.uint32), v.numpy().view(np.uint32))
        dicts.append(d)
    for r in reqs:
        if r.rejected:
            continue
        ev, est = dicts[r.table].execute(r.ops.cpu().numpy(), r.keys.cpu().numpy().view(np.uint32),
                                         r.vals.cpu().numpy().view(np.uint32))
        assert np.array_equal(r.status.cpu().numpy(), est), r.rid
        assert np.array_equal(H.to_host_u32(r.vals_out), ev), r.rid
    return dicts


@pytest.mark.parametrize("depth", [1, 2])
def test_served_equals_alone(mods, depth):
    H, S, W = mods
    nt, pre = 8, 5000
    tabs = _tables(H, W, nt, pre, 1 << 13, 1 << 22)
    counts = [pre] * nt
    reqs = S.make_trace(torch, nt, 300, rate_per_s=30_000.0, seed=7 + depth, counts=counts,
                        max_log2_ops=14)
    srv = S.HiveServer(tabs, hbm_budget_bytes=64e9, max_batch_ops=1 << 18, max_batch_reqs=64,
                       depth=depth)
    out = srv.run(reqs)
    srv.close()
    assert out["rejected"] == 0 and out["requests"] == 300
    assert out["batches"] < 300  # requests were coalesced
    served = [(r.status.clone(), r.vals_out.clone()) for r in reqs]
    # alone: one request at a time on fresh tables, in arrival order
    alone = _tables(H, W, nt, pre, 1 << 13, 1 << 22)
    for r in reqs:
        vo, st = alone[r.table].execute(r.ops, r.keys, r.vals)
        assert torch.equal(st, served[r.rid][0]), r.rid
        assert torch.equal(vo, served[r.rid][1]), r.rid
    dicts = _oracle_check(H, W, reqs, nt, pre)
    for t in range(nt):
        assert tabs[t].size() == len(dicts[t])
        assert oracle.check_image(tabs[t].dump(), 32, dicts[t])[0] == 0
        assert tabs[t].check() == 0
    for tb in tabs + alone:
        tb.close()


def test_fifo_reference_matches(mods):
    H, S, W = mods
    nt, pre = 4, 2000
    tabs = _tables(H, W, nt, pre, 1 << 12, 1 << 20)
    counts = [pre] * nt
    reqs = S.make_trace(torch, nt, 80, rate_per_s=50_000.0, seed=3, counts=counts, max_log2_ops=12)
    out = S.run_fifo(tabs, reqs)
    assert out["requests"] == 80
    _oracle_check(H, W, reqs, nt, pre)
    for tb in tabs:
        tb.close()


def test_budget_admission_rejects_what_cannot_fit(mods):
    H, S, W = mods
    nt, pre = 4, 1000
    tabs = _tables(H, W, nt, pre, 1 << 12, 1 << 22)
    counts = [pre] * nt
    reqs = S.make_trace(torch, nt, 60, rate_per_s=50_000.0, seed=5, counts=counts, max_log2_ops=15)
    committed = sum(t.capacity() for t in tabs) * S.SLOT_BYTES
    srv = S.HiveServer(tabs, hbm_budget_bytes=committed * 4, max_batch_ops=1 << 17, max_batch_reqs=16)
    out = srv.run(reqs)
    srv.close()
    assert out["rejected"] > 0 and out["requests"] > 0
    assert sum(t.capacity() for t in tabs) * S.SLOT_BYTES <= committed * 4 + 1
    _oracle_check(H, W, reqs, nt, pre)
    for tb in tabs:
        tb.close()
