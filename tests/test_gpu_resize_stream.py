"""Resize stream at full batch size: batches of 2^22 mixed ops on one
resizable table that starts with 2^20 live keys, three growth batches
(insert:erase:find 40/20/40) then three shrink batches (20/40/40), finds
Zipf(0.99) over live keys not updated in the batch, thresholds 0.9 / 0.4.
Every per-op result, the size and the capacity after every batch must match
the oracle and its linear-hashing policy model; invariants hold after each
phase."""
import numpy as np
import pytest

import oracle
from paper_2510_15095_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
S = 32


def test_resize_stream_2e22_batches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive as H
    H.load_library()
    n_batch = 1 << 22
    start, ctr = W.take_keys(33, 0, 1 << 20)
    t = H.HiveTable(1 << 21, max_slots=1 << 25, resizable=True, resize_batch=1024, shrink=(2, 5))
    pol = oracle.Policy((1 << 21) // S, (1 << 25) // S, K=1024, shrink=(2, 5))
    d = oracle.Dict()
    vals = W.values_for(start, 33)
    pol.grow(0, start.size)
    t.insert(H.to_device_u32(start), H.to_device_u32(vals))
    d.insert(start, vals)
    pol.shrink(len(d))
    assert t.capacity() == S * pol.state[0]
    rng = np.random.default_rng(33)
    live = start
    for phase, (fi, fe) in (("grow", (2, 1)), ("shrink", (1, 2))):
        for b in range(3):
            n_ins, n_er = n_batch * fi // 5, n_batch * fe // 5
            new, ctr = W.take_keys(33, ctr, n_ins)
            ops, keys, vals = W.mixed_batch(rng, live, new, n_ins, n_er, n_batch - n_ins - n_er,
                                            seed=33 + b, zipf_s=0.99)
            pol.grow(len(d), n_ins)
            vo, st = t.execute(torch.from_numpy(ops).cuda(), H.to_device_u32(keys),
                               H.to_device_u32(vals))
            ev, est = d.execute(ops, keys, vals)
            pol.shrink(len(d))
            assert np.array_equal(st.cpu().numpy(), est), (phase, b)
            assert np.array_equal(H.to_host_u32(vo), ev), (phase, b)
            assert t.capacity() == S * pol.state[0], (phase, b, t.capacity(), pol.state)
            assert t.size() == len(d)
            live, _ = d.dump()
        code, where = oracle.check_image(t.dump(), S, d, pol)
        assert code == 0, (phase, code, where)
    s = t.stats()
    assert s["splits"] > 0 and s["merges"] > 0
    assert t.check() == 0
    t.close()
