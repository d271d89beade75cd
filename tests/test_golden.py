"""Regression fixtures in tests/golden/ (written by tests/golden/make_golden.py
from the oracle): the oracle must keep reproducing them, and the CUDA path
must reproduce the op-stream outcomes."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STATES = [(1023, 0), (1023, 511), (32767, 100)]


def rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [list(map(int, line.split())) for line in f if not line.startswith("#")]


def test_bithash_and_address_fixture():
    for r in rows("bithash.txt"):
        k, h1, h2 = r[:3]
        assert oracle.bithash1(k) == h1 and oracle.bithash2(k) == h2, k
        addr = [oracle.lh_address(h, M, p) for M, p in STATES for h in (h1, h2)]
        assert addr == r[3:], k


def test_op_stream_fixture():
    r = np.array(rows("ops.txt"), dtype=np.int64)
    d = oracle.Dict()
    ev, est = d.execute(r[:, 0].astype(np.uint8), r[:, 1].astype(np.uint32),
                        r[:, 2].astype(np.uint32))
    assert np.array_equal(est, r[:, 3]) and np.array_equal(ev, r[:, 4])


def _phases(n):
    """The stream's five phases (40 inserts, 8 re-inserts, 24 finds, 16
    erases, 8 finds), one call each, so that the batch contract holds within
    every call; applied in order they equal the oracle's op-by-op order."""
    return np.split(np.arange(n), [40, 48, 72, 88])


@pytest.mark.gpu
@pytest.mark.parametrize("bs", [32, 16])
def test_op_stream_fixture_on_gpu(bs):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive as H
    r = np.array(rows("ops.txt"), dtype=np.int64)
    ops, keys, vals = r[:, 0].astype(np.uint8), r[:, 1].astype(np.uint32), r[:, 2].astype(np.uint32)
    t = H.HiveTable(1 << 10, bucket_slots=bs)
    st_all = np.zeros(ops.size, np.int64)
    v_all = np.zeros(ops.size, np.int64)
    assert ops.size == 96
    for idx in _phases(ops.size):
        vo, st = t.execute(torch.from_numpy(ops[idx]).cuda(), H.to_device_u32(keys[idx]),
                           H.to_device_u32(vals[idx]))
        st_all[idx] = st.cpu().numpy()
        v_all[idx] = H.to_host_u32(vo)
    assert np.array_equal(st_all, r[:, 3]) and np.array_equal(v_all, r[:, 4])
    t.close()
