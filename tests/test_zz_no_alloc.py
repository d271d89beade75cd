"""hive_insert_noalloc against hive_insert, through the C ABI.

hive_insert_noalloc serves callers that must not call cudaMalloc (device memory
pre-reserved by another allocator, or a loop that cannot stall behind the
device synchronisation that precedes hive_insert's scratch growth).  It keeps
its scratch list in one fixed file-scope device array instead.  This test
drives two identical fixed tables, one through each entry point, with the same
two batches in a row -- the second filling the table to 97% so that inserts
overflow into the eviction kernel and the shared array is used twice -- and
requires identical per-op statuses, find results and sizes (integers, so the
tolerance is zero).  It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2510_15095_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def test_noalloc_matches_insert_on_two_calls(H):
    slots = 1 << 16
    keys, c = W.take_keys(31, 0, slots * 97 // 100)
    vals = W.values_for(keys, 31)
    absent, _ = W.take_keys(31, c, 5000)
    a = H.HiveTable(slots, stash_permille=20)
    b = H.HiveTable(slots, stash_permille=20)
    half = slots // 2
    for lo, hi in ((0, half), (half, keys.size)):
        k = H.to_device_u32(keys[lo:hi])
        v = H.to_device_u32(vals[lo:hi])
        sa = a.insert(k, v).cpu().numpy()
        sb = b.insert_noalloc(k, v).cpu().numpy()
        assert np.array_equal(sa, sb)
        assert (sb == H.INSERTED).all()
        q = H.to_device_u32(np.concatenate([keys[:hi], absent]))
        va, fa = a.find(q)
        vb, fb = b.find(q)
        assert torch.equal(va, vb) and torch.equal(fa, fb)
        assert a.size() == b.size() == hi
    assert b.stats()["overflowed"] > 0  # the scratch list was used
    assert b.check() == 0
    a.close()
    b.close()


def test_noalloc_rejects_oversize_and_resizable(H):
    L = H.load_library()
    t = H.HiveTable(1 << 12)
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    # n above 2^18 is refused before anything is queued
    code = L.hive_insert_noalloc(t._h, e.data_ptr(), e.data_ptr(), (1 << 18) + 1, None, None)
    assert code == 1 and b"exceeds" in L.hive_last_error()
    r = H.HiveTable(1 << 12, max_slots=1 << 14, resizable=True)
    code = L.hive_insert_noalloc(r._h, e.data_ptr(), e.data_ptr(), 1, None, None)
    assert code == 1 and b"fixed-capacity" in L.hive_last_error()
    assert t.size() == 0 and r.size() == 0
    t.close()
    r.close()


def test_noalloc_against_the_oracle_up_to_full(H):
    """The allocation-free insert against the oracle dictionary directly, on
    a small fixed table driven past its capacity: every status (FULL
    included) and every find must be the dictionary's outcome, with the FULL
    ops left out.  Which ops get FULL depends on the layout, so the check is
    that the outcome is valid: the stored keys are exactly the non-FULL ones
    and at most slots + stash words are stored."""
    slots = 1 << 10
    n = 3000
    keys, _ = W.take_keys(37, 0, n)
    vals = W.values_for(keys, 37)
    t = H.HiveTable(slots, stash_permille=0)  # stash floor of 1024 words
    st = t.insert_noalloc(H.to_device_u32(keys), H.to_device_u32(vals)).cpu().numpy()
    full = st == H.FULL
    assert set(np.unique(st)) <= {H.INSERTED, H.FULL}
    assert full.sum() >= n - (slots + 1024) and full.sum() > 0
    d = oracle.Dict()
    assert (d.insert(keys[~full], vals[~full]) == H.INSERTED).all()
    v, f = t.find(H.to_device_u32(keys))
    ev, ef = d.find(keys)
    assert np.array_equal(H.to_host_u32(v), ev) and np.array_equal(f.cpu().numpy(), ef)
    assert t.size() == len(d)
    assert t.check() == 4  # HIVE_ERR_FULL, then cleared
    # a second call re-inserts the kept keys with new values: all REPLACED
    kept = keys[~full]
    nv = W.values_for(kept, 38)
    st2 = t.insert_noalloc(H.to_device_u32(kept), H.to_device_u32(nv)).cpu().numpy()
    assert np.array_equal(st2, d.insert(kept, nv))
    v, f = t.find(H.to_device_u32(keys))
    ev, ef = d.find(keys)
    assert np.array_equal(H.to_host_u32(v), ev) and np.array_equal(f.cpu().numpy(), ef)
    t.close()
