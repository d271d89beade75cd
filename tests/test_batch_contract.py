"""Host-side batch-contract check (hive_check_batch), on the CPU.

The contract (Section III-D runs a batch's ops concurrently): no key is
updated twice in one call, and in a mixed batch no key is both updated and
searched.  The library's check groups ops by key with a radix sort; here it is
compared with the definition written out as a quadratic scan, and the
workload generators used by the tests and the benchmark are shown to keep
the contract."""
import ctypes as C

import numpy as np
import pytest

from paper_2510_15095_gb300 import workload as W

OP_INSERT, OP_FIND, OP_ERASE = 0, 1, 2


@pytest.fixture(scope="module")
def H():
    from paper_2510_15095_gb300 import build as B
    from paper_2510_15095_gb300 import hive
    hive.load_library(B.build())  # host code only: loads and runs without a GPU
    return hive


def first_bad_brute(keys, ops, op, key_limit):
    """Smallest i such that ops [0, i] break the contract: some earlier op on
    the same (non-reserved) key where one of the two is an update."""
    n = len(keys)
    upd = lambda j: (ops[j] if ops is not None else op) in (OP_INSERT, OP_ERASE)  # noqa: E731
    for i in range(n):
        if keys[i] >= key_limit:
            continue
        for j in range(i):
            if keys[j] == keys[i] and (upd(i) or upd(j)):
                return i
    return None


def test_small_cases(H):
    assert H.check_batch([5, 6, 7]) is None
    assert H.check_batch([5, 6, 5]) == 2                       # insert twice
    assert H.check_batch([5, 6, 5], op=OP_ERASE) == 2          # erase twice
    assert H.check_batch([5, 6, 5], op=OP_FIND) is None        # finds may repeat
    assert H.check_batch([5, 6, 5], ops=[1, 1, 1]) is None
    assert H.check_batch([5, 6, 5], ops=[1, 0, 0]) == 2        # find, then update
    assert H.check_batch([5, 6, 5], ops=[0, 1, 1]) == 2        # update, then find
    assert H.check_batch([5, 5, 6, 6], ops=[1, 1, 2, 0]) == 3  # the earliest break wins
    assert H.check_batch([0xFFFFFFFF, 6, 0xFFFFFFFF]) is None  # reserved keys touch nothing
    assert H.check_batch([0xFFFE, 0xFFFE], key_limit=0xFFFE) is None
    assert H.check_batch([0xFFFD, 0xFFFD], key_limit=0xFFFE) == 1
    assert H.check_batch(np.array([-3, -3], dtype=np.int32)) == 1  # int32 storage = unsigned bits
    assert H.check_batch([]) is None
    # unknown op codes count as finds (as in the kernels)
    assert H.check_batch([9, 9], ops=[7, 7]) is None
    assert H.check_batch([9, 9], ops=[7, 0]) == 1


def test_error_text_and_null_keys(H):
    L = H.load_library()
    k = np.array([3, 4, 3], dtype=np.uint32)
    bad = C.c_uint64(99)
    assert L.hive_check_batch(None, OP_INSERT, k.ctypes.data, 3, 0xFFFFFFFE, C.byref(bad)) == 1
    assert bad.value == 2
    assert b"key 3" in L.hive_last_error()
    assert L.hive_check_batch(None, OP_INSERT, None, 3, 0xFFFFFFFE, None) == 1
    assert L.hive_check_batch(None, OP_INSERT, None, 0, 0xFFFFFFFE, C.byref(bad)) == 0
    assert bad.value == 0


@pytest.mark.parametrize("seed", range(12))
def test_against_the_definition(H, seed):
    """Random batches with many collisions, including keys equal in one
    16-bit half only (the radix passes must not merge them) and reserved keys."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 120))
    lo = rng.integers(0, 4, n).astype(np.uint32)
    hi = rng.integers(0, 4, n).astype(np.uint32)
    keys = (hi << np.uint32(16)) | lo
    keys[rng.random(n) < 0.1] = 0xFFFFFFFE
    key_limit = 0xFFFFFFFE if seed % 3 else 0x00030000
    for ops, op in ((None, OP_INSERT), (None, OP_ERASE), (None, OP_FIND),
                    (rng.integers(0, 3, n).astype(np.uint8), OP_FIND),
                    ((rng.random(n) < 0.9).astype(np.uint8), OP_FIND)):  # mostly finds
        exp = first_bad_brute(keys, ops, op, key_limit)
        assert H.check_batch(keys, ops=ops, op=op, key_limit=key_limit) == exp, (ops, op)


def test_large_batch_and_planted_repeat(H):
    keys, _ = W.take_keys(31, 0, 1 << 20)
    assert H.check_batch(keys) is None
    planted = keys.copy()
    planted[777_777] = planted[123]
    assert H.check_batch(planted) == 777_777
    ops = np.full(keys.size, OP_FIND, np.uint8)
    assert H.check_batch(planted, ops=ops) is None
    ops[777_777] = OP_ERASE
    assert H.check_batch(planted, ops=ops) == 777_777


def test_workload_generators_keep_the_contract(H):
    torch = pytest.importorskip("torch")
    count = 0
    for salt in range(3):
        ops, keys, vals, count, _ = W.mixed_step_t(torch, 7, count, 1 << 16, "cpu", salt=salt)
        assert H.check_batch(keys.numpy(), ops=ops.numpy()) is None
    ops, keys, _, _, _ = W.mixed_step_t(torch, 7, 1 << 14, 1 << 16, "cpu", (2, 5), (1, 5))
    assert H.check_batch(keys.numpy(), ops=ops.numpy()) is None
    rng = np.random.default_rng(5)
    live, c = W.take_keys(3, 0, 50_000)
    new, _ = W.take_keys(3, c, 20_000)
    for zipf in (None, 0.99):
        o, k, _ = W.mixed_batch(rng, live, new, 20_000, 10_000, 30_000, 3, zipf_s=zipf)
        assert H.check_batch(k, ops=o) is None


def test_resize_stream_batches_keep_the_contract(H):
    torch = pytest.importorskip("torch")
    live = torch.arange(0, 1 << 14, dtype=torch.int64)
    ctr = 1 << 14
    for b in range(4):
        ins, er = ((2, 5), (1, 5)) if b < 2 else ((1, 5), (2, 5))  # growth, then shrink
        ops, keys, _, live, ctr = W.stream_step_t(torch, 11, live, ctr, 1 << 14, "cpu", ins, er)
        assert H.check_batch(keys.numpy(), ops=ops.numpy()) is None


def test_serving_trace_requests_keep_the_contract(H):
    """Each request of the serving trace is one batch on its table (the server
    puts at most one request per table in a multi-table batch)."""
    torch = pytest.importorskip("torch")
    from paper_2510_15095_gb300 import serving as SV
    counts = [1 << 12] * 4
    before = list(counts)
    reqs = SV.make_trace(torch, 4, 40, rate_per_s=1000.0, seed=9, counts=counts, max_log2_ops=12,
                         device="cpu")
    arr = [r.arrival for r in reqs]
    assert arr[0] == 0.0 and all(b >= a for a, b in zip(arr, arr[1:]))
    added = [0] * 4
    for r in reqs:
        assert 0 <= r.table < 4 and 1 <= r.n <= 1 << 12
        assert int((r.ops == OP_INSERT).sum()) == r.n_insert
        added[r.table] += r.n_insert
        assert H.check_batch(r.keys.numpy(), ops=r.ops.numpy()) is None
    assert [c - b for c, b in zip(counts, before)] == added
