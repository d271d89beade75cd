"""The device hash mixes against the oracle's, on every 32-bit key.

hive_hash computes BitHash1 and BitHash2 (Section III-C) with the same device
functions the table kernels use.  A sample of keys is compared element by
element; then all 2^32 keys are covered by a checksum: the sum over k of
(BitHash1(k) + 2^32 BitHash2(k)) * (2k + 1) modulo 2^64, per range of 2^28
keys, computed on the GPU from hive_hash's outputs and on the host by the
oracle (in threads: the oracle's C call releases the interpreter lock).  All
weights are odd, so a single wrong output anywhere changes its range's sum.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHUNK = 1 << 28


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def test_hash_sample_elementwise(H):
    rng = np.random.default_rng(123)
    keys = np.concatenate([rng.integers(0, 1 << 32, 1 << 20, dtype=np.uint64).astype(np.uint32),
                           np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF],
                                    dtype=np.uint32)])
    h1, h2 = H.hash_keys(H.to_device_u32(keys))
    assert np.array_equal(H.to_host_u32(h1), oracle.bithash_many(1, keys))
    assert np.array_equal(H.to_host_u32(h2), oracle.bithash_many(2, keys))


def _device_checksum(H, lo, hi):
    k = torch.arange(lo, hi, dtype=torch.int64, device="cuda")
    keys = torch.where(k >= (1 << 31), k - (1 << 32), k).to(torch.int32)
    h1, h2 = H.hash_keys(keys)
    w = (h1.to(torch.int64) & 0xFFFFFFFF) | ((h2.to(torch.int64) & 0xFFFFFFFF) << 32)
    s = int((w * (2 * k + 1)).sum().item())  # int64 arithmetic wraps modulo 2^64
    return s & ((1 << 64) - 1)


def test_hash_all_keys_by_checksum(H):
    ranges = [(lo, lo + CHUNK) for lo in range(0, 1 << 32, CHUNK)]
    with ThreadPoolExecutor(max_workers=16) as ex:
        futs = [ex.submit(oracle.bithash_checksum, lo, hi) for lo, hi in ranges]
        dev = [_device_checksum(H, lo, hi) for lo, hi in ranges]
        host = [f.result() for f in futs]
    bad = [i for i, (a, b) in enumerate(zip(dev, host)) if a != b]
    assert not bad, f"key ranges {bad[:4]} (of 2^28 keys each) differ"

