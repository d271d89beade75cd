"""Hash-quality study of Section III-C: the Collision Speedup Ratio
CSR = E[Y] / Y_observed (Theorem 1) of BitHash1 and BitHash2 for m = 512^2
buckets and n from 2^11 to 2048^2 keys.

The paper reports that BitHash clusters mildly at low load (CSR < 1) and
converges to uniform spread as n grows.  With consecutive keys, BitHash1
shows exactly that; both mixes are within 1% of uniform hashing once n is a
sizeable fraction of m, for consecutive and random keys alike.  (The figure's
values are not recoverable from the paper, so only these trends are checked.)
"""
import numpy as np
import pytest

import oracle

M = 512 * 512


def expected_collisions(n, m):
    return n - m * (1.0 - (1.0 - 1.0 / m) ** n)


def csr(which, keys):
    b = oracle.bithash_many(which, keys) % M
    return expected_collisions(keys.size, M) / max(keys.size - np.unique(b).size, 1)


def test_bithash1_clusters_mildly_at_low_load():
    for n in (1 << 11, 1 << 13, 1 << 15):
        c = csr(1, np.arange(1, n + 1, dtype=np.uint32))
        assert 0.8 < c < 1.0, (n, c)


@pytest.mark.parametrize("which", [1, 2])
@pytest.mark.parametrize("kind", ["consecutive", "random"])
def test_converges_to_uniform(which, kind):
    rng = np.random.default_rng(which)
    for n in (1 << 17, 1 << 19, 2048 * 2048):
        keys = (np.arange(1, n + 1, dtype=np.uint32) if kind == "consecutive"
                else rng.choice(1 << 32, n, replace=False).astype(np.uint32))
        c = csr(which, keys)
        assert abs(c - 1.0) < 0.01, (which, kind, n, c)


def _fill_overflow(hashes, n_buckets, slots, n_keys):
    """Greedy balanced placement (the bucket with the most free slots, ties
    to the earlier hash) of n_keys keys; returns the fraction of keys whose
    candidate buckets were all full (the ones that would need eviction)."""
    load = np.zeros(n_buckets, np.int64)
    cand = np.stack([h % n_buckets for h in hashes], axis=1)
    over = 0
    for row in cand[:n_keys]:
        free = slots - load[row]
        j = int(np.argmax(free))
        if free[j] <= 0:
            over += 1
            continue
        load[row[j]] += 1
    return over / n_keys


def test_three_choices_cut_overflow_but_two_suffice():
    """Section V (hash functions): a third hash function improves the spread
    of keys only marginally.  With balanced two-choice placement of 16-slot
    buckets filled to 95%, few keys find both buckets full; a third choice
    (here a Fibonacci multiply-shift of our own, since the paper's third
    function is third-party code) removes most of those, at the price of one
    more bucket probe for every lookup."""
    n_buckets, slots = 1 << 12, 16
    n = n_buckets * slots * 95 // 100
    keys = np.arange(1, n + 1, dtype=np.uint32) * np.uint32(2654435761)
    h1 = oracle.bithash_many(1, keys).astype(np.int64)
    h2 = oracle.bithash_many(2, keys).astype(np.int64)
    h3 = ((keys.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(32)).astype(np.int64)
    two = _fill_overflow([h1, h2], n_buckets, slots, n)
    three = _fill_overflow([h1, h2, h3], n_buckets, slots, n)
    assert two < 0.02          # two choices already place more than 98% at 95% load
    assert three < two / 2     # a third choice removes most of the rest
