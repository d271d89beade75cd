"""Pins for the oracle's dictionary (Section III-D of the paper).

The dictionary is checked against a brute-force linear-scan list map on tiny
random op sequences, against the closed form size = inserted - erased, and for
the order independence that the batch contract promises.  The parallel CPU
baseline (the dictionary sharded by key over host threads) is checked against
the dictionary.
"""
import numpy as np
import pytest

import oracle
from oracle import ERASED, FOUND, INSERTED, NOT_FOUND, REPLACED, RESERVED
from paper_2510_15095_gb300 import workload as W


class BruteMap:
    """Set semantics of Section III-D on a Python list, one linear scan per op."""

    def __init__(self):
        self.items = []  # list of [key, value]

    def _index(self, k):
        for i, kv in enumerate(self.items):
            if kv[0] == k:
                return i
        return -1

    def insert(self, k, v):
        if k >= 0xFFFFFFFE:
            return RESERVED
        i = self._index(k)
        if i < 0:
            self.items.append([k, v])
            return INSERTED
        self.items[i][1] = v
        return REPLACED

    def erase(self, k):
        if k >= 0xFFFFFFFE:
            return RESERVED
        i = self._index(k)
        if i < 0:
            return NOT_FOUND
        self.items.pop(i)
        return ERASED

    def find(self, k):
        if k >= 0xFFFFFFFE:
            return 0, 0
        i = self._index(k)
        return (self.items[i][1], 1) if i >= 0 else (0, 0)


def _random_ops(rng, n, key_space):
    keys = rng.integers(0, key_space, n).astype(np.uint32)
    # sprinkle reserved keys and key 0
    special = rng.random(n)
    keys[special < 0.03] = 0xFFFFFFFF
    keys[(special >= 0.03) & (special < 0.05)] = 0xFFFFFFFE
    keys[(special >= 0.05) & (special < 0.07)] = 0
    vals = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    ops = rng.integers(0, 3, n).astype(np.uint8)
    return ops, keys, vals


@pytest.mark.parametrize("seed", range(40))
def test_execute_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    d = oracle.Dict()
    b = BruteMap()
    for _ in range(4):
        n = int(rng.integers(0, 200))
        ops, keys, vals = _random_ops(rng, n, key_space=int(rng.integers(1, 64)))
        out, st = d.execute(ops, keys, vals)
        for i in range(n):
            k, v = int(keys[i]), int(vals[i])
            if ops[i] == oracle.OP_INSERT:
                exp_st, exp_v = b.insert(k, v), 0
            elif ops[i] == oracle.OP_ERASE:
                exp_st, exp_v = b.erase(k), 0
            else:
                exp_v, f = b.find(k)
                exp_st = RESERVED if k >= 0xFFFFFFFE else (FOUND if f else NOT_FOUND)
            assert st[i] == exp_st, (i, k)
            assert out[i] == exp_v, (i, k)
        kk, vv = d.dump()
        ref = sorted((kv[0], kv[1]) for kv in b.items)
        assert list(zip(kk.tolist(), vv.tolist())) == ref


@pytest.mark.parametrize("seed", range(10))
def test_bulk_calls_match_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    d = oracle.Dict()
    b = BruteMap()
    keys = rng.integers(0, 50, 120).astype(np.uint32)
    vals = rng.integers(0, 1000, 120).astype(np.uint32)
    st = d.insert(keys, vals)
    assert [b.insert(int(k), int(v)) for k, v in zip(keys, vals)] == st.tolist()
    q = rng.integers(0, 60, 80).astype(np.uint32)
    v, f = d.find(q)
    assert [b.find(int(k)) for k in q] == list(zip(v.tolist(), f.tolist()))
    e = rng.integers(0, 60, 40).astype(np.uint32)
    st = d.erase(e)
    assert [b.erase(int(k)) for k in e] == st.tolist()
    assert len(d) == len(b.items)


def test_size_closed_form():
    """size = (#INSERTED) - (#ERASED) over any op stream."""
    rng = np.random.default_rng(7)
    d = oracle.Dict()
    ins = era = 0
    for _ in range(30):
        ops, keys, vals = _random_ops(rng, 500, key_space=300)
        _, st = d.execute(ops, keys, vals)
        ins += int((st == INSERTED).sum())
        era += int((st == ERASED).sum())
        assert len(d) == ins - era


def test_reserved_keys_never_stored():
    d = oracle.Dict()
    st = d.insert([0xFFFFFFFF, 0xFFFFFFFE, 0, 5], [1, 2, 3, 4])
    assert st.tolist() == [RESERVED, RESERVED, INSERTED, INSERTED]
    v, f = d.find([0xFFFFFFFF, 0xFFFFFFFE, 0, 5])
    assert f.tolist() == [0, 0, 1, 1] and v.tolist() == [0, 0, 3, 4]
    assert d.erase([0xFFFFFFFF]).tolist() == [RESERVED]
    assert len(d) == 2


@pytest.mark.parametrize("seed", range(10))
def test_contract_batches_are_order_independent(seed):
    """Under the batch contract (no key in two updates, no key both updated and
    searched) any permutation of a batch gives the same per-op results and map:
    the property that makes GPU results unique and comparable bit-exactly."""
    rng = np.random.default_rng(seed)
    base = np.unique(rng.integers(0, 10_000, 400)).astype(np.uint32)
    pool = rng.permutation(np.arange(10_000, dtype=np.uint32))
    upd = pool[:300]
    rest = np.setdiff1d(pool[300:1000], upd)
    ops = np.concatenate([np.zeros(150, np.uint8), np.full(150, 2, np.uint8), np.ones(200, np.uint8)])
    keys = np.concatenate([upd[:150], upd[150:], rng.choice(rest, 200)]).astype(np.uint32)
    vals = rng.integers(0, 2**32, ops.size, dtype=np.uint64).astype(np.uint32)
    results = []
    for trial in range(3):
        perm = rng.permutation(ops.size)
        d = oracle.Dict()
        d.insert(base, base * 3)
        out, st = d.execute(ops[perm], keys[perm], vals[perm])
        inv = np.argsort(perm)
        results.append((out[inv].tolist(), st[inv].tolist(), [a.tolist() for a in d.dump()]))
    assert results[0] == results[1] == results[2]


@pytest.mark.parametrize("threads", [1, 2, 5])
def test_sharded_baseline_equals_the_dictionary(threads):
    """The parallel CPU baseline (key-sharded maps on host threads) gives every
    per-op result the single dictionary gives, whatever the thread count."""
    rng = np.random.default_rng(70 + threads)
    keys, c = W.take_keys(71, 0, 20_000)
    vals = W.values_for(keys, 71)
    keys[::997] = 0xFFFFFFFF  # reserved keys go through too
    absent, _ = W.take_keys(71, c, 10_000)
    fk = np.concatenate([keys[::2], absent])
    rng.shuffle(fk)
    d = oracle.Dict()
    ist = d.insert(keys, vals)
    fv, ff = d.find(fk)
    live, _ = d.dump()
    new, _ = W.take_keys(72, 0, 3_000)
    ops, mk, mv = W.mixed_batch(rng, live, new, 3_000, 3_000, 6_000, seed=72)
    mvo, mst = d.execute(ops, mk, mv)
    sec, a, b, f, e, g = oracle.sharded_step(threads, keys, vals, fk, ops, mk, mv)
    assert sec > 0
    for got, exp in ((a, ist), (b, fv), (f, ff), (e, mvo), (g, mst)):
        assert np.array_equal(got, exp)
