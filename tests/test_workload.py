"""Checks of the seeded input generators (not of the table)."""
import numpy as np
import pytest

from paper_2510_15095_gb300 import workload as W


def test_feistel_is_bijection_on_small_domains():
    for bits in (2, 4, 8, 12, 16):
        x = np.arange(1 << bits, dtype=np.uint64)
        y = W.feistel_bits(x, seed=3, bits=bits)
        assert np.array_equal(np.sort(y), x)


def test_take_keys_unique_disjoint_in_range():
    a, c = W.take_keys(9, 0, 200_000)
    b, _ = W.take_keys(9, c, 100_000)
    assert a.dtype == np.uint32 and a.size == 200_000 and b.size == 100_000
    allk = np.concatenate([a, b])
    assert np.unique(allk).size == allk.size
    assert allk.min() >= 1 and allk.max() <= 0xFFFFFFFD


def test_plain_phase_sizes():
    w = W.plain_phases(seed=1)
    assert w["insert_keys"].size == 838_861
    assert w["find_keys"].size == 2 * 838_861
    assert w["erase_keys"].size == 419_430
    assert np.unique(w["erase_keys"]).size == 419_430


def test_permute_index_is_permutation():
    for n in (1, 2, 7, 1000, 4097):
        y = W.permute_index(np.arange(n), n, seed=4)
        assert np.array_equal(np.sort(y), np.arange(n))


def test_zipf_frequencies():
    rng = np.random.default_rng(0)
    n, s, cnt = 50, 0.99, 400_000
    r = W.zipf_ranks(rng, n, s, cnt)
    assert r.min() >= 1 and r.max() <= n
    pmf = np.arange(1, n + 1, dtype=np.float64) ** -s
    pmf /= pmf.sum()
    obs = np.bincount(r, minlength=n + 1)[1:] / cnt
    assert np.max(np.abs(obs - pmf)) < 0.004


def test_mixed_batch_contract():
    rng = np.random.default_rng(2)
    live, c = W.take_keys(5, 0, 10_000)
    new, _ = W.take_keys(5, c, 5_000)
    ops, keys, vals = W.mixed_batch(rng, live, new, 4000, 2000, 4000, seed=5, zipf_s=0.99)
    upd = keys[ops != W.OP_FIND]
    assert np.unique(upd).size == upd.size
    finds = keys[ops == W.OP_FIND]
    assert not np.isin(finds, upd).any()
    assert np.isin(keys[ops == W.OP_ERASE], live).all()
    assert not np.isin(keys[ops == W.OP_INSERT], live).any()
