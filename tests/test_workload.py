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


def _inv_xorshift(y, s):
    x = y
    for _ in range(32 // s + 1):
        x = y ^ (x >> s)
    return x & 0xFFFFFFFF


def test_splitmix32_undoes_step_by_step():
    """The value generator is the golden-ratio increment followed by the
    MurmurHash3 finalizer; undoing each published step in reverse order must
    give the input back (a wrong constant, shift or order breaks it)."""
    xs = np.array([0, 1, 2, 0x61C88646, 0x61C88647, 0xFFFFFFFF, 0xDEADBEEF]
                  + np.random.default_rng(3).integers(0, 1 << 32, 3000).tolist(), np.uint64)
    ys = W.splitmix32(xs)
    m = 1 << 32
    for x, y in zip(xs.tolist(), ys.tolist()):
        z = _inv_xorshift(int(y), 16)
        z = (z * pow(0xC2B2AE35, -1, m)) % m
        z = _inv_xorshift(z, 13)
        z = (z * pow(0x85EBCA6B, -1, m)) % m
        z = _inv_xorshift(z, 16)
        assert (z - 0x9E3779B9) % m == x
    assert int(W.splitmix32(np.array([(1 << 32) - 0x9E3779B9]))[0]) == 0  # fmix32(0) = 0


def test_torch_generators_match_numpy():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.arange(0, 5000, dtype=np.uint64),
                        np.random.default_rng(4).integers(0, 1 << 32, 20000).astype(np.uint64),
                        np.array([(1 << 32) - 1, (1 << 32) - 2], np.uint64)])
    xt = torch.from_numpy(x.astype(np.int64))
    assert np.array_equal(W.splitmix32_t(xt).numpy().astype(np.uint64), W.splitmix32(x).astype(np.uint64))
    for bits in (16, 32):
        xb = x & np.uint64((1 << bits) - 1)
        got = W.feistel_bits_t(torch.from_numpy(xb.astype(np.int64)), 9, bits).numpy()
        assert np.array_equal(got.astype(np.uint64), W.feistel_bits(xb, 9, bits).astype(np.uint64))
