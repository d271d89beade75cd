"""GPU parity of the tables with 32-bit entries (hive32_*) against the CPU
oracle: a key-only set of 32-bit keys and a map of 16-bit keys to 16-bit
values, 32 slots per 128-byte bucket.  Per-op statuses and find results are
compared bit-exactly, and after each phase the table image (converted to the
oracle checker's (value, key) words) must satisfy every structural invariant."""
import numpy as np
import pytest

import oracle
from paper_2510_15095_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E32 = np.uint32(0xFFFFFFFF)


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def up(H, a):
    return H.to_device_u32(np.ascontiguousarray(a, dtype=np.uint32))


def to_words64(w32, layout):
    """32-bit entries as the oracle checker's 64-bit (value << 32 | key) words."""
    w32 = np.asarray(w32, dtype=np.uint32)
    if layout == 0:
        key = (w32 & 0xFFFF).astype(np.uint64)
        val = (w32 >> 16).astype(np.uint64)
    else:
        key = w32.astype(np.uint64)
        val = np.zeros_like(key)
    out = (val << np.uint64(32)) | key
    out[w32 == E32] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return out


def check_image(t, d):
    img = t.dump()
    assert img["pending"] == 0
    im = dict(img)
    im["buckets"] = to_words64(img["buckets"], img["layout"])
    im["stash"] = to_words64(img["stash"], img["layout"])
    code, where = oracle.check_image(im, 32, d, None)
    assert code == 0, f"invariant {code} fails at {where}"
    assert img["size"] == len(d)


def check_status(got, exp, what):
    got = got.cpu().numpy()
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]} got {got[bad[:5]]} exp {exp[bad[:5]]}"


def check_find(H, t, d, keys):
    v, f = t.find(up(H, keys))
    ev, ef = d.find(keys)
    gv, gf = H.to_host_u32(v), f.cpu().numpy()
    bad = np.flatnonzero((gv != ev) | (gf != ef))
    assert bad.size == 0, f"{bad.size} find mismatches, first keys {keys[bad[:5]]}"


@pytest.mark.parametrize("load_pct", [80, 95])
def test_key_only_set(H, load_pct):
    slots = 1 << 18
    n = slots * load_pct // 100
    keys, c = W.take_keys(41, 0, n)
    absent, _ = W.take_keys(41, c, n)
    zeros = np.zeros(n, np.uint32)
    t = H.Hive32Table(slots, H.KEY_ONLY, stash_permille=50)
    d = oracle.Dict()
    for part in (keys[: n // 2], keys[n // 2:]):
        check_status(t.insert(up(H, part)), d.insert(part, np.zeros(part.size, np.uint32)), "insert")
    # inserting present keys reports REPLACED
    check_status(t.insert(up(H, keys[:1000])), d.insert(keys[:1000], zeros[:1000]), "re-insert")
    check_find(H, t, d, np.concatenate([keys, absent]))
    check_image(t, d)
    er = keys[::3].copy()
    check_status(t.erase(up(H, er)), d.erase(er), "erase")
    check_find(H, t, d, keys)
    check_image(t, d)
    assert t.size() == len(d) and t.check() == 0
    if load_pct == 95:
        assert t.stats()["overflowed"] > 0
    t.close()


def test_key16_val16_map(H):
    """16-bit keys: 60,000 of the 65,534 valid keys in 65,536 slots (92%)."""
    rng = np.random.default_rng(5)
    keys = rng.permutation(0xFFFE)[:60_000].astype(np.uint32)
    vals = rng.integers(0, 1 << 16, keys.size).astype(np.uint32)
    t = H.Hive32Table(1 << 16, H.KEY16_VAL16, stash_permille=50)
    d = oracle.Dict()
    for part in np.array_split(np.arange(keys.size), 3):
        check_status(t.insert(up(H, keys[part]), up(H, vals[part])),
                     d.insert(keys[part], vals[part]), "insert")
    check_find(H, t, d, np.arange(0xFFFE, dtype=np.uint32))
    check_image(t, d)
    # replace a quarter with new values, erase another quarter
    rv = rng.integers(0, 1 << 16, keys.size // 4).astype(np.uint32)
    check_status(t.insert(up(H, keys[: keys.size // 4]), up(H, rv)),
                 d.insert(keys[: keys.size // 4], rv), "replace")
    er = keys[keys.size // 4: keys.size // 2].copy()
    check_status(t.erase(up(H, er)), d.erase(er), "erase")
    check_find(H, t, d, np.arange(0xFFFE, dtype=np.uint32))
    check_image(t, d)
    assert t.check() == 0
    t.close()


def test_key16_out_of_range_is_reserved(H):
    t = H.Hive32Table(1 << 10, H.KEY16_VAL16)
    keys = np.array([1, 0xFFFE, 0xFFFF, 0x10000, 7, 9], np.uint32)
    vals = np.array([5, 5, 5, 5, 1 << 16, 3], np.uint32)
    st = t.insert(up(H, keys), up(H, vals)).cpu().numpy()
    assert list(st) == [H.INSERTED, H.RESERVED_KEY, H.RESERVED_KEY, H.RESERVED_KEY,
                        H.RESERVED_KEY, H.INSERTED]
    assert t.check() == 2 and t.size() == 2
    v, f = t.find(up(H, np.array([1, 9, 7], np.uint32)))
    assert list(H.to_host_u32(v)) == [5, 3, 0] and list(f.cpu().numpy()) == [1, 1, 0]
    t.close()


@pytest.mark.parametrize("layout", [0, 1])
def test_hive32_mixed_batches(H, layout):
    rng = np.random.default_rng(12 + layout)
    if layout == 0:
        pool = rng.permutation(0xFFFE).astype(np.uint32)
        slots = 1 << 16
        live, pool = pool[:40_000], pool[40_000:]
        vmask = 0xFFFF
    else:
        pool, _ = W.take_keys(77, 0, 1 << 18)
        slots = 1 << 18
        live, pool = pool[: 150_000], pool[150_000:]
        vmask = 0
    t = H.Hive32Table(slots, layout, stash_permille=50)
    d = oracle.Dict()
    lv = (W.values_for(live, 3) & vmask).astype(np.uint32)
    check_status(t.insert(up(H, live), up(H, lv)), d.insert(live, lv), "load")
    for b in range(5):
        n_new = 2_000 if layout == 0 else 10_000
        new, pool = pool[:n_new], pool[n_new:]
        ops, keys, vals = W.mixed_batch(rng, live, new, n_new, n_new, 3 * n_new, seed=b,
                                        zipf_s=0.99 if b % 2 else None)
        vals = (vals & vmask).astype(np.uint32)
        vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals))
        ev, est = d.execute(ops, keys, vals)
        check_status(st, est, f"batch {b}")
        assert np.array_equal(H.to_host_u32(vo), ev)
        live, _ = d.dump()
        assert t.size() == len(d)
        check_image(t, d)
    assert t.check() == 0
    t.close()


def test_hive32_large_key_only(H):
    """2^24 slots at 95%, finds at 50% hit: sampled against the oracle."""
    slots = 1 << 24
    n = slots * 95 // 100
    keys, c = W.take_keys(91, 0, n)
    absent, _ = W.take_keys(91, c, 1 << 20)
    t = H.Hive32Table(slots, H.KEY_ONLY)
    st = t.insert(up(H, keys))
    assert bool((st == H.INSERTED).all())
    assert t.size() == n and t.check() == 0
    q = np.concatenate([keys[:: 16], absent])
    _, f = t.find(up(H, q))
    f = f.cpu().numpy()
    assert f[: keys[::16].size].all() and not f[keys[::16].size:].any()
    t.close()
