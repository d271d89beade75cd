"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results must match bit-exactly: every find value and flag, every
per-op status, the size, the final key->value map, and (for resizable
tables) the capacity after every call.  After each phase the table image is
checked against the structural invariants.
"""
import numpy as np
import pytest

import oracle
from paper_2510_15095_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = 32


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def up(H, a):
    return H.to_device_u32(a)


def check_find(H, t, d, keys):
    v, f = t.find(up(H, keys))
    ev, ef = d.find(keys)
    gv, gf = H.to_host_u32(v), f.cpu().numpy()
    bad = np.flatnonzero((gv != ev) | (gf != ef))
    assert bad.size == 0, f"{bad.size} find mismatches, first at {bad[:5]}: key={keys[bad[:5]]} gpu={gv[bad[:5]]},{gf[bad[:5]]} exp={ev[bad[:5]]},{ef[bad[:5]]}"


def check_status(got, exp, what):
    got = got.cpu().numpy()
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, f"{what}: {bad.size} status mismatches, first {bad[:5]} got {got[bad[:5]]} exp {exp[bad[:5]]}"


def check_image(t, d, policy=None):
    img = t.dump()
    code, where = oracle.check_image(img, img["S"], d, policy)
    assert code == 0, f"invariant {code} fails at {where}"
    assert img["size"] == len(d)
    return img


@pytest.mark.parametrize("bs", [32, 16])
def test_plain_2e20_phases(H, bs):
    """Fixed 2^20-slot table: insert 838,861 (80%), find all plus as many
    absent keys, erase a seeded half, find again (32- and 16-slot buckets)."""
    w = W.plain_phases(seed=1)
    t = H.HiveTable(1 << 20, bucket_slots=bs)
    d = oracle.Dict()
    check_status(t.insert(up(H, w["insert_keys"]), up(H, w["insert_vals"])),
                 d.insert(w["insert_keys"], w["insert_vals"]), "insert")
    assert t.size() == 838_861
    check_find(H, t, d, w["find_keys"])
    check_image(t, d)
    check_status(t.erase(up(H, w["erase_keys"])), d.erase(w["erase_keys"]), "erase")
    check_find(H, t, d, w["find_keys"])
    check_image(t, d)
    assert t.check() == 0
    t.close()


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 4097])
def test_ragged_sizes(H, n):
    keys, c = W.take_keys(7, 0, n)
    vals = W.values_for(keys, 7)
    t = H.HiveTable(1 << 14)
    d = oracle.Dict()
    if n:
        check_status(t.insert(up(H, keys), up(H, vals)), d.insert(keys, vals), "insert")
        absent, _ = W.take_keys(7, c, n)
        q = np.concatenate([keys, absent, keys[: n // 2]])  # repeated finds are allowed
        check_find(H, t, d, q)
    else:
        e = torch.empty(0, dtype=torch.int32, device="cuda")
        t.insert(e, e)
        t.find(e)
        t.erase(e)
    assert t.size() == len(d)
    check_image(t, d)
    t.close()


def test_reserved_keys_and_key_zero(H):
    keys = np.array([0, 5, 0xFFFFFFFE, 0xFFFFFFFF, 7, 0xFFFFFFFD], np.uint32)
    vals = np.arange(6, dtype=np.uint32) + 100
    t = H.HiveTable(1 << 10)
    d = oracle.Dict()
    check_status(t.insert(up(H, keys), up(H, vals)), d.insert(keys, vals), "insert")
    assert t.check() == 2  # HIVE_ERR_RESERVED_KEY, then cleared
    assert t.check() == 0
    check_find(H, t, d, keys)
    check_status(t.erase(up(H, keys[::-1].copy())), d.erase(keys[::-1].copy()), "erase")
    check_image(t, d)
    t.close()


def test_replace_then_find(H):
    keys, _ = W.take_keys(3, 0, 50_000)
    t = H.HiveTable(1 << 17)
    d = oracle.Dict()
    for rnd in range(3):
        vals = W.values_for(keys, 100 + rnd)
        check_status(t.insert(up(H, keys), up(H, vals)), d.insert(keys, vals), f"insert {rnd}")
    check_find(H, t, d, keys)
    assert t.stats()["replaced"] == 100_000
    check_image(t, d)
    t.close()


@pytest.mark.parametrize("load_pct,slots,bs", [(95, 1 << 12, 32), (99, 1 << 12, 32),
                                               (95, 1 << 16, 32), (98, 1 << 16, 32),
                                               (95, 1 << 12, 16), (98, 1 << 16, 16)])
def test_high_load_eviction_and_stash(H, load_pct, slots, bs):
    """Near-full tables exercise steps 3 and 4 (eviction, stash)."""
    n = slots * load_pct // 100
    keys, c = W.take_keys(17 + load_pct, 0, n)
    vals = W.values_for(keys, 17)
    t = H.HiveTable(slots, stash_permille=50, bucket_slots=bs)
    d = oracle.Dict()
    # two halves so the second insert meets a loaded table
    for part in (keys[: n // 2], keys[n // 2:]):
        check_status(t.insert(up(H, part), up(H, W.values_for(part, 17))),
                     d.insert(part, W.values_for(part, 17)), "insert")
    stats = t.stats()
    assert stats["overflowed"] > 0
    absent, _ = W.take_keys(17 + load_pct, c, n)
    check_find(H, t, d, np.concatenate([keys, absent]))
    img = check_image(t, d)
    # erase a third, including stashed keys, then refill and re-check
    er = keys[::3].copy()
    check_status(t.erase(up(H, er)), d.erase(er), "erase")
    check_find(H, t, d, keys)
    check_image(t, d)
    check_status(t.insert(up(H, er), up(H, vals[::3].copy())), d.insert(er, vals[::3].copy()), "reinsert")
    check_find(H, t, d, keys)
    check_image(t, d)
    assert t.check() == 0
    t.close()


def test_full_table_reports_full(H):
    """More keys than slots + stash: FULL ops are not applied; every other op is.
    The FULL set is not unique, so the check is that the outcome is valid."""
    slots = 1 << 10
    n = 3000
    keys, _ = W.take_keys(5, 0, n)
    vals = W.values_for(keys, 5)
    t = H.HiveTable(slots, stash_permille=0)  # stash floor of 1024 words
    st = t.insert(up(H, keys), up(H, vals)).cpu().numpy()
    full = st == H.FULL
    assert set(np.unique(st)) <= {H.INSERTED, H.FULL}
    assert full.sum() >= n - (slots + 1024)  # at most slots + stash words are stored
    d = oracle.Dict()
    d.insert(keys[~full], vals[~full])
    check_find(H, t, d, keys)
    check_image(t, d)
    assert t.check() == 4  # HIVE_ERR_FULL
    t.close()


@pytest.mark.parametrize("seed,bs", [(1, 32), (2, 32), (3, 32), (4, 16)])
def test_mixed_batches(H, seed, bs):
    rng = np.random.default_rng(seed)
    t = H.HiveTable(1 << 16, bucket_slots=bs)
    d = oracle.Dict()
    live, c = W.take_keys(seed, 0, 30_000)
    check_status(t.insert(up(H, live), up(H, W.values_for(live, seed))),
                 d.insert(live, W.values_for(live, seed)), "load")
    for b in range(6):
        new, c = W.take_keys(seed, c, 8_000)
        ops, keys, vals = W.mixed_batch(rng, live, new, 8_000, 6_000, 10_000, seed=seed + b,
                                        zipf_s=0.99 if b % 2 else None)
        vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals))
        ev, est = d.execute(ops, keys, vals)
        check_status(st, est, f"batch {b}")
        assert np.array_equal(H.to_host_u32(vo), ev)
        live, _ = d.dump()
        assert t.size() == len(d)
        check_image(t, d)
    t.close()


@pytest.mark.parametrize("bs", [16, 32])
def test_large_mixed_batches_claim_phase(H, bs):
    """Mixed batches of 2^18 ops and more claim their new keys in a second
    kernel, after the batch's finds, erases and replaces; at 95% load many of
    them find both buckets full when probed and are placed into slots the
    same batch's erases freed, or go on to eviction.  Every status, value,
    size and invariant equals the oracle's, batch after batch."""
    rng = np.random.default_rng(77 + bs)
    slots = 1 << 20
    t = H.HiveTable(slots, bucket_slots=bs)
    d = oracle.Dict()
    live, c = W.take_keys(77, 0, slots * 95 // 100)
    check_status(t.insert(up(H, live), up(H, W.values_for(live, 77))),
                 d.insert(live, W.values_for(live, 77)), "load")
    for b, n in enumerate((1 << 18, 3 << 18)):
        new, c = W.take_keys(77, c, n // 4)
        ops, keys, vals = W.mixed_batch(rng, live, new, n // 4, n // 4, n // 2, seed=78 + b,
                                        zipf_s=0.99 if b else None)
        vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals))
        ev, est = d.execute(ops, keys, vals)
        check_status(st, est, f"batch {b}")
        assert np.array_equal(H.to_host_u32(vo), ev)
        live, _ = d.dump()
        assert t.size() == len(d)
        check_image(t, d)
    s = t.stats()
    assert s["overflowed"] > 0 and s["claimed_fast"] > 0
    assert t.check() == 0
    t.close()


@pytest.mark.parametrize("bs,on_demand", [(32, False), (16, False), (32, True), (16, True)])
def test_resizable_grow_and_shrink(H, bs, on_demand):
    """Linear-hashing growth and contraction track the oracle's capacity model
    call by call, with invariants (including the load-factor band) after each;
    bucket memory allocated up front or mapped on demand."""
    K = 64
    t = H.HiveTable(1 << 12, max_slots=1 << 22, resizable=True, resize_batch=K, shrink=(2, 5),
                    bucket_slots=bs, map_on_demand=on_demand)
    pol = oracle.Policy((1 << 12) // bs, (1 << 22) // bs, S=bs, K=K, shrink=(2, 5))
    d = oracle.Dict()
    rng = np.random.default_rng(9)
    live = np.zeros(0, np.uint32)
    c = 0
    for b in range(12):
        grow = b < 7
        n_ins, n_er = (40_000, 10_000) if grow else (5_000, 40_000)
        n_er = min(n_er, live.size)
        new, c = W.take_keys(21, c, n_ins)
        ops, keys, vals = W.mixed_batch(rng, live, new, n_ins, n_er, 20_000, seed=b, zipf_s=0.99)
        pol.grow(len(d), n_ins)
        vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals))
        ev, est = d.execute(ops, keys, vals)
        pol.shrink(len(d))
        check_status(st, est, f"batch {b}")
        assert np.array_equal(H.to_host_u32(vo), ev)
        assert t.capacity() == bs * pol.state[0], (b, t.capacity(), pol.state)
        live, _ = d.dump()
        check_image(t, d, pol)
    assert t.stats()["splits"] > 0 and t.stats()["merges"] > 0
    t.close()


def test_resizable_bulk_insert_erase(H):
    t = H.HiveTable(1 << 10, max_slots=1 << 24, resizable=True, resize_batch=1024)
    pol = oracle.Policy(32, 1 << 19, K=1024)
    d = oracle.Dict()
    keys, _ = W.take_keys(4, 0, 1 << 20)
    vals = W.values_for(keys, 4)
    for part in np.array_split(np.arange(keys.size), 4):
        pol.grow(len(d), part.size)
        check_status(t.insert(up(H, keys[part]), up(H, vals[part])), d.insert(keys[part], vals[part]), "ins")
        pol.shrink(len(d))
        assert t.capacity() == S * pol.state[0]
    check_find(H, t, d, keys)
    check_image(t, d, pol)
    for part in np.array_split(np.arange(keys.size), 4):
        check_status(t.erase(up(H, keys[part])), d.erase(keys[part]), "erase")
        pol.shrink(len(d))
        assert t.capacity() == S * pol.state[0]
        check_image(t, d, pol)
    assert t.size() == 0
    t.close()


@pytest.mark.parametrize("bs", [16, 32])
def test_2e26_slots_95pct_load(H, bs):
    """The load-factor sweep table at full size: 2^26 slots filled to 95%
    (63,753,421 keys) in one launch, then 2^26 finds at 50% hit rate and the
    2^24-op mixed batch (1:2:1 at 95%), in the bench's launch configuration
    (16-slot buckets with the persisting L2 window, the bench's tuned choice),
    and with the paper's 32-slot buckets, whose rounds stage through bulk
    copies.  Every result is checked
    against the properties that hold at any size (hit -> the key's value,
    miss -> not found, new insert -> INSERTED, erase of a live key -> ERASED);
    a 2^21 sample of the finds is checked against the oracle; the dump passes
    the invariants."""
    slots = 1 << 26
    w = W.fill_and_query(seed=2, slots=slots, load_num=19, load_den=20, n_find=1 << 26)
    t = H.HiveTable(slots, bucket_slots=bs, l2_persist=bs == 16)
    st = t.insert(up(H, w["insert_keys"]), up(H, w["insert_vals"])).cpu().numpy()
    assert (st == H.INSERTED).all()
    assert t.size() == w["insert_keys"].size
    v, f = t.find(up(H, w["find_keys"]))
    gv, gf = H.to_host_u32(v), f.cpu().numpy().astype(bool)
    hit = w["is_hit"]
    assert np.array_equal(gf, hit)
    assert np.array_equal(gv[hit], W.values_for(w["find_keys"][hit], 2))
    assert (gv[~hit] == 0).all()
    rng = np.random.default_rng(0)
    d = oracle.Dict()
    d.insert(w["insert_keys"], w["insert_vals"])
    sample = rng.integers(0, w["find_keys"].size, 1 << 21)
    ev, ef = d.find(w["find_keys"][sample])
    assert np.array_equal(gv[sample], ev) and np.array_equal(gf[sample].astype(np.uint8), ef)
    # the mixed batch: new inserts, erases of live keys, finds of other live keys
    n_mix = 1 << 24
    new, _ = W.take_keys(2, 1 << 31, n_mix // 4)
    ops, keys, vals = W.mixed_batch(rng, w["insert_keys"], new, n_mix // 4, n_mix // 4,
                                    n_mix // 2, seed=2)
    vo, ms = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals))
    vo, ms = H.to_host_u32(vo), ms.cpu().numpy()
    ins, era, fnd = ops == 0, ops == 2, ops == 1
    assert (ms[ins] == H.INSERTED).all() and (ms[era] == H.ERASED).all()
    assert (ms[fnd] == H.FOUND).all()
    assert np.array_equal(vo[fnd], W.values_for(keys[fnd], 2))
    d.execute(ops, keys, vals)
    assert t.size() == len(d)
    check_image(t, d)
    assert t.check() == 0
    t.close()


@pytest.mark.parametrize("way", ["direct", "staged"])
def test_host_buffer_calls_match_device_calls(H, way, monkeypatch):
    """hive_*_host on host arrays: with pinned arrays on a GPU with coherent
    host access the kernels work on them in place ("direct"); with
    HIVE_HOSTIO_STAGED=1 they stream through device staging in chunks of
    2^22 ops ("staged").  With 5 million ops (two full chunks and a ragged
    tail) the results must equal the device-pointer calls bit for bit; the
    mixed batch uses pageable buffers, which always take the staged way."""
    if way == "staged":
        monkeypatch.setenv("HIVE_HOSTIO_STAGED", "1")
    n = 5_000_000
    keys, c = W.take_keys(41, 0, n)
    vals = W.values_for(keys, 41)
    absent, _ = W.take_keys(41, c, n // 2)
    q = np.concatenate([keys[::2], absent])
    a = H.HiveTable(1 << 23)
    b = H.HiveTable(1 << 23)
    st_a = a.insert(up(H, keys), up(H, vals)).cpu()
    hk = torch.from_numpy(keys.view(np.int32)).pin_memory()
    hv = torch.from_numpy(vals.view(np.int32)).pin_memory()
    st_b = torch.empty(n, dtype=torch.uint8).pin_memory()
    b.insert_host(hk, hv, st_b)
    assert torch.equal(st_a, st_b)
    va, fa = a.find(up(H, q))
    hq = torch.from_numpy(q.view(np.int32)).pin_memory()
    vb = torch.empty(q.size, dtype=torch.int32).pin_memory()
    fb = torch.empty(q.size, dtype=torch.uint8).pin_memory()
    if way == "direct" and H.host_direct_access():
        # in place: the table has no staging yet and this call allocates none,
        # so a failing allocation is not met
        H.debug_fail_alloc(1)
    try:
        b.find_host(hq, vb, fb)
    finally:
        H.debug_fail_alloc(0)
    assert torch.equal(va.cpu(), vb) and torch.equal(fa.cpu(), fb)
    # found flags may be left out
    vb2 = torch.empty(q.size, dtype=torch.int32).pin_memory()
    b.find_host(hq, vb2)
    assert torch.equal(vb, vb2)
    rng = np.random.default_rng(4)
    new, _ = W.take_keys(41, c + n, 100_000)
    ops, mk, mv = W.mixed_batch(rng, keys, new, 100_000, 100_000, 300_000, seed=41)
    vo_a, st_a = a.execute(torch.from_numpy(ops).cuda(), up(H, mk), up(H, mv))
    vo_b = torch.empty(ops.size, dtype=torch.int32)
    st_b = torch.empty(ops.size, dtype=torch.uint8)  # pageable
    b.execute_host(torch.from_numpy(ops), torch.from_numpy(mk.view(np.int32)),
                   torch.from_numpy(mv.view(np.int32)), vo_b, st_b)
    assert torch.equal(vo_a.cpu(), vo_b) and torch.equal(st_a.cpu(), st_b)
    # the same mixed batch shape again, pinned, on both tables
    ops2, mk2, mv2 = W.mixed_batch(rng, keys, new, 50_000, 100_000, 200_000, seed=42)
    vo_a, st_a = a.execute(torch.from_numpy(ops2).cuda(), up(H, mk2), up(H, mv2))
    vo_b = torch.empty(ops2.size, dtype=torch.int32).pin_memory()
    st_b = torch.empty(ops2.size, dtype=torch.uint8).pin_memory()
    b.execute_host(torch.from_numpy(ops2).pin_memory(),
                   torch.from_numpy(mk2.view(np.int32)).pin_memory(),
                   torch.from_numpy(mv2.view(np.int32)).pin_memory(), vo_b, st_b)
    assert torch.equal(vo_a.cpu(), vo_b) and torch.equal(st_a.cpu(), st_b)
    assert a.size() == b.size()
    assert a.check() == 0 and b.check() == 0
    a.close()
    b.close()


def test_resizable_memory_follows_capacity(H):
    """A resizable table maps bucket memory as it splits and returns it after
    merges: committed bucket bytes grow and shrink with the capacity inside a
    bucket range reserved once for max_slots.  (The per-batch work lists grow
    with the largest batch seen, on both counts.)"""
    t = H.HiveTable(1 << 12, max_slots=1 << 24, resizable=True, resize_batch=1024,
                    map_on_demand=True)
    c0, r0 = t.memory()
    keys, _ = W.take_keys(55, 0, 1 << 21)
    vals = W.values_for(keys, 55)
    t.insert(up(H, keys), up(H, vals))
    c1, r1 = t.memory()
    # at least 2^21 keys worth of the reserved bucket range got mapped
    assert (r0 - c0) - (r1 - c1) >= 16 * (1 << 20), (c0, r0, c1, r1)
    d = oracle.Dict()
    d.insert(keys, vals)
    check_find(H, t, d, keys[::7])
    t.erase(up(H, keys[: (1 << 21) - (1 << 14)]))
    d.erase(keys[: (1 << 21) - (1 << 14)])
    c2, r2 = t.memory()
    assert r2 == r1 and c2 < c1 - 12 * (1 << 20), (c0, c1, c2)  # the bucket memory went back
    check_find(H, t, d, keys[::7])
    check_image(t, d)
    # grows again into freshly mapped, freshly emptied memory
    t.insert(up(H, keys[: 1 << 20]), up(H, vals[: 1 << 20]))
    d.insert(keys[: 1 << 20], vals[: 1 << 20])
    check_find(H, t, d, keys[::5])
    check_image(t, d)
    t.close()
