"""GPU parity of the single-kernel mixed batch (hive_execute_fused) against
the CPU oracle: per-op statuses and find values bit-exact, size, the final
key->value map and the structural invariants after every batch, including
near-full tables where eviction chains run beside the lookups of the same
launch."""
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


def up(H, a):
    return H.to_device_u32(a)


def run_batch(H, t, d, ops, keys, vals, what):
    vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals), fused=True)
    ev, est = d.execute(ops, keys, vals)
    got = st.cpu().numpy()
    bad = np.flatnonzero(got != est)
    assert bad.size == 0, f"{what}: {bad.size} status mismatches, first {bad[:5]} ops {ops[bad[:5]]} got {got[bad[:5]]} exp {est[bad[:5]]}"
    gv = H.to_host_u32(vo)
    bad = np.flatnonzero(gv != ev)
    assert bad.size == 0, f"{what}: {bad.size} value mismatches, first {bad[:5]}"


def check_image(t, d, policy=None):
    img = t.dump()
    code, where = oracle.check_image(img, img["S"], d, policy)
    assert code == 0, f"invariant {code} fails at {where}"
    assert img["size"] == len(d)


@pytest.mark.parametrize("seed,bs", [(1, 32), (2, 16)])
def test_fused_mixed_batches(H, seed, bs):
    """Moderate load: the fused launch returns what the oracle returns."""
    rng = np.random.default_rng(seed)
    t = H.HiveTable(1 << 16, bucket_slots=bs)
    d = oracle.Dict()
    live, c = W.take_keys(seed, 0, 30_000)
    t.insert(up(H, live), up(H, W.values_for(live, seed)))
    d.insert(live, W.values_for(live, seed))
    for b in range(6):
        new, c = W.take_keys(seed, c, 8_000)
        ops, keys, vals = W.mixed_batch(rng, live, new, 8_000, 6_000, 10_000, seed=seed + b,
                                        zipf_s=0.99 if b % 2 else None)
        run_batch(H, t, d, ops, keys, vals, f"batch {b}")
        live, _ = d.dump()
        assert t.size() == len(d)
        check_image(t, d)
    assert t.check() == 0
    t.close()


@pytest.mark.parametrize("slots,bs,load_pct", [(1 << 12, 32, 96), (1 << 12, 16, 95),
                                               (1 << 16, 32, 97), (1 << 16, 16, 96)])
def test_fused_eviction_beside_lookups(H, slots, bs, load_pct):
    """Near-full tables: each batch inserts new keys (which run cuckoo chains
    and stash appends) while finds and erases of live keys, Zipf-skewed onto
    few hot keys, run in the same launch."""
    seed = 30 + bs
    rng = np.random.default_rng(seed)
    t = H.HiveTable(slots, bucket_slots=bs, stash_permille=50)
    d = oracle.Dict()
    n0 = slots * load_pct // 100
    live, c = W.take_keys(seed, 0, n0)
    t.insert(up(H, live), up(H, W.values_for(live, seed)))
    d.insert(live, W.values_for(live, seed))
    n_b = max(slots // 32, 64)
    over = 0
    for b in range(10):
        new, c = W.take_keys(seed, c, n_b)
        ops, keys, vals = W.mixed_batch(rng, live, new, n_b, n_b, 4 * n_b, seed=seed + b,
                                        zipf_s=0.99)
        before = t.stats()["overflowed"]
        run_batch(H, t, d, ops, keys, vals, f"batch {b}")
        over += t.stats()["overflowed"] - before
        live, _ = d.dump()
        assert t.size() == len(d)
        check_image(t, d)
    assert over > 0, "no insert reached the eviction chain"
    assert t.check() == 0
    t.close()


@pytest.mark.parametrize("bs", [16, 32])
def test_fused_equals_phased_large(H, bs):
    """2^22 slots at 95% load, 2^20-op batches: the fused and the phased
    launches give identical per-op results and identical maps."""
    slots = 1 << 22
    rng = np.random.default_rng(7)
    keys0, c = W.take_keys(7, 0, slots * 95 // 100)
    vals0 = W.values_for(keys0, 7)
    a = H.HiveTable(slots, bucket_slots=bs)
    b = H.HiveTable(slots, bucket_slots=bs)
    for t in (a, b):
        t.insert(up(H, keys0), up(H, vals0))
    live = keys0
    for it in range(3):
        new, c = W.take_keys(7, c, 1 << 18)
        ops, keys, vals = W.mixed_batch(rng, live, new, 1 << 18, 1 << 18, 1 << 19, seed=it,
                                        zipf_s=0.99 if it else None)
        o = torch.from_numpy(ops).cuda()
        k, v = up(H, keys), up(H, vals)
        va, sa = a.execute(o, k, v, fused=True)
        vb, sb = b.execute(o, k, v)
        assert torch.equal(sa, sb) and torch.equal(va, vb)
        assert a.size() == b.size()
        erased = keys[(ops == 2) & (sb.cpu().numpy() == H.ERASED)]
        live = np.setdiff1d(np.concatenate([live, keys[ops == 0]]), erased)
    fa, ffa = a.find(up(H, live))
    fb, ffb = b.find(up(H, live))
    assert torch.equal(fa, fb) and bool((ffa == 1).all()) and bool((ffb == 1).all())
    assert a.check() == 0 and b.check() == 0
    a.close()
    b.close()


@pytest.mark.parametrize("bs", [32, 16])
def test_fused_resizable(H, bs):
    """A resizable table driven by fused batches follows the oracle's capacity
    model call by call."""
    K = 64
    t = H.HiveTable(1 << 12, max_slots=1 << 22, resizable=True, resize_batch=K, shrink=(2, 5),
                    bucket_slots=bs)
    pol = oracle.Policy((1 << 12) // bs, (1 << 22) // bs, S=bs, K=K, shrink=(2, 5))
    d = oracle.Dict()
    rng = np.random.default_rng(11)
    live = np.zeros(0, np.uint32)
    c = 0
    for b in range(10):
        grow = b < 6
        n_ins, n_er = (40_000, 10_000) if grow else (5_000, 40_000)
        n_er = min(n_er, live.size)
        new, c = W.take_keys(23, c, n_ins)
        ops, keys, vals = W.mixed_batch(rng, live, new, n_ins, n_er, 20_000, seed=b, zipf_s=0.99)
        pol.grow(len(d), n_ins)
        run_batch(H, t, d, ops, keys, vals, f"batch {b}")
        pol.shrink(len(d))
        assert t.capacity() == bs * pol.state[0], (b, t.capacity(), pol.state)
        live, _ = d.dump()
        check_image(t, d, pol)
    assert t.stats()["splits"] > 0 and t.stats()["merges"] > 0
    t.close()


def test_fused_ragged_and_reserved(H):
    t = H.HiveTable(1 << 12)
    d = oracle.Dict()
    keys, _ = W.take_keys(3, 0, 37)
    keys = keys.copy()
    keys[5] = 0xFFFFFFFF
    keys[9] = 0xFFFFFFFE
    ops = np.zeros(37, np.uint8)
    vals = W.values_for(keys, 3)
    run_batch(H, t, d, ops, keys, vals, "ragged")
    assert t.check() == 2  # HIVE_ERR_RESERVED_KEY
    vo, st = t.execute(torch.zeros(0, dtype=torch.uint8, device="cuda"),
                       torch.zeros(0, dtype=torch.int32, device="cuda"), fused=True)
    assert st.numel() == 0
    t.close()


@pytest.mark.parametrize("bs", [16, 32])
def test_fused_full_table_reports_full(H, bs):
    """A mixed batch with more new keys than slots + stash, in one kernel: the
    inserts that find no room at all report FULL and are not applied; every
    other op is, finds and erases of the preloaded keys included.  The FULL
    set is not unique, so the check is that the outcome is valid."""
    slots = 1 << 10
    keys0, c = W.take_keys(9, 0, slots // 2)
    vals0 = W.values_for(keys0, 9)
    t = H.HiveTable(slots, bucket_slots=bs, stash_permille=0)  # stash floor of 1024 words
    t.insert(up(H, keys0), up(H, vals0))
    d = oracle.Dict()
    d.insert(keys0, vals0)
    rng = np.random.default_rng(9)
    new, _ = W.take_keys(9, c, 3000)
    ops, keys, vals = W.mixed_batch(rng, keys0, new, 3000, 100, 200, seed=9)
    vo, st = t.execute(torch.from_numpy(ops).cuda(), up(H, keys), up(H, vals), fused=True)
    st = st.cpu().numpy()
    full = st == H.FULL
    assert full.any() and not (full & (ops != 0)).any()  # only inserts can be FULL
    assert full.sum() >= 3000 + slots // 2 - 100 - (slots + 1024)
    ev, est = d.execute(ops[~full], keys[~full], vals[~full])
    assert np.array_equal(st[~full], est)
    assert np.array_equal(H.to_host_u32(vo)[~full], ev)
    check_image(t, d)
    assert t.check() == 4  # HIVE_ERR_FULL
    t.close()


@pytest.mark.parametrize("bs", [16, 32])
def test_fused_version_count_wraps(H, bs):
    """Every bucket's count of finished moves starts one short of its wrap:
    chains beside Zipf-skewed finds and erases wrap it, and lookups still
    settle (no TIMEOUT) with every result the oracle's."""
    slots = 1 << 12
    seed = 40 + bs
    rng = np.random.default_rng(seed)
    t = H.HiveTable(slots, bucket_slots=bs, stash_permille=50)
    with pytest.raises(H.HiveError):
        t.debug_set_versions(1)  # words in transit: refused
    t.debug_set_versions(0xFFFF << 16)
    d = oracle.Dict()
    live, c = W.take_keys(seed, 0, slots * 95 // 100)
    t.insert(up(H, live), up(H, W.values_for(live, seed)))
    d.insert(live, W.values_for(live, seed))
    over = 0
    for b in range(6):
        new, c = W.take_keys(seed, c, 128)
        ops, keys, vals = W.mixed_batch(rng, live, new, 128, 128, 512, seed=seed + b, zipf_s=0.99)
        before = t.stats()["overflowed"]
        run_batch(H, t, d, ops, keys, vals, f"batch {b}")
        over += t.stats()["overflowed"] - before
        live, _ = d.dump()
        check_image(t, d)
    assert over > 0, "no insert reached the eviction chain"
    assert t.check() == 0  # no lookup ran out of retries
    t.close()
