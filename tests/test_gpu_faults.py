"""Failure paths of the library, made to run from the host.

No test here faults, traps or hangs the GPU.  A held bucket lock (set by a
memset from the host) makes eviction waits give up after their bounded number
of tries; a staged-copy wait limit of one poll makes the probe rounds give up
while the copies are in flight; an allocation countdown on the host makes a
device allocation fail.  In every case the results must still be exactly the
oracle dictionary's, and the sticky error or return code must say what
happened.
"""
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
    yield hive
    hive.debug_fail_alloc(0)


def up(H, a):
    return H.to_device_u32(a)


def check_find(H, t, d, keys):
    v, f = t.find(up(H, keys))
    ev, ef = d.find(keys)
    assert np.array_equal(H.to_host_u32(v), ev) and np.array_equal(f.cpu().numpy(), ef)


def check_image(t, d):
    img = t.dump()
    code, where = oracle.check_image(img, img["S"], d, None)
    assert code == 0, f"invariant {code} fails at {where}"
    assert img["size"] == len(d)


@pytest.mark.parametrize("bs,slots,load", [(16, 1 << 12, 97), (32, 1 << 10, 99)])
def test_lock_timeout_falls_back_to_the_stash(H, bs, slots, load):
    """Every bucket lock held: each eviction round gives up after
    lock_spin_limit tries, the chain's word goes to the stash, TIMEOUT is
    raised, and every status and find still equals the oracle's."""
    n = slots * load // 100
    keys, c = W.take_keys(501, 0, n)
    vals = W.values_for(keys, 501)
    t = H.HiveTable(slots, bucket_slots=bs, lock_spin_limit=8)
    d = oracle.Dict()
    t.debug_hold_lock(None, True)
    st = t.insert(up(H, keys), up(H, vals)).cpu().numpy()
    assert np.array_equal(st, d.insert(keys, vals))
    s = t.stats()
    assert s["overflowed"] > 0 and s["lock_timeouts"] > 0 and s["stashed"] > 0
    assert s["lock_acquired"] == 0
    assert t.check() == 5  # HIVE_ERR_TIMEOUT, then cleared
    absent, _ = W.take_keys(501, c, n)
    check_find(H, t, d, np.concatenate([keys, absent]))
    # a mixed batch while the locks are still held: erases and finds of live
    # keys, inserts of new ones
    rng = np.random.default_rng(5)
    live, _ = d.dump()
    new, _ = W.take_keys(502, 0, 60)
    ops, mk, mv = W.mixed_batch(rng, live, new, 60, 200, 300, seed=502)
    vo, ms = t.execute(torch.from_numpy(ops).cuda(), up(H, mk), up(H, mv))
    ev, es = d.execute(ops, mk, mv)
    assert np.array_equal(ms.cpu().numpy(), es) and np.array_equal(H.to_host_u32(vo), ev)
    t.check()
    # free the locks: the image satisfies every invariant (locks 0 included)
    t.debug_hold_lock(None, False)
    check_image(t, d)
    er = keys[::4].copy()
    assert np.array_equal(t.erase(up(H, er)).cpu().numpy(), d.erase(er))
    check_find(H, t, d, keys)
    assert t.check() == 0
    t.close()


def test_single_held_lock(H):
    """One held lock: only chains that need that bucket give up."""
    slots = 1 << 12
    t = H.HiveTable(slots, bucket_slots=16, lock_spin_limit=4)
    d = oracle.Dict()
    with pytest.raises(H.HiveError):
        t.debug_hold_lock(slots // 16, True)  # not a bucket in use
    t.debug_hold_lock(3, True)
    keys, _ = W.take_keys(511, 0, slots * 97 // 100)
    vals = W.values_for(keys, 511)
    assert np.array_equal(t.insert(up(H, keys), up(H, vals)).cpu().numpy(), d.insert(keys, vals))
    check_find(H, t, d, keys)
    t.check()
    t.debug_hold_lock(3, False)
    check_image(t, d)
    t.close()


@pytest.mark.parametrize("resizable", [False, True])
def test_staged_copy_wait_gives_up(H, resizable):
    """256-byte buckets stage their probe rounds with bulk copies on an
    mbarrier.  With a wait limit of one poll, each warp's first round gives up
    while its copies are in flight, raises TIMEOUT and redoes the round (and
    every later one) with direct loads; the copies still land and are waited
    for before the warp exits.  Results equal the oracle's, and a resizable
    table ends at the capacity that the same calls give with the default
    limit."""
    slots = 1 << 16
    n = slots * 9 // 10
    keys, c = W.take_keys(521, 0, n)
    vals = W.values_for(keys, 521)
    absent, _ = W.take_keys(521, c, n)
    rng = np.random.default_rng(9)
    kw = dict(max_slots=slots * 4, resizable=True) if resizable else {}
    d = oracle.Dict()
    d.insert(keys, vals)
    live, _ = d.dump()
    new, _ = W.take_keys(522, 0, 4000)
    ops, mk, mv = W.mixed_batch(rng, live, new, 4000, 4000, 8000, seed=522)
    er = keys[1::3].copy()
    caps = []
    for limit in (1, 0):
        t = H.HiveTable(slots, bucket_slots=32, stage_wait_limit=limit, **kw)
        d = oracle.Dict()
        st = t.insert(up(H, keys), up(H, vals)).cpu().numpy()
        assert np.array_equal(st, d.insert(keys, vals))
        check_find(H, t, d, np.concatenate([keys, absent]))
        vo, ms = t.execute(torch.from_numpy(ops).cuda(), up(H, mk), up(H, mv))
        ev, es = d.execute(ops, mk, mv)
        assert np.array_equal(ms.cpu().numpy(), es) and np.array_equal(H.to_host_u32(vo), ev)
        assert np.array_equal(t.erase(up(H, er)).cpu().numpy(), d.erase(er))
        check_find(H, t, d, keys)
        assert t.check() == (5 if limit == 1 else 0)  # HIVE_ERR_TIMEOUT with one poll
        check_image(t, d)
        caps.append(t.capacity())
        t.close()
    assert caps[0] == caps[1]


def test_allocation_failure_returns_oom(H):
    """A failed device allocation returns OOM and leaves the table as it was."""
    for k in (1, 3, 6):
        H.debug_fail_alloc(k)
        with pytest.raises(H.HiveError) as e:
            H.HiveTable(1 << 12)
        assert "OOM" in str(e.value)
    H.debug_fail_alloc(0)
    t = H.HiveTable(1 << 18)
    d = oracle.Dict()
    keys, c = W.take_keys(531, 0, 1000)
    vals = W.values_for(keys, 531)
    assert np.array_equal(t.insert(up(H, keys), up(H, vals)).cpu().numpy(), d.insert(keys, vals))
    # a batch larger than the op lists makes the call reallocate them: the
    # first allocation fails, nothing is queued, the table keeps its data
    big, _ = W.take_keys(532, 0, 1 << 17)
    bvals = W.values_for(big, 532)
    H.debug_fail_alloc(1)
    with pytest.raises(H.HiveError) as e:
        t.insert(up(H, big), up(H, bvals))
    assert "OOM" in str(e.value)
    assert t.size() == 1000
    check_find(H, t, d, keys)
    # the same call succeeds once the allocations do
    assert np.array_equal(t.insert(up(H, big), up(H, bvals)).cpu().numpy(), d.insert(big, bvals))
    check_find(H, t, d, np.concatenate([keys, big]))
    # staged host-buffer calls (pageable arrays) allocate their device
    # staging on first use
    hk = torch.from_numpy(keys.view(np.int32).copy())
    hv = torch.empty(keys.size, dtype=torch.int32)
    hf = torch.empty(keys.size, dtype=torch.uint8)
    H.debug_fail_alloc(2)
    with pytest.raises(H.HiveError) as e:
        t.find_host(hk, hv, hf)
    assert "OOM" in str(e.value)
    H.debug_fail_alloc(0)
    t.find_host(hk, hv, hf)
    assert np.array_equal(hv.numpy().view(np.uint32), vals) and bool((hf.numpy() == 1).all())
    check_image(t, d)
    assert t.check() == 0
    t.close()
