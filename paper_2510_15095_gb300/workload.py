"""Seeded synthetic workloads for the Hive table (inputs only; no table arithmetic).

This module is the one piece of code that both the CPU oracle tests and the CUDA
path's tests and benchmark use.  It holds only input generation: unique 32-bit
key streams, the value function, hit/miss query mixes and a Zipf sampler.  None
of the table's own arithmetic (hashing, bucket addressing, placement, resize
policy) lives here.

The paper evaluates on synthetic, uniformly distributed 32-bit key/value pairs
(Section V, "Experimental Setup"); everything below produces such inputs from a
seed so that every run is reproducible.

* Unique keys: a 4-round Feistel network over 32-bit counters is a bijection,
  so distinct counters give distinct keys.  Keys outside [1, 2^32-3] are
  dropped, which keeps the table's reserved words out of the workload.
  Absent keys come from counters beyond those used for inserted keys, so they
  are absent by construction.
* Values: ``splitmix32(key ^ seed)``: add the 32-bit golden-ratio increment
  0x9E3779B9, then apply the public-domain MurmurHash3 32-bit finalizer
  (Appleby's ``fmix32``).
* Zipf(s): rejection-inversion sampling (Hoermann and Derflinger, "Rejection-
  inversion to generate variates from monotone discrete distributions", 1996)
  over ranks 1..N, with ranks mapped to keys by a seeded cycle-walking Feistel
  permutation of [0, N).
"""
from __future__ import annotations

import numpy as np

U32 = np.uint32
MASK32 = 0xFFFFFFFF
KEY_MIN = 1
KEY_MAX = 0xFFFFFFFD  # workload keys lie in [1, 2^32-3]

OP_INSERT = 0
OP_FIND = 1
OP_ERASE = 2


def _u32(x):
    return np.asarray(x, dtype=np.uint64) & MASK32


def _round_keys(seed: int, rounds: int = 4):
    """Per-round 32-bit keys derived from the seed with a simple LCG walk."""
    out = []
    s = (int(seed) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF
    for _ in range(rounds):
        s = (s * 6364136223846793005 + 1442695040888963407) & 0xFFFFFFFFFFFFFFFF
        out.append((s >> 32) & 0xFFFFFFFF)
    return out


def _feistel_f(r: np.ndarray, k: int, half_bits: int) -> np.ndarray:
    """Round function on a half word (uint64 arrays holding half_bits-bit values)."""
    hm = (1 << half_bits) - 1
    x = (r ^ (k & hm)) & hm
    x = (x * 0x2C1B3C6D + (k >> 7)) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x297A2D39) & 0xFFFFFFFF
    x ^= x >> 12
    return x & hm


def feistel_bits(x, seed: int, bits: int) -> np.ndarray:
    """A seeded bijection on ``bits``-bit integers (bits even, 2..32)."""
    assert bits % 2 == 0 and 2 <= bits <= 32
    half = bits // 2
    hm = (1 << half) - 1
    x = np.asarray(x, dtype=np.uint64)
    left = (x >> half) & hm
    right = x & hm
    for k in _round_keys(seed):
        left, right = right, left ^ _feistel_f(right, k, half)
    return ((left << half) | right).astype(np.uint64)


def feistel32(x, seed: int) -> np.ndarray:
    """Seeded bijection on 32-bit counters."""
    return feistel_bits(x, seed, 32)


def take_keys(seed: int, counter0: int, n: int):
    """The first ``n`` valid keys of stream ``seed`` from counter ``counter0`` on.

    Returns ``(keys uint32[n], next_counter)``.  Keys drawn from disjoint
    counter ranges of one stream are disjoint sets.
    """
    n = int(n)
    if n == 0:
        return np.zeros(0, dtype=U32), counter0
    extra = 64
    while True:
        ctr = np.arange(counter0, counter0 + n + extra, dtype=np.uint64)
        assert ctr[-1] <= MASK32, "key stream exhausted"
        k = feistel32(ctr, seed)
        ok = (k >= KEY_MIN) & (k <= KEY_MAX)
        idx = np.flatnonzero(ok)
        if idx.size >= n:
            last = int(idx[n - 1])
            return k[idx[:n]].astype(U32), counter0 + last + 1
        extra *= 4


def splitmix32(x) -> np.ndarray:
    """Golden-ratio increment followed by the MurmurHash3 fmix32 finalizer."""
    z = (np.asarray(x, dtype=np.uint64) + 0x9E3779B9) & MASK32
    z = ((z ^ (z >> 16)) * 0x85EBCA6B) & MASK32
    z = ((z ^ (z >> 13)) * 0xC2B2AE35) & MASK32
    z = z ^ (z >> 16)
    return z.astype(U32)


def values_for(keys, seed: int) -> np.ndarray:
    return splitmix32(np.asarray(keys, dtype=np.uint64) ^ (int(seed) & MASK32))


def permute_index(idx, n: int, seed: int) -> np.ndarray:
    """Seeded permutation of [0, n) by cycle-walking a Feistel bijection."""
    n = int(n)
    idx = np.asarray(idx, dtype=np.uint64)
    if n <= 1:
        return idx.copy()
    bits = max(2, int(n - 1).bit_length())
    bits += bits & 1
    y = feistel_bits(idx, seed, bits)
    bad = y >= n
    while bad.any():
        y[bad] = feistel_bits(y[bad], seed, bits)
        bad = y >= n
    return y


def zipf_ranks(rng: np.random.Generator, n_items: int, s: float, count: int) -> np.ndarray:
    """``count`` Zipf(s) ranks in [1, n_items] by rejection-inversion (s != 1)."""
    assert s > 0 and abs(s - 1.0) > 1e-9
    n_items = int(n_items)
    one_m_s = 1.0 - s

    def h(x):
        return np.exp(-s * np.log(x))

    def h_int(x):  # integral of t^-s from 1 to x, stable near s == 1
        lx = np.log(x)
        t = one_m_s * lx
        with np.errstate(divide="ignore", invalid="ignore"):
            f = np.where(np.abs(t) > 1e-8, np.expm1(t) / np.where(t == 0, 1, t), 1.0 + t / 2)
        return f * lx

    def h_int_inv(y):
        t = y * one_m_s
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(np.abs(t) > 1e-8, np.log1p(t) / np.where(t == 0, 1, t), 1.0 - t / 2)
        return np.exp(g * y)

    hx1 = float(h_int(np.float64(1.5))) - 1.0
    hn = float(h_int(np.float64(n_items + 0.5)))
    sq = 2.0 - float(h_int_inv(h_int(np.float64(2.5)) - h(np.float64(2.0))))
    out = np.empty(count, dtype=np.int64)
    todo = np.arange(count)
    while todo.size:
        u = hn + rng.random(todo.size) * (hx1 - hn)
        x = h_int_inv(u)
        k = np.clip(np.floor(x + 0.5), 1, n_items)
        acc = (k - x <= sq) | (u >= h_int(k + 0.5) - h(k))
        out[todo[acc]] = k[acc].astype(np.int64)
        todo = todo[~acc]
    return out


# ----------------------------------------------------------------------------
# Workload recipes (sizes follow the configurations the table is measured on)
# ----------------------------------------------------------------------------

def plain_phases(seed: int = 1, slots: int = 1 << 20, load_num: int = 4, load_den: int = 5):
    """Fixed table of ``slots`` slots: insert to load, find hits+absent,
    erase a seeded half, find again.  Defaults: 2^20 slots at 80% load, i.e.
    838,861 inserts (round to nearest), 838,861 absent finds, 419,430 erases.
    """
    n_ins = (slots * load_num * 2 + load_den) // (2 * load_den)
    keys, ctr = take_keys(seed, 0, n_ins)
    vals = values_for(keys, seed)
    absent, _ = take_keys(seed, ctr, n_ins)
    rng = np.random.default_rng(seed)
    find_keys = np.concatenate([keys, absent])
    find_keys = find_keys[rng.permutation(find_keys.size)]
    erase_keys = keys[rng.permutation(n_ins)[: n_ins // 2]]
    return {"insert_keys": keys, "insert_vals": vals, "find_keys": find_keys,
            "erase_keys": erase_keys, "absent_keys": absent}


def fill_and_query(seed: int, slots: int, load_num: int, load_den: int,
                   n_find: int, hit_num: int = 1, hit_den: int = 2,
                   zipf_s: float | None = None):
    """Load-factor sweep input: unique inserts to ``load`` of ``slots`` and
    ``n_find`` queries at the given hit rate (uniform or Zipf over ranks)."""
    n_ins = (slots * load_num * 2 + load_den) // (2 * load_den)
    keys, ctr = take_keys(seed, 0, n_ins)
    vals = values_for(keys, seed)
    rng = np.random.default_rng(seed ^ 0x5EED)
    is_hit = rng.random(n_find) < (hit_num / hit_den)
    n_hit = int(is_hit.sum())
    n_miss = n_find - n_hit
    n_absent_pool = max(n_miss, 1) if zipf_s is None else max(min(n_ins, n_miss), 1)
    absent, _ = take_keys(seed, ctr, n_absent_pool)
    if zipf_s is None:
        hit_idx = rng.integers(0, n_ins, n_hit)
        miss_keys = absent[:n_miss] if n_miss <= absent.size else absent[rng.integers(0, absent.size, n_miss)]
    else:
        r = zipf_ranks(rng, n_ins, zipf_s, n_hit) - 1
        hit_idx = permute_index(r, n_ins, seed ^ 0x21F).astype(np.int64)
        r2 = zipf_ranks(rng, absent.size, zipf_s, n_miss) - 1
        miss_keys = absent[permute_index(r2, absent.size, seed ^ 0x3A7).astype(np.int64)]
    q = np.empty(n_find, dtype=U32)
    q[is_hit] = keys[hit_idx]
    q[~is_hit] = miss_keys
    return {"insert_keys": keys, "insert_vals": vals, "find_keys": q, "is_hit": is_hit}


def mixed_batch(rng: np.random.Generator, live_keys: np.ndarray, new_keys: np.ndarray,
                n_ins: int, n_erase: int, n_find: int, seed: int,
                zipf_s: float | None = None):
    """One mixed batch: ``n_ins`` inserts of new keys, ``n_erase`` erases of
    distinct live keys, ``n_find`` finds over live keys not updated in this batch
    (uniform or Zipf).  Op order is a seeded shuffle.  Returns (ops, keys, vals)."""
    assert new_keys.size >= n_ins
    nl = live_keys.size
    perm = rng.permutation(nl)
    erase = live_keys[perm[:n_erase]]
    keep = live_keys[perm[n_erase:]]
    ins = new_keys[:n_ins]
    if n_find and keep.size:
        if zipf_s is None:
            fidx = rng.integers(0, keep.size, n_find)
        else:
            r = zipf_ranks(rng, keep.size, zipf_s, n_find) - 1
            fidx = permute_index(r, keep.size, seed ^ 0x77).astype(np.int64)
        finds = keep[fidx]
    else:
        finds = np.zeros(0, dtype=U32)
        n_find = 0
    ops = np.concatenate([np.full(n_ins, OP_INSERT, np.uint8), np.full(n_erase, OP_ERASE, np.uint8),
                          np.full(n_find, OP_FIND, np.uint8)])
    keys = np.concatenate([ins, erase, finds]).astype(U32)
    vals = np.concatenate([values_for(ins, seed), np.zeros(n_erase + n_find, U32)]).astype(U32)
    order = rng.permutation(ops.size)
    return ops[order], keys[order], vals[order]


# ----------------------------------------------------------------------------
# The same generators on torch tensors (CUDA or CPU), for large workloads that
# are generated where they are used.  Same seeds give the same keys as above.
# ----------------------------------------------------------------------------

def _mul32_t(x, c: int):
    """(x * c) mod 2^32 for int64 tensors holding values < 2^32, overflow-free."""
    lo = x & 0xFFFF
    hi = x >> 16
    return (lo * c + (((hi * c) & 0xFFFF) << 16)) & MASK32


def feistel_bits_t(x, seed: int, bits: int):
    assert bits % 2 == 0 and 2 <= bits <= 32
    half = bits // 2
    hm = (1 << half) - 1
    left = (x >> half) & hm
    right = x & hm
    for k in _round_keys(seed):
        f = (right ^ (k & hm)) & hm
        f = (_mul32_t(f, 0x2C1B3C6D) + (k >> 7)) & MASK32
        f = f ^ (f >> 15)
        f = _mul32_t(f, 0x297A2D39)
        f = f ^ (f >> 12)
        left, right = right, left ^ (f & hm)
    return (left << half) | right


def splitmix32_t(x):
    z = (x + 0x9E3779B9) & MASK32
    z = _mul32_t(z ^ (z >> 16), 0x85EBCA6B)
    z = _mul32_t(z ^ (z >> 13), 0xC2B2AE35)
    return z ^ (z >> 16)


def mixed_step_t(torch, seed: int, count: int, n_ops: int, device, ins_frac=(1, 2),
                 erase_frac=(1, 4), salt: int = 0, absent_base: int = 1 << 31):
    """One batch of mixed ops for a table whose inserted keys are the stream
    positions [0, count) of `seed`: n_ops * ins_frac inserts, n_ops * erase_frac
    erases, the rest finds.  Inserts take the next positions; erases and finds
    each take half live keys (distinct positions of a random permutation of
    [0, count), so no key is both updated and searched) and half absent keys
    (positions from absent_base up, never inserted; erases and finds use
    disjoint halves).  Returns (ops u8, keys i32, vals i32, new count, n_insert)
    as tensors on `device`."""
    g = torch.Generator(device=device)
    g.manual_seed((seed * 1000003 + count * 7919 + salt) & 0x7FFFFFFFFFFF)
    n_ins = n_ops * ins_frac[0] // ins_frac[1]
    n_er = n_ops * erase_frac[0] // erase_frac[1]
    n_fd = n_ops - n_ins - n_er
    er_live = min(n_er // 2, count)
    fd_live = min(n_fd // 2, count - er_live)
    i64 = torch.int64
    perm = (torch.randperm(count, generator=g, device=device)[: er_live + fd_live] if count
            else torch.zeros(0, dtype=i64, device=device))
    ins_pos = torch.arange(count, count + n_ins, device=device, dtype=i64)
    er_abs = n_er - er_live
    fd_abs = n_fd - fd_live
    quarter = 1 << 29
    # distinct absent positions: consecutive from a random start (the Feistel
    # bijection turns them into unrelated keys)
    start = int(torch.randint(0, quarter, (1,), generator=g, device=device).item())
    er_abs_pos = absent_base + (start + torch.arange(er_abs, device=device, dtype=i64)) % quarter
    fd_abs_pos = absent_base + quarter + torch.randint(0, quarter, (fd_abs,), generator=g,
                                                       device=device)
    pos = torch.cat([ins_pos, perm[:er_live], er_abs_pos, perm[er_live:], fd_abs_pos])
    ops = torch.cat([torch.full((n_ins,), OP_INSERT, dtype=torch.uint8, device=device),
                     torch.full((er_live + er_abs,), OP_ERASE, dtype=torch.uint8, device=device),
                     torch.full((fd_live + fd_abs,), OP_FIND, dtype=torch.uint8, device=device)])
    keys = feistel_bits_t(pos, seed, 32)
    vals = splitmix32_t(keys ^ (seed & MASK32))
    vals = torch.where(ops == OP_INSERT, vals, torch.zeros_like(vals))
    order = torch.randperm(ops.numel(), generator=g, device=device)
    to32 = lambda t: (t - ((t >> 31) << 32)).to(torch.int32)  # noqa: E731  two's complement view
    return ops[order], to32(keys[order]), to32(vals[order]), count + n_ins, n_ins


def multi_table_step(torch, seed: int, count: int, n_ops: int, device, salt: int = 0):
    """Mixed ops insert:find:erase = 2:1:1 (see mixed_step_t)."""
    return mixed_step_t(torch, seed, count, n_ops, device, (1, 2), (1, 4), salt)


def preload_t(torch, seed: int, n: int, device):
    """The first n stream positions of `seed` as (keys i32, vals i32) tensors."""
    pos = torch.arange(n, device=device, dtype=torch.int64)
    keys = feistel_bits_t(pos, seed, 32)
    vals = splitmix32_t(keys ^ (seed & MASK32))
    to32 = lambda t: (t - ((t >> 31) << 32)).to(torch.int32)  # noqa: E731
    return to32(keys), to32(vals)


def zipf_ranks_t(torch, n_items: int, s: float, count: int, generator, device):
    """Zipf(s) ranks in [1, n_items] on torch tensors (rejection-inversion,
    as zipf_ranks above)."""
    f64 = torch.float64
    one_m_s = 1.0 - s

    def h(x):
        return torch.exp(-s * torch.log(x))

    def h_int(x):
        lx = torch.log(x)
        t = one_m_s * lx
        safe = torch.where(t.abs() > 1e-8, t, torch.ones_like(t))
        f = torch.where(t.abs() > 1e-8, torch.expm1(t) / safe, 1.0 + t / 2)
        return f * lx

    def h_int_inv(y):
        t = y * one_m_s
        safe = torch.where(t.abs() > 1e-8, t, torch.ones_like(t))
        g = torch.where(t.abs() > 1e-8, torch.log1p(t) / safe, 1.0 - t / 2)
        return torch.exp(g * y)

    c = lambda v: torch.tensor(v, dtype=f64, device=device)  # noqa: E731
    hx1 = float(h_int(c(1.5))) - 1.0
    hn = float(h_int(c(n_items + 0.5)))
    sq = 2.0 - float(h_int_inv(h_int(c(2.5)) - h(c(2.0))))
    out = torch.empty(count, dtype=torch.int64, device=device)
    todo = torch.arange(count, device=device)
    while todo.numel():
        u = hn + torch.rand(todo.numel(), generator=generator, dtype=f64, device=device) * (hx1 - hn)
        x = h_int_inv(u)
        k = torch.clamp(torch.floor(x + 0.5), 1, n_items)
        acc = (k - x <= sq) | (u >= h_int(k + 0.5) - h(k))
        out[todo[acc]] = k[acc].to(torch.int64)
        todo = todo[~acc]
    return out


def stream_step_t(torch, seed: int, live_pos, counter: int, n_ops: int, device,
                  ins_frac=(2, 5), erase_frac=(1, 5), zipf_s: float | None = 0.99, salt: int = 0):
    """One batch of the resize stream: `live_pos` (int64 tensor) holds the
    stream positions of the live keys, `counter` the next unused position.
    Inserts take new positions; erases take distinct live keys; finds take live
    keys that this batch does not erase, Zipf(zipf_s)-distributed over a seeded
    permutation of the live set (uniform when zipf_s is None).  Returns (ops,
    keys, vals, new live_pos, new counter)."""
    g = torch.Generator(device=device)
    g.manual_seed((seed * 1000003 + counter * 7919 + salt) & 0x7FFFFFFFFFFF)
    nl = int(live_pos.numel())
    n_ins = n_ops * ins_frac[0] // ins_frac[1]
    n_er = min(n_ops * erase_frac[0] // erase_frac[1], nl)
    n_fd = n_ops - n_ins - n_er
    perm = torch.randperm(nl, generator=g, device=device)
    er_idx = perm[:n_er]
    keep = torch.ones(nl, dtype=torch.bool, device=device)
    keep[er_idx] = False
    kept = live_pos[keep]
    nk = int(kept.numel())
    if n_fd and nk:
        if zipf_s is None:
            fidx = torch.randint(0, nk, (n_fd,), generator=g, device=device)
        else:
            r = zipf_ranks_t(torch, nk, zipf_s, n_fd, g, device) - 1
            bits = max(2, int(nk - 1).bit_length())
            bits += bits & 1
            y = feistel_bits_t(r, seed ^ 0x5A5A, bits)
            bad = y >= nk
            while bool(bad.any()):
                y[bad] = feistel_bits_t(y[bad], seed ^ 0x5A5A, bits)
                bad = y >= nk
            fidx = y
        fd_pos = kept[fidx]
    else:
        n_fd = 0
        fd_pos = torch.zeros(0, dtype=torch.int64, device=device)
    ins_pos = torch.arange(counter, counter + n_ins, device=device, dtype=torch.int64)
    pos = torch.cat([ins_pos, live_pos[er_idx], fd_pos])
    ops = torch.cat([torch.full((n_ins,), OP_INSERT, dtype=torch.uint8, device=device),
                     torch.full((n_er,), OP_ERASE, dtype=torch.uint8, device=device),
                     torch.full((n_fd,), OP_FIND, dtype=torch.uint8, device=device)])
    keys = feistel_bits_t(pos, seed, 32)
    vals = splitmix32_t(keys ^ (seed & MASK32))
    vals = torch.where(ops == OP_INSERT, vals, torch.zeros_like(vals))
    order = torch.randperm(ops.numel(), generator=g, device=device)
    to32 = lambda t: (t - ((t >> 31) << 32)).to(torch.int32)  # noqa: E731
    new_live = torch.cat([kept, ins_pos])
    return ops[order], to32(keys[order]), to32(vals[order]), new_live, counter + n_ins
