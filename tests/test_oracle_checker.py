"""Pins for the oracle's invariant checker: a valid table image built on the CPU
passes, and each planted corruption is reported under its own invariant."""
import numpy as np
import pytest

import oracle

S = 32
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _build_image(nb, n_keys, seed, stash_keys=0):
    """Place keys in the first free slot of their BitHash1 bucket, else their
    BitHash2 bucket, else the stash (sorted) -- a valid quiescent layout."""
    pow2 = 1
    while pow2 * 2 <= nb:
        pow2 *= 2
    M, p = pow2 - 1, nb - pow2
    rng = np.random.default_rng(seed)
    keys = rng.choice(0xFFFFFFFE, n_keys, replace=False).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, n_keys, dtype=np.uint64).astype(np.uint32)
    a1 = oracle.lh_address_many(oracle.bithash_many(1, keys), M, p)
    a2 = oracle.lh_address_many(oracle.bithash_many(2, keys), M, p)
    buckets = np.full(nb * S, EMPTY, dtype=np.uint64)
    fill = np.zeros(nb, np.int64)
    stash = []
    for k, v, b1, b2 in zip(keys.tolist(), vals.tolist(), a1.tolist(), a2.tolist()):
        w = (v << 32) | k
        for b in (b1, b2):
            if fill[b] < S:
                buckets[b * S + fill[b]] = w
                fill[b] += 1
                break
        else:
            stash.append(w)
    for _ in range(stash_keys):
        pass
    masks = np.zeros(nb, np.uint32)
    for b in range(nb):
        free = [i for i in range(S) if buckets[b * S + i] == EMPTY]
        masks[b] = sum(1 << i for i in free) & 0xFFFFFFFF
    stash = np.array(sorted(stash, key=lambda w: w & 0xFFFFFFFF), dtype=np.uint64)
    img = {"buckets": buckets, "masks": masks, "locks": np.zeros(nb, np.uint32), "nb": nb,
           "M": M, "p": p, "stash": stash, "stash_cap": max(64, stash.size), "size": n_keys,
           "pending": 0}
    d = oracle.Dict()
    d.insert(keys, vals)
    return img, d


@pytest.mark.parametrize("nb,n", [(8, 200), (11, 300), (5, 170)])
def test_valid_image_passes(nb, n):
    img, d = _build_image(nb, n, seed=nb)
    assert oracle.check_image(img, S, d) == (0, 0)


def _occupied(img):
    return np.flatnonzero(img["buckets"] != EMPTY)


def test_planted_mask_bit():
    img, d = _build_image(8, 200, 1)
    i = int(_occupied(img)[3])
    img["masks"][i // S] |= np.uint32(1 << (i % S))
    assert oracle.check_image(img, S, d)[0] == 1


def test_planted_wrong_bucket():
    img, d = _build_image(8, 100, 2)
    M, p = img["M"], img["p"]
    for i in _occupied(img):
        k = int(img["buckets"][i]) & 0xFFFFFFFF
        homes = {oracle.lh_address(oracle.bithash1(k), M, p), oracle.lh_address(oracle.bithash2(k), M, p)}
        other = next(b for b in range(img["nb"]) if b not in homes)
        j = int(np.flatnonzero(img["buckets"][other * S:(other + 1) * S] == EMPTY)[0]) + other * S
        img["buckets"][j] = img["buckets"][i]
        img["buckets"][i] = EMPTY
        img["masks"][i // S] |= np.uint32(1 << (i % S))
        img["masks"][j // S] &= np.uint32(~(1 << (j % S)) & 0xFFFFFFFF)
        break
    assert oracle.check_image(img, S, d)[0] == 2


def test_planted_duplicate():
    img, d = _build_image(8, 100, 3)
    M, p = img["M"], img["p"]
    for i in _occupied(img):
        k = int(img["buckets"][i]) & 0xFFFFFFFF
        b2 = oracle.lh_address(oracle.bithash2(k), M, p)
        b1 = oracle.lh_address(oracle.bithash1(k), M, p)
        if b1 == b2:
            continue
        j = int(np.flatnonzero(img["buckets"][b2 * S:(b2 + 1) * S] == EMPTY)[0]) + b2 * S
        img["buckets"][j] = img["buckets"][i]
        img["masks"][b2] &= np.uint32(~(1 << (j % S)) & 0xFFFFFFFF)
        img["size"] += 1
        break
    assert oracle.check_image(img, S, d)[0] == 3


def test_planted_size_and_value():
    img, d = _build_image(8, 100, 4)
    img["size"] += 1
    assert oracle.check_image(img, S, d)[0] == 4
    img["size"] -= 1
    i = int(_occupied(img)[0])
    img["buckets"][i] ^= np.uint64(1 << 40)  # flip a value bit
    assert oracle.check_image(img, S, d)[0] == 4
    assert oracle.check_image(img, S, None) == (0, 0)


def test_planted_lock_and_lh_fields():
    img, d = _build_image(8, 100, 5)
    img["locks"][2] = 1
    assert oracle.check_image(img, S, d)[0] == 5
    img["locks"][2] = 0
    img["pending"] = 1
    assert oracle.check_image(img, S, d)[0] == 5


def test_planted_stash_order():
    img, d = _build_image(2, 140, 6)  # 64 slots for 140 keys: stash holds the rest
    assert img["stash"].size >= 2
    assert oracle.check_image(img, S, d) == (0, 0)
    img["stash"] = img["stash"][::-1].copy()
    assert oracle.check_image(img, S, d)[0] == 6


def test_policy_thresholds():
    img, d = _build_image(8, 200, 7)  # 200 / 256 = 0.78
    pol = oracle.Policy(8, 1024)
    assert oracle.check_image(img, S, d, pol) == (0, 0)
    img2, d2 = _build_image(8, 240, 8)  # 0.9375 > 0.9
    assert oracle.check_image(img2, S, d2, pol)[0] == 7
    pol4 = oracle.Policy(4, 1024)  # nb=8 > nb_init=4 and 60/256 < 0.4
    img3, d3 = _build_image(8, 60, 9)
    assert oracle.check_image(img3, S, d3, pol4)[0] == 7
