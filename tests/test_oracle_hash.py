"""Pins for the oracle's BitHash1/BitHash2 (Section III-C, Listing 1) and for
Theorem 1's collision count.

Each published mixing step of Listing 1 is a bijection of 32-bit words; the
test below undoes the steps one by one, in reverse order, and checks that this
inverse recovers the input from the oracle's hash.  A wrong shift amount,
constant, operator or step order in the oracle's forward code breaks the round
trip.  Theorem 1's expected collision count is itself pinned against exact
enumeration on tiny cases, then used to check that both mixes spread keys like
uniform hashing once n is comparable to the number of buckets.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

M32 = (1 << 32) - 1


def _inv_xorshift_right(y, s, c=0):
    """Solve (x ^ c) ^ (x >> s) == y for x."""
    z = y ^ c  # x ^ (x >> s) = y ^ c
    x = z
    for _ in range(32 // s + 1):
        x = z ^ (x >> s)
    return x & M32


def _inv_affine(y, a, c):
    """Solve a*x + c == y (mod 2^32), a odd."""
    return ((y - c) * pow(a, -1, 1 << 32)) & M32


def _inv_add_xor_left(y, c, s):
    """Solve (x + c) ^ (x << s) == y (mod 2^32): the low bits fix upward."""
    x = 0
    for _ in range(32 // s + 1):
        x = ((y ^ (x << s)) - c) & M32
    return x


def inv_bithash1(y):
    # Listing 1, BitHash1 steps (before the reduction), undone last to first:
    #   key = ~key + (key << 15); key ^= key >> 12; key += key << 2;
    #   key ^= key >> 4;  key *= 2057;  key ^= key >> 16
    x = _inv_xorshift_right(y, 16)
    x = _inv_affine(x, 2057, 0)
    x = _inv_xorshift_right(x, 4)
    x = _inv_affine(x, 1 + (1 << 2), 0)
    x = _inv_xorshift_right(x, 12)
    # ~x + (x << 15) = (2^15 - 1) x - 1
    x = _inv_affine(x, (1 << 15) - 1, M32)
    return x


def inv_bithash2(y):
    # Listing 1, BitHash2 steps, undone last to first.
    x = _inv_xorshift_right(y, 16, 0xB55A4F09)
    x = _inv_affine(x, 1 + (1 << 3), 0xFD7046C5)
    x = _inv_add_xor_left(x, 0xD3A2646C, 9)
    x = _inv_affine(x, 1 + (1 << 5), 0x165667B1)
    x = _inv_xorshift_right(x, 19, 0xC761C23C)
    x = _inv_affine(x, 1 + (1 << 12), 0x7ED55D16)
    return x


SAMPLE = [0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFD, 0xFFFFFFFE, 0xFFFFFFFF, 0xDEADBEEF]


@pytest.mark.parametrize("which,inv", [(1, inv_bithash1), (2, inv_bithash2)])
def test_bithash_inverts_step_by_step(which, inv):
    rng = np.random.default_rng(which)
    xs = np.array(SAMPLE + rng.integers(0, 1 << 32, 20000, dtype=np.uint64).tolist(), np.uint32)
    hs = oracle.bithash_many(which, xs)
    for x, h in zip(xs.tolist(), hs.tolist()):
        assert inv(h) == x, (which, hex(x), hex(h))


def test_scalar_and_array_forms_agree():
    xs = ((np.arange(1000, dtype=np.uint64) * 2654435761) % (1 << 32)).astype(np.uint32)
    assert oracle.bithash_many(1, xs).tolist() == [oracle.bithash1(int(x)) for x in xs]
    assert oracle.bithash_many(2, xs).tolist() == [oracle.bithash2(int(x)) for x in xs]


def expected_collisions(n, m):
    """Theorem 1: E[Y] = n - m (1 - (1 - 1/m)^n)."""
    return n - m * (1.0 - (1.0 - 1.0 / m) ** n)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 2), (3, 2), (4, 3), (5, 3), (3, 4)])
def test_theorem1_by_enumeration(n, m):
    """Exact E[Y] over all m^n equally likely assignments."""
    tot = 0
    for a in itertools.product(range(m), repeat=n):
        loads = np.bincount(np.array(a), minlength=m)
        tot += int(np.maximum(loads - 1, 0).sum())
    assert math.isclose(tot / m ** n, expected_collisions(n, m), rel_tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("which", [1, 2])
@pytest.mark.parametrize("keys_kind", ["sequential", "random"])
def test_csr_near_one_at_unit_load(which, keys_kind):
    """CSR = E[Y]/Y_obs for m = 512^2 buckets and n = m keys is close to 1
    (the paper reports BitHash converging to uniform spread as n grows)."""
    m = 512 * 512
    n = m
    if keys_kind == "sequential":
        keys = np.arange(1, n + 1, dtype=np.uint32)
    else:
        keys = np.random.default_rng(5).choice(1 << 32, n, replace=False).astype(np.uint32)
    b = oracle.bithash_many(which, keys) % m
    y_obs = n - np.unique(b).size
    csr = expected_collisions(n, m) / y_obs
    assert 0.98 < csr < 1.02, csr


def test_checksum_catches_one_wrong_output():
    """The range checksum that the exhaustive GPU test compares: it equals
    its definition written over the array form of the mixes, and one changed
    output changes it."""
    k = np.arange(4096, 8192, dtype=np.uint64)
    h1 = oracle.bithash_many(1, k.astype(np.uint32)).astype(np.uint64)
    h2 = oracle.bithash_many(2, k.astype(np.uint32)).astype(np.uint64)
    acc = int(((h1 | (h2 << np.uint64(32))) * (2 * k + 1)).sum(dtype=np.uint64))
    assert acc == oracle.bithash_checksum(4096, 8192)
    h1[1000] ^= np.uint64(1 << 7)
    bad = int(((h1 | (h2 << np.uint64(32))) * (2 * k + 1)).sum(dtype=np.uint64))
    assert bad != acc
