"""Pins for the oracle's linear-hashing address and resize policy
(Section IV-C of the paper; Litwin's linear hashing).

The address is checked against the textbook closed forms: with no split
pending it is h mod 2^m; it always lies in [0, 2^m + p); splitting bucket p
moves only that bucket's keys, to p or p + 2^m; and over a full residue range
each split bucket receives exactly half the keys of an unsplit one.  The policy
model is checked against an independent one-bucket-at-a-time simulation and for
the threshold properties it promises.
"""
import numpy as np
import pytest

import oracle


def _states():
    yield 0, 0
    for m in range(1, 9):
        M = (1 << m) - 1
        for p in sorted({0, 1, M // 2, M}):
            yield M, p


@pytest.mark.parametrize("M,p", list(_states()))
def test_address_closed_forms(M, p):
    span = 1 << 14
    h = np.arange(span, dtype=np.uint32)
    a = oracle.lh_address_many(h, M, p)
    nb = M + 1 + p
    assert a.max() < nb
    if p == 0:
        assert np.array_equal(a, h % (M + 1))
    counts = np.bincount(a, minlength=nb)
    full = span // (M + 1)
    for b in range(nb):
        split = b < p or b > M
        assert counts[b] == (full // 2 if split else full), (b, counts[b])


@pytest.mark.parametrize("M,p", [(M, p) for M, p in _states() if p <= M])
def test_split_moves_only_bucket_p(M, p):
    rng = np.random.default_rng(M * 131 + p)
    h = rng.integers(0, 1 << 32, 50000, dtype=np.uint64).astype(np.uint32)
    before = oracle.lh_address_many(h, M, p)
    M2, p2 = (M, p + 1) if p + 1 <= M else (2 * M + 1, 0)
    after = oracle.lh_address_many(h, M2, p2)
    moved = before != after
    assert np.all(before[moved] == p)
    assert np.all(after[moved] == p + M + 1)
    stay = before == p
    assert np.all(np.isin(after[stay], [p, p + M + 1]))


def _lattice(nb_init, K, nb_max):
    """Independent simulation: add buckets one at a time (nb = 2^m + p), and
    record the capacity after each launch of at most K splits that never
    crosses a round boundary."""
    out = [nb_init]
    pow2 = 1
    while pow2 * 2 <= nb_init:
        pow2 *= 2
    nb = nb_init
    while nb < nb_max:
        # buckets left in this round: round ends at nb == 2 * pow2
        room = 2 * pow2 - nb
        step = min(K, room, nb_max - nb)
        nb += step
        if nb == 2 * pow2:
            pow2 *= 2
        out.append(nb)
    return out


@pytest.mark.parametrize("nb_init,K", [(1, 1), (3, 2), (32, 8), (1000, 64), (1 << 10, 256)])
def test_grow_matches_lattice_and_threshold(nb_init, K):
    S = 32
    nb_max = nb_init * 64
    lat = _lattice(nb_init, K, nb_max)
    rng = np.random.default_rng(nb_init)
    size = 0
    pol = oracle.Policy(nb_init, nb_max, S=S, K=K)
    for _ in range(40):
        n_ins = int(rng.integers(0, nb_init * S // 2 + 2))
        pol.grow(size, n_ins)
        nb, M, p = pol.state
        assert nb == M + 1 + p and p <= M
        # smallest lattice capacity meeting 10*(size+n) <= 9*S*nb
        want = next((c for c in lat if 10 * (size + n_ins) <= 9 * S * c), nb_max)
        want = max(want, lat[0])
        # growth never shrinks: the model keeps the larger of current and needed
        assert nb == max(want, nb) and nb in lat
        if nb < nb_max:
            assert 10 * (size + n_ins) <= 9 * S * nb
        size += n_ins // 2


@pytest.mark.parametrize("nb_init,K", [(4, 2), (32, 8), (1000, 64)])
def test_split_merge_are_inverse(nb_init, K):
    pol = oracle.Policy(nb_init, nb_init * 100, K=K)
    states = [pol.state]
    for _ in range(60):
        pol.split_step()
        states.append(pol.state)
    for i in range(60):
        pol.merge_step()
        assert pol.state == states[-2 - i]


@pytest.mark.parametrize("seed", range(5))
def test_shrink_properties(seed):
    rng = np.random.default_rng(seed)
    S, K, nb_init = 32, 16, 64
    pol = oracle.Policy(nb_init, 1 << 20, S=S, K=K)
    size = 0
    for _ in range(50):
        if rng.random() < 0.5:
            n = int(rng.integers(0, 20000))
            pol.grow(size, n)
            size += n
        else:
            size = int(size * rng.random())
        pol.shrink(size)
        nb, M, p = pol.state
        assert nb == M + 1 + p
        assert 10 * size <= 9 * S * nb or nb == (1 << 20)
        assert nb == nb_init or 5 * size >= 2 * S * nb
