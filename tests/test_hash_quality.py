"""Hash-quality study of Section III-C: the Collision Speedup Ratio
CSR = E[Y] / Y_observed (Theorem 1) of BitHash1 and BitHash2 for m = 512^2
buckets and n from 2^11 to 2048^2 keys.

The paper reports that BitHash clusters mildly at low load (CSR < 1) and
converges to uniform spread as n grows.  With consecutive keys, BitHash1
shows exactly that; both mixes are within 1% of uniform hashing once n is a
sizeable fraction of m, for consecutive and random keys alike.  (The figure's
values are not recoverable from the paper, so only these trends are checked.)
"""
import numpy as np
import pytest

import oracle

M = 512 * 512


def expected_collisions(n, m):
    return n - m * (1.0 - (1.0 - 1.0 / m) ** n)


def csr(which, keys):
    b = oracle.bithash_many(which, keys) % M
    return expected_collisions(keys.size, M) / max(keys.size - np.unique(b).size, 1)


def test_bithash1_clusters_mildly_at_low_load():
    for n in (1 << 11, 1 << 13, 1 << 15):
        c = csr(1, np.arange(1, n + 1, dtype=np.uint32))
        assert 0.8 < c < 1.0, (n, c)


@pytest.mark.parametrize("which", [1, 2])
@pytest.mark.parametrize("kind", ["consecutive", "random"])
def test_converges_to_uniform(which, kind):
    rng = np.random.default_rng(which)
    for n in (1 << 17, 1 << 19, 2048 * 2048):
        keys = (np.arange(1, n + 1, dtype=np.uint32) if kind == "consecutive"
                else rng.choice(1 << 32, n, replace=False).astype(np.uint32))
        c = csr(which, keys)
        assert abs(c - 1.0) < 0.01, (which, kind, n, c)
