"""Pins of the oracle's key mapping (Sec. 3.2, Algorithm 1; Sec. 3.4).

The hash is our reading of "a GPU-optimized hash derived from Murmur3": the
MurmurHash3 64-bit finaliser. It is pinned by its inverse (written from the
modular inverses of its multipliers, so a wrong constant or shift fails),
by avalanche, and by the uniformity of buckets and digests.
"""
import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1
C1 = 0xFF51AFD7ED558CCD
C2 = 0xC4CEB9FE1A85EC53


def unfmix(h: int) -> int:
    # x ^= x >> 33 is its own inverse for a shift >= 32; multiplications by odd
    # constants invert by the modular inverse.
    h ^= h >> 33
    h = (h * pow(C2, -1, 1 << 64)) & M64
    h ^= h >> 33
    h = (h * pow(C1, -1, 1 << 64)) & M64
    h ^= h >> 33
    return h


def test_fmix64_inverts_to_key():
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 63, size=2000, dtype=np.uint64)
    h = oracle.fmix64(keys)
    assert all(unfmix(int(x)) == int(k) for x, k in zip(h, keys))
    assert oracle.fmix64(np.array([0], np.uint64))[0] == 0


def test_fmix64_avalanche():
    rng = np.random.default_rng(12)
    keys = rng.integers(0, 1 << 63, size=600, dtype=np.uint64)
    base = oracle.fmix64(keys)
    flips = np.zeros((64, 64))
    for bit in range(64):
        h = oracle.fmix64(keys ^ np.uint64(1 << bit))
        d = base ^ h
        for ob in range(64):
            flips[bit, ob] = np.mean((d >> np.uint64(ob)) & np.uint64(1))
    assert flips.min() > 0.40 and flips.max() < 0.60


@pytest.mark.parametrize("nb", [1, 64, 1024, 1 << 16])
def test_bucket_and_digest_uniform(nb):
    from paper_2603_17168_gb300 import workloads as w
    rng = np.random.default_rng(13)
    # sequential Zipf ranks are the hardest case for a weak mixer
    keys = np.concatenate([w.rank_to_key(np.arange(1, 200001, dtype=np.uint64)),
                           w.uniform_keys(rng, 200000)])
    b1, b2, dg = oracle.map_keys(nb, True, keys)
    assert b1.max() < nb and b2.max() < nb
    if nb > 1:
        c = np.bincount(b1.astype(np.int64), minlength=nb)
        e = keys.size / nb
        chi2 = ((c - e) ** 2 / e).sum()
        dof = nb - 1
        assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof)
        # the second hash is independent of the first
        assert abs(np.mean(b1 == b2) - 1 / nb) < 6 * np.sqrt(1 / nb / keys.size) + 1e-9
    # digests live in 1..255; raw 0 folds onto 1 (0 marks empty slots)
    assert dg.min() >= 1
    c = np.bincount(dg, minlength=256).astype(float)
    p = np.full(256, 1 / 256)
    p[0] = 0
    p[1] = 2 / 256
    e = keys.size * p
    chi2 = ((c[1:] - e[1:]) ** 2 / e[1:]).sum()
    assert abs(chi2 - 254) < 6 * np.sqrt(2 * 254)


def test_digest_independent_of_bucket():
    # bits 32..39 are disjoint from the bucket bits while B <= 2^32: within
    # one bucket the digest is still uniform
    rng = np.random.default_rng(14)
    keys = rng.integers(1, 1 << 63, size=400000, dtype=np.uint64)
    b1, _, dg = oracle.map_keys(1 << 12, False, keys)
    sel = dg[b1 < 16]
    c = np.bincount(sel, minlength=256)[2:].astype(float)
    e = c.sum() / 254
    chi2 = ((c - e) ** 2 / e).sum()
    assert abs(chi2 - 253) < 6 * np.sqrt(2 * 253)
