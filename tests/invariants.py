"""Table invariants shared by the oracle tests and the GPU parity tests.

A table state is given as arrays of its entries (keys, scores, buckets); the
candidate buckets of a key come from the oracle's own key mapping, passed in
as (b1, b2) arrays so this module does no hashing itself.
"""
from __future__ import annotations

import numpy as np

SLOTS = 128


def sk_min_per_bucket(keys, scores, buckets, num_buckets):
    """(min score, key at that min) per bucket in (score, key) order; buckets
    with no entries get (2^64-1, 2^64-1)."""
    big = np.iinfo(np.uint64).max
    ms = np.full(num_buckets, big, np.uint64)
    mk = np.full(num_buckets, big, np.uint64)
    o = np.lexsort((keys, scores))           # ascending (score, key)
    b = buckets[o].astype(np.int64)
    first = np.unique(b, return_index=True)[1]
    ms[b[first]] = scores[o][first]
    mk[b[first]] = keys[o][first]
    return ms, mk


def sk_less(s1, k1, s2, k2):
    s1, k1, s2, k2 = (np.asarray(x, np.uint64) for x in (s1, k1, s2, k2))
    return (s1 < s2) | ((s1 == s2) & (k1 < k2))


def check_state(keys, scores, buckets, num_buckets, b1, b2, capacity=None):
    """Structural invariants: unique keys, each in one of its candidate
    buckets, at most 128 entries per bucket, size <= capacity."""
    keys = np.asarray(keys, np.uint64)
    buckets = np.asarray(buckets, np.uint64)
    assert np.unique(keys).size == keys.size, "duplicate keys in table"
    assert np.all((buckets == b1) | (buckets == b2)), "entry outside its candidate buckets"
    counts = np.bincount(buckets.astype(np.int64), minlength=num_buckets)
    assert counts.max(initial=0) <= SLOTS, "bucket over capacity"
    if capacity is not None:
        assert keys.size <= capacity
    return counts


def check_admission(keys, scores, buckets, num_buckets, rej_keys, rej_scores, rej_b1, rej_b2,
                    ev_keys, ev_scores, ev_b1, ev_b2):
    """At the end of a batch, every key that is not resident because of it
    (rejected by admission, displaced by a later key of the same batch, or an
    evicted resident) is below the (score, key) minimum of at least one of its
    candidate buckets, and that bucket is full. For a single-bucket table that
    is its one bucket; for a dual table a refused key is below both, but a key
    that entered one bucket by load (phase D1) and was displaced there is only
    below that bucket's minimum."""
    counts = np.bincount(np.asarray(buckets, np.int64), minlength=num_buckets)
    ms, mk = sk_min_per_bucket(np.asarray(keys, np.uint64), np.asarray(scores, np.uint64),
                               np.asarray(buckets, np.uint64), num_buckets)
    for k, s, b1, b2, what in ((rej_keys, rej_scores, rej_b1, rej_b2, "rejected"),
                               (ev_keys, ev_scores, ev_b1, ev_b2, "evicted")):
        b1, b2 = np.asarray(b1, np.int64), np.asarray(b2, np.int64)
        ok1 = (counts[b1] == SLOTS) & sk_less(s, k, ms[b1], mk[b1])
        ok2 = (counts[b2] == SLOTS) & sk_less(s, k, ms[b2], mk[b2])
        assert np.all(ok1 | ok2), f"{what} key not below a full candidate bucket's minimum"
