"""Pins of the oracle's find_or_insert against its pinned insert_or_assign
and find: on twin tables, find_or_insert of a batch must leave exactly the
state that insert_or_assign leaves when the rows of keys already resident
are replaced by the values they hold (so that writing them changes
nothing), return those stored rows for every key resident afterwards, the
caller's rows for refused keys, and found = residency at batch start.
Checked for single and dual buckets, several policies and duplicate-heavy
batches that overflow the table."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w


@pytest.mark.parametrize("policy,dual", [(oracle.LRU, False), (oracle.LFU, True),
                                         (oracle.CUSTOM, False), (oracle.LFU, False)])
def test_find_or_insert_is_upsert_without_overwrite(policy, dual):
    rng = np.random.default_rng(4200 + policy * 2 + dual)
    nb, dim = 8, 3
    a = oracle.OracleTable(nb, dim, policy, dual)
    b = oracle.OracleTable(nb, dim, policy, dual)
    z = w.Zipf(1.1, 3000)
    for _ in range(8):
        keys = z.keys(rng, 700)
        vals = w.normal_values(rng, keys.size, dim)
        sc = rng.integers(0, 100, keys.size, dtype=np.uint64) if policy == oracle.CUSTOM else None
        # resident rows as they are now
        cur, was = b.find(keys, np.zeros((keys.size, dim), np.float32))[:2]
        rows, found = a.find_or_insert(keys, vals, sc)
        vb = np.where(was[:, None], cur, vals).astype(np.float32)
        b.insert_or_assign(keys, vb, sc)
        ka, sa, va, ba = a.export()
        kb, sb, vbb, bb = b.export()
        assert np.array_equal(ka, kb) and np.array_equal(sa, sb) and np.array_equal(ba, bb)
        assert np.array_equal(va.view(np.uint32), vbb.view(np.uint32))
        assert np.array_equal(found.astype(bool), was)
        now, res = b.find(keys, np.zeros((keys.size, dim), np.float32))[:2]
        want = np.where(res[:, None], now, vals)
        assert np.array_equal(rows.view(np.uint32), want.astype(np.float32).view(np.uint32))
    assert a.size() >= 0.95 * nb * 128  # the batches filled the table


def test_find_or_insert_on_resident_keys_only_touches_scores():
    rng = np.random.default_rng(4300)
    t = oracle.OracleTable(4, 2, oracle.LFU)
    keys = w.uniform_keys(rng, 300, distinct=True)
    vals = w.normal_values(rng, 300, 2)
    t.insert_or_assign(keys, vals)
    k0, s0, v0, b0 = t.export()
    rows, found = t.find_or_insert(keys[:100], w.normal_values(rng, 100, 2))
    k1, s1, v1, b1 = t.export()
    assert np.array_equal(k0, k1) and np.array_equal(v0.view(np.uint32), v1.view(np.uint32))
    assert found.all()
    assert np.array_equal(rows.view(np.uint32), vals[:100].view(np.uint32))
    j = np.searchsorted(k0, keys[:100])
    assert np.array_equal(s1[j], s0[j] + 1)  # one access each under LFU
