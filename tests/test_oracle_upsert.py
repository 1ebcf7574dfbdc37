"""Pins of the oracle's insert_or_assign / assign / erase (Algorithm 2,
Sec. 3.3; Table 9 (admission burst, Exp. 3d); the batch semantics stated in oracle/hkv_oracle.c)."""
import heapq

import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w
from tests import invariants as inv


def state(t):
    k, s, v, b = t.export()
    return k, s, v.view(np.uint32), b


def same_state(a, b):
    return all(np.array_equal(x, y) for x, y in zip(state(a), state(b)))


def key_status(keys, status):
    d = {}
    for k, st in zip(keys.tolist(), status.tolist()):
        assert d.setdefault(k, st) == st, "occurrences of one key disagree"
    return d


def random_batches(rng, n_batches, batch, universe, dim, policy):
    out = []
    for _ in range(n_batches):
        k = w.uniform_keys(rng, batch, universe=universe)          # with duplicates
        v = w.normal_values(rng, batch, dim)
        s = rng.integers(0, 50, batch, dtype=np.uint64) if policy == oracle.CUSTOM else None
        out.append((k, v, s))
    return out


@pytest.mark.parametrize("policy", [oracle.LRU, oracle.LFU, oracle.CUSTOM, oracle.EPOCH_LFU,
                                    oracle.CUSTOM_TS_FREQ])
@pytest.mark.parametrize("nb", [1, 2, 4, 16])
def test_literal_loop_equals_topk_closed_form(policy, nb):
    """Streaming Algorithm 2 over the batch == per-bucket top-S by (score, key)."""
    rng = np.random.default_rng(100 + nb * 7 + policy)
    dim = 3
    a = oracle.OracleTable(nb, dim, policy)
    b = oracle.OracleTable(nb, dim, policy)
    for e, (k, v, s) in enumerate(random_batches(rng, 12, nb * 90, nb * 400, dim, policy)):
        a.set_epoch(e)
        b.set_epoch(e)
        sa, eka, esa, eva = a.insert_or_assign(k, v, s)
        sb, ekb, esb, evb = b.insert_or_assign_topk(k, v, s)
        assert np.array_equal(sa, sb)
        oa, ob = np.argsort(eka), np.argsort(ekb)
        assert np.array_equal(eka[oa], ekb[ob]) and np.array_equal(esa[oa], esb[ob])
        assert np.array_equal(eva[oa].view(np.uint32), evb[ob].view(np.uint32))
        assert same_state(a, b)


@pytest.mark.parametrize("nb", [1, 2, 4])
def test_single_bucket_result_is_order_independent(nb):
    rng = np.random.default_rng(200 + nb)
    dim = 2
    base = w.uniform_keys(rng, nb * 150, distinct=True)
    batch = w.uniform_keys(rng, min(600, nb * 200), distinct=True)
    vals = w.normal_values(rng, batch.size, dim)
    sc = rng.integers(0, 40, batch.size, dtype=np.uint64)
    ref = None
    for p in range(12):
        t = oracle.OracleTable(nb, dim, oracle.CUSTOM)
        t.insert_or_assign(base, np.zeros((base.size, dim), np.float32),
                           rng.integers(0, 40, base.size, dtype=np.uint64) * 0 + np.uint64(20))
        perm = np.random.default_rng(p).permutation(batch.size)
        st, ek, es, _ = t.insert_or_assign(batch[perm], vals[perm], sc[perm])
        got = (state(t), key_status(batch[perm], st), sorted(ek.tolist()))
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(x, y) for x, y in zip(got[0], ref[0]))
            assert got[1] == ref[1] and got[2] == ref[2]


def test_one_bucket_is_a_top_k_cache():
    # B = 1 with distinct custom scores: the table is the 128 largest
    # (score, key) pairs ever offered, a textbook top-k.
    rng = np.random.default_rng(301)
    t = oracle.OracleTable(1, 1, oracle.CUSTOM)
    keys = w.uniform_keys(rng, 3000, distinct=True)
    scores = rng.integers(0, 1000, keys.size, dtype=np.uint64)
    for lo in range(0, keys.size, 250):
        t.insert_or_assign(keys[lo:lo + 250], np.zeros((250, 1), np.float32), scores[lo:lo + 250])
    want = heapq.nlargest(128, zip(scores.tolist(), keys.tolist()))
    k, s, _, _ = t.export()
    assert sorted(zip(s.tolist(), k.tolist())) == sorted(want)


def test_last_write_wins_and_lfu_multiplicity():
    t = oracle.OracleTable(8, 2, oracle.LFU)
    k = np.array([5, 7, 5, 5, 9, 7], np.uint64)
    v = np.arange(12, dtype=np.float32).reshape(6, 2)
    st, ek, _, _ = t.insert_or_assign(k, v)
    assert st.tolist() == [oracle.ST_INSERTED] * 6 and ek.size == 0
    vals, found, scores = t.find(np.array([5, 7, 9], np.uint64))
    assert found.all()
    assert vals.tolist() == [[6, 7], [10, 11], [8, 9]]
    assert scores.tolist() == [3, 2, 1]
    st, _, _, _ = t.insert_or_assign(np.array([5, 5, 11], np.uint64), np.ones((3, 2), np.float32))
    assert st.tolist() == [oracle.ST_UPDATED, oracle.ST_UPDATED, oracle.ST_INSERTED]
    _, _, scores = t.find(np.array([5, 11], np.uint64))
    assert scores.tolist() == [5, 1]


def full_table(nb, rng, dim=1, lo=2, hi=10**8):
    """A table with every bucket full, custom scores in [lo, hi]."""
    t = oracle.OracleTable(nb, dim, oracle.CUSTOM)
    keys = w.uniform_keys(rng, nb * 128 * 3, distinct=True)
    b1, _, _ = oracle.map_keys(nb, False, keys)
    sel = np.concatenate([np.flatnonzero(b1 == b)[:128] for b in range(nb)])
    assert sel.size == nb * 128
    t.insert_or_assign(keys[sel], np.zeros((sel.size, dim), np.float32),
                       rng.integers(lo, hi, sel.size, dtype=np.uint64))
    assert t.size() == nb * 128
    return t


def test_admission_burst_table9():
    # Table 9 (Exp. 3d): a low-score burst is fully rejected and leaves the table as it
    # was; a high-score burst is fully admitted, each key displacing an
    # original. Scaled to a full 2^17-slot table (the paper's 16M slots at
    # lambda = 0.96 still has free slots, which admit regardless of score).
    rng = np.random.default_rng(401)
    nb = 1 << 10
    t = full_table(nb, rng)
    before = state(t)
    burst = w.uniform_keys(rng, 32768, distinct=True)
    zeros = np.zeros((burst.size, 1), np.float32)
    st, ek, _, _ = t.insert_or_assign(burst, zeros, np.full(burst.size, 1, np.uint64))
    assert np.all(st == oracle.ST_REJECTED) and ek.size == 0
    assert all(np.array_equal(x, y) for x, y in zip(before, state(t)))
    st, ek, es, _ = t.insert_or_assign(burst, zeros, np.full(burst.size, 10**9, np.uint64))
    assert np.all(st == oracle.ST_INSERTED)
    assert ek.size == burst.size and np.all(es < 10**9)
    assert t.contains(burst).all() and t.size() == nb * 128


@pytest.mark.parametrize("dual", [False, True])
def test_invariants_hold_after_every_batch(dual):
    rng = np.random.default_rng(501 + dual)
    nb, dim = 64, 2
    t = oracle.OracleTable(nb, dim, oracle.CUSTOM, dual)
    last = {}
    for step in range(30):
        k = w.uniform_keys(rng, 1500, universe=40000)
        v = w.normal_values(rng, k.size, dim)
        s = rng.integers(0, 1000, k.size, dtype=np.uint64)
        st, ek, es, ev = t.insert_or_assign(k, v, s)
        ks, ss, vs, bs = t.export()
        b1, b2, _ = oracle.map_keys(nb, dual, ks)
        inv.check_state(ks, ss, bs, nb, b1, b2, t.capacity)
        # the (score, key) of each rejected key: its last occurrence's score
        lastpos = {kk: i for i, kk in enumerate(k.tolist())}
        rej = np.array(sorted({kk for kk, x in zip(k.tolist(), st.tolist()) if x == oracle.ST_REJECTED}),
                       np.uint64)
        rs = np.array([s[lastpos[int(x)]] for x in rej], np.uint64)
        rb1, rb2, _ = oracle.map_keys(nb, dual, rej)
        eb1, eb2, _ = oracle.map_keys(nb, dual, ek)
        inv.check_admission(ks, ss, bs, nb, rej, rs, rb1, rb2, ek, es, eb1, eb2)
        # every hit returns the last value written
        for kk, i in lastpos.items():
            if st[i] != oracle.ST_REJECTED:
                last[kk] = v[i].tobytes()
        for kk in ek.tolist():
            last.pop(kk, None)
        for kk in rej.tolist():
            last.pop(kk, None)
        q = np.array(list(last.keys()), np.uint64)
        vals, found, _ = t.find(q)
        assert found.all()
        assert all(vals[j].tobytes() == last[int(q[j])] for j in range(q.size))
        assert len(last) == t.size()


def test_deterministic_mode_and_reserved_keys():
    t = oracle.OracleTable(4, 1, oracle.LRU)
    with pytest.raises(oracle.OracleError) as e:
        t.insert_or_assign(np.array([3, 4, 3], np.uint64), np.zeros((3, 1)), deterministic=True)
    assert e.value.code == oracle.ERR_DUPLICATE_KEY
    with pytest.raises(oracle.OracleError) as e:
        t.insert_or_assign(np.array([3, 2**63], np.uint64), np.zeros((2, 1)))
    assert e.value.code == oracle.ERR_RESERVED_KEY
    assert t.size() == 0 and t.step == 0
    st, _, _, _ = t.insert_or_assign(np.array([], np.uint64), np.zeros((0, 1)))
    assert st.size == 0 and t.step == 0


def test_erase_then_reinsert_and_assign():
    rng = np.random.default_rng(601)
    t = oracle.OracleTable(8, 2, oracle.LFU)
    k = w.uniform_keys(rng, 500, distinct=True)
    t.insert_or_assign(k, w.normal_values(rng, 500, 2))
    t.erase(np.concatenate([k[:100], k[:10]]))
    assert t.size() == 400 and not t.contains(k[:100]).any() and t.contains(k[100:]).all()
    st, _, _, _ = t.insert_or_assign(k[:50], np.ones((50, 2), np.float32))
    assert np.all(st == oracle.ST_INSERTED)
    _, _, sc = t.find(k[:50])
    assert np.all(sc == 1)
    # assign ignores missing keys and never changes the structure
    before = t.size()
    t.assign(np.concatenate([k[50:100], k[200:210], k[200:210]]), np.full((70, 2), 7, np.float32))
    assert t.size() == before
    vals, found, sc = t.find(k[200:210])
    assert found.all() and np.all(vals == 7) and np.all(sc == 3)
    assert not t.contains(k[50:100]).any()


def test_export_load_round_trip():
    rng = np.random.default_rng(701)
    for dual in (False, True):
        a = oracle.OracleTable(32, 3, oracle.LFU, dual)
        for _ in range(6):
            kk = w.uniform_keys(rng, 3000, universe=20000)
            a.insert_or_assign(kk, w.normal_values(rng, kk.size, 3))
        k, s, v, b = a.export()
        c = oracle.OracleTable(32, 3, oracle.LFU, dual)
        c.load(k, s, v, b)
        assert same_state(a, c)
        with pytest.raises(oracle.OracleError):
            c.load(k[:1], s[:1], v[:1], b[:1])          # duplicate key
