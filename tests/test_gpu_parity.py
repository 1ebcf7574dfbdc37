"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bars: single-bucket upsert and every find are bit-exact (table state as a
sorted (key, score, value, bucket) multiset, statuses, evicted sets, hit
masks, values and scores; values are stored, never computed, so no
tolerance applies). Dual-bucket upsert is order-dependent under concurrency
(phase D1 reads live occupancy): it must pass every invariant, keep the
retained-key count within 0.1% of the oracle's, and find on its state must
match the oracle loaded with that state bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w
from tests import invariants as inv

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import NAN_BITS, dev, export_state, host, nan_filled, same_state  # noqa: E402


def gpu_upsert(t, keys, vals, scores=None, want_values=True):
    n = keys.size
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    ek = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    es = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    ev = torch.empty((max(n, 1), t.dim), dtype=torch.float32, device="cuda") if want_values else None
    ne = torch.zeros(1, dtype=torch.int64, device="cuda")
    t.insert_or_assign(dev(keys), dev(vals.reshape(n, t.dim)),
                       None if scores is None else dev(scores), st, ek, es, ev, ne)
    t.sync()
    m = int(ne.item())
    o = np.argsort(host(ek[:m]), kind="stable")
    evv = host(ev[:m])[o] if want_values else None
    return host(st), host(ek[:m])[o], host(es[:m])[o], evv


def sorted_evicted(ek, es, ev):
    o = np.argsort(ek, kind="stable")
    return ek[o], es[o], ev[o]


def compare_upsert(t, o, keys, vals, scores=None, deterministic=False):
    ost, oek, oes, oev = o.insert_or_assign(keys, vals, scores, deterministic=deterministic)
    gst, gek, ges, gev = gpu_upsert(t, keys, vals, scores)
    assert np.array_equal(gst, ost), "statuses differ"
    oek, oes, oev = sorted_evicted(oek, oes, oev)
    assert np.array_equal(gek, oek) and np.array_equal(ges, oes), "evicted sets differ"
    assert np.array_equal(gev.view(np.uint32), oev.view(np.uint32)), "evicted values differ"
    return gst


def compare_find(t, o, q):
    n = q.size
    out = nan_filled(n, t.dim)
    found = torch.empty(n, dtype=torch.uint8, device="cuda")
    sc = torch.zeros(n, dtype=torch.int64, device="cuda")
    t.find(dev(q), out, found, sc)
    torch.cuda.synchronize()
    ov = np.zeros((n, t.dim), np.uint32)
    ov[:] = NAN_BITS
    ov = ov.view(np.float32)
    ov, of, os_ = o.find(q, ov)
    gf = host(found).astype(bool)
    assert np.array_equal(gf, of), "hit masks differ"
    assert np.array_equal(host(out).view(np.uint32), ov.view(np.uint32)), "values differ"
    assert np.array_equal(host(sc)[gf], os_[of]), "scores differ"
    assert np.array_equal(host(t.contains(dev(q))).astype(bool), of), "contains differs"
    return gf


def test_tiny_config_bit_exact():
    """512 buckets x 128 slots, dim 8, LRU (score = step), deterministic,
    16 batches of 4,096 distinct uniform keys (evictions from lambda ~ 0.7),
    then 4,096 finds with exactly 50% hits."""
    cfg = w.TINY
    rng = np.random.default_rng(w.seed_for(1))
    nb, dim = cfg["num_buckets"], cfg["dim"]
    t = hkv.Table(nb * 128, dim, hkv.LRU, dual_bucket=False, deterministic=True)
    o = oracle.OracleTable(nb, dim, oracle.LRU)
    for _ in range(cfg["batches"]):
        keys = w.uniform_keys(rng, cfg["batch"], distinct=True)
        vals = w.normal_values(rng, keys.size, dim)
        compare_upsert(t, o, keys, vals, deterministic=True)
        same_state(export_state(t), o.export())
        assert t.size() == o.size()
    assert t.get_step() == o.step == 16
    assert o.size() > 0.95 * nb * 128
    resident = o.export()[0]
    q = np.concatenate([rng.choice(resident, cfg["finds"] // 2, replace=False),
                        w.uniform_keys(rng, cfg["finds"] // 2)])
    rng.shuffle(q)
    hits = compare_find(t, o, q)
    assert hits.sum() == cfg["finds"] // 2


@pytest.mark.parametrize("policy,dim", [(hkv.LFU, 16), (hkv.CUSTOM, 3), (hkv.CUSTOM_TS_FREQ, 4),
                                        (hkv.EPOCH_LRU, 1), (hkv.EPOCH_LFU, 7), (hkv.LRU, 32)])
def test_single_bucket_duplicates_bit_exact(policy, dim):
    """Zipf batches full of duplicates, sizes spanning several dedup tiles
    with ragged tails, plus the degenerate sizes 0 and 1."""
    rng = np.random.default_rng(1000 + policy * 10 + dim)
    nb = 64
    t = hkv.Table(nb * 128, dim, policy)
    o = oracle.OracleTable(nb, dim, policy)
    z = w.Zipf(1.05, 30000)
    for e, n in enumerate([5000, 1, 0, 2048, 7001, 3, 12000, 4096]):
        t.set_epoch(e)
        o.set_epoch(e)
        keys = z.keys(rng, n)
        vals = w.normal_values(rng, n, dim)
        sc = rng.integers(0, 60, n, dtype=np.uint64) if policy == hkv.CUSTOM else None
        compare_upsert(t, o, keys, vals, sc)
        same_state(export_state(t), o.export())
    q = np.concatenate([z.keys(rng, 3000), w.uniform_keys(rng, 1000)])
    compare_find(t, o, q)


def test_one_bucket_and_large_batch():
    rng = np.random.default_rng(1100)
    t = hkv.Table(1, 2, hkv.CUSTOM)               # rounds up to one bucket
    assert t.capacity == 128 and t.num_buckets == 1
    o = oracle.OracleTable(1, 2, oracle.CUSTOM)
    for _ in range(5):
        keys = w.uniform_keys(rng, 700, distinct=True)
        compare_upsert(t, o, keys, w.normal_values(rng, 700, 2),
                       rng.integers(0, 10**6, 700, dtype=np.uint64))
        same_state(export_state(t), o.export())
    # a batch four times the capacity of a 2^20-slot table
    nb = 1 << 13
    t2 = hkv.Table(nb * 128, 4, hkv.LRU)
    o2 = oracle.OracleTable(nb, 4, oracle.LRU)
    keys = w.uniform_keys(rng, 1 << 22)
    compare_upsert(t2, o2, keys, w.normal_values(rng, keys.size, 4))
    same_state(export_state(t2), o2.export())


def test_assign_erase_and_reinsert_bit_exact():
    rng = np.random.default_rng(1200)
    nb, dim = 32, 8
    for policy in (hkv.LFU, hkv.CUSTOM, hkv.LRU):
        t = hkv.Table(nb * 128, dim, policy)
        o = oracle.OracleTable(nb, dim, policy)
        keys = w.uniform_keys(rng, 3000, distinct=True)
        sc = rng.integers(0, 100, keys.size, dtype=np.uint64)
        compare_upsert(t, o, keys, w.normal_values(rng, keys.size, dim), sc)
        a = np.concatenate([keys[:500], keys[:100], w.uniform_keys(rng, 200)])
        av = w.normal_values(rng, a.size, dim)
        asc = rng.integers(0, 100, a.size, dtype=np.uint64)
        t.assign(dev(a), dev(av), dev(asc))
        o.assign(a, av, asc if policy == hkv.CUSTOM else None)
        t.assign(dev(keys[500:600]), None, dev(asc[:100]))      # scores only
        o.assign(keys[500:600], _current_values(o, keys[500:600]),
                 asc[:100] if policy == hkv.CUSTOM else None)
        same_state(export_state(t), o.export())
        er = np.concatenate([keys[1000:1400], keys[1000:1010], w.uniform_keys(rng, 50)])
        t.erase(dev(er))
        o.erase(er)
        same_state(export_state(t), o.export())
        compare_upsert(t, o, keys[1000:1200], w.normal_values(rng, 200, dim), sc[:200])
        same_state(export_state(t), o.export())
        compare_find(t, o, np.concatenate([keys, er]))


def _current_values(o, keys):
    v, f, _ = o.find(keys)
    return v


@pytest.mark.parametrize("det", [True, False])
def test_dual_bucket_erase_and_reinsert(det):
    """Erase on dual-bucket tables (Sec. 3.5, erase is an inserter) of keys
    that sit in their second bucket as well as their first, then fresh keys
    past lambda = 1, so that phase D1 of Algorithm 3 reads the occupancy the
    erase lowered. Deterministic mode: statuses, evicted sets and the full
    state including buckets equal the oracle's bit for bit after every call.
    Concurrent mode: every invariant after every batch, exactly the resident
    erased keys gone, the retained count within 0.1% of the oracle's, and
    find on the GPU's state equal to the oracle loaded with it."""
    rng = np.random.default_rng(9600 + det)
    nb, dim = 1 << 10, 8
    cap = nb * 128
    t = hkv.Table(cap, dim, hkv.LFU, dual_bucket=True, deterministic=det)
    o = oracle.OracleTable(nb, dim, oracle.LFU, True)

    def upsert(keys):
        vals = w.normal_values(rng, keys.size, dim)
        if det:
            compare_upsert(t, o, keys, vals, deterministic=True)
            same_state(export_state(t), o.export())
        else:
            gst, gek, ges, _ = gpu_upsert(t, keys, vals)
            o.insert_or_assign(keys, vals)
            _check_batch_invariants(t, nb, keys, gst, gek, ges)

    fill = w.uniform_keys(rng, int(0.985 * cap), distinct=True)
    for chunk in np.array_split(fill, 5):
        upsert(chunk)
    gk, gs, gv, gb = export_state(t)
    b1, b2, _ = oracle.map_keys(nb, True, gk)
    second = gk[(gb == b2) & (b2 != b1)]
    first = gk[gb == b1]
    assert second.size > 500, second.size
    er = np.concatenate([rng.choice(second, second.size // 2, replace=False),
                         rng.choice(first, 3000, replace=False), w.uniform_keys(rng, 64)])
    rng.shuffle(er)
    before = gk.size
    t.erase(dev(er))
    o.erase(er)
    t.sync()
    gk2 = export_state(t)[0]
    assert not np.any(np.isin(er, gk2)), "an erased key is still resident"
    assert gk2.size == before - int(np.isin(er, gk).sum())
    assert t.size() == gk2.size
    if det:
        same_state(export_state(t), o.export())
    for _ in range(4):
        upsert(w.uniform_keys(rng, cap // 6, distinct=True))
    assert o.size() == cap
    gs_, os_ = t.size(), o.size()
    assert abs(gs_ - os_) <= 0.001 * os_, (gs_, os_)
    q = np.concatenate([o.export()[0][:4000], er[:2000], w.uniform_keys(rng, 2000)])
    if det:
        compare_find(t, o, q)
    else:
        gk, gs, gv, gb = export_state(t)
        ref = oracle.OracleTable(nb, dim, oracle.LFU, True)
        ref.load(gk, gs, gv, gb)
        compare_find(t, ref, np.concatenate([gk[:4000], er[:2000], w.uniform_keys(rng, 2000)]))


def test_errors_leave_table_unchanged():
    rng = np.random.default_rng(1300)
    t = hkv.Table(16 * 128, 4, hkv.LRU, deterministic=True)
    o = oracle.OracleTable(16, 4, oracle.LRU)
    keys = w.uniform_keys(rng, 1000, distinct=True)
    compare_upsert(t, o, keys, w.normal_values(rng, 1000, 4), deterministic=True)
    before = export_state(t)
    bad = keys.copy()
    bad[500] = np.uint64(2**63 + 5)
    with pytest.raises(hkv.HKVError) as e:
        gpu_upsert(t, bad, w.normal_values(rng, 1000, 4))
    assert e.value.code == 2
    dup = np.concatenate([keys[:10], keys[:1]])
    with pytest.raises(hkv.HKVError) as e:
        gpu_upsert(t, dup, w.normal_values(rng, 11, 4))
    assert e.value.code == 3
    t.erase(dev(np.array([5, 2**64 - 1], np.uint64)))
    with pytest.raises(hkv.HKVError):
        t.sync()
    same_state(export_state(t), before)
    # empty batches are no-ops
    gpu_upsert(t, np.zeros(0, np.uint64), np.zeros((0, 4), np.float32))
    t.find(dev(np.zeros(0, np.uint64)))
    t.assign(dev(np.zeros(0, np.uint64)))
    t.erase(dev(np.zeros(0, np.uint64)))
    same_state(export_state(t), before)
    # a batch the device refuses still consumed its step number
    assert t.get_step() == 3


def _check_batch_invariants(t, nb, keys, st, ek, es):
    """Invariants after one LFU batch: a new key's score is its multiplicity."""
    gk, gs, gv, gb = export_state(t)
    b1, b2, _ = oracle.map_keys(nb, True, gk)
    inv.check_state(gk, gs, gb, nb, b1, b2, t.capacity)
    uk, last, mult = np.unique(keys[::-1], return_index=True, return_counts=True)
    last = keys.size - 1 - last
    ust = st[last]
    resident = np.isin(uk, gk)
    assert np.all(resident[ust == hkv.ST_INSERTED])
    assert not np.any(resident[ust == hkv.ST_REJECTED])
    rej = uk[ust == hkv.ST_REJECTED]
    rs = mult.astype(np.uint64)[ust == hkv.ST_REJECTED]
    rb1, rb2, _ = oracle.map_keys(nb, True, rej)
    eb1, eb2, _ = oracle.map_keys(nb, True, ek)
    inv.check_admission(gk, gs, gb, nb, rej, rs, rb1, rb2, ek, es, eb1, eb2)
    assert not np.any(np.isin(ek, gk)), "an evicted key is still resident"
    return gk, gs, gv, gb


def test_dual_bucket_invariants_count_and_find():
    """Single-table shape at reduced size: 2^12 buckets, dim 32, LFU,
    dual-bucket, uniform fill to lambda = 0.5 / 0.9 / 1.0, then Zipf(1.05)
    batches over a 2^32 universe."""
    rng = np.random.default_rng(w.seed_for(2))
    nb, dim = 1 << 12, 32
    t = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True)
    o = oracle.OracleTable(nb, dim, oracle.LFU, True)
    z = w.Zipf(1.05, 1 << 32)
    cap = nb * 128
    for lam in (0.5, 0.9, 1.0):
        for _ in range(40):
            if t.size() >= lam * cap * 0.999:
                break
            keys = w.uniform_keys(rng, 1 << 16, universe=1 << 32)
            vals = w.normal_values(rng, keys.size, dim)
            gst, gek, ges, _ = gpu_upsert(t, keys, vals)
            o.insert_or_assign(keys, vals)
            _check_batch_invariants(t, nb, keys, gst, gek, ges)
        gs_, os_ = t.size(), o.size()
        assert abs(gs_ - os_) <= 0.001 * os_, (lam, gs_, os_)
        for _ in range(3):
            keys = z.keys(rng, 1 << 17)
            vals = w.normal_values(rng, keys.size, dim)
            resident_before = set(export_state(t)[0].tolist())
            gst, gek, ges, _ = gpu_upsert(t, keys, vals)
            o.insert_or_assign(keys, vals)
            gk, gs, gv, gb = _check_batch_invariants(t, nb, keys, gst, gek, ges)
            assert set(gek.tolist()) <= resident_before, "evicted a key that was not resident"
            # last value written wins
            pos = {int(k): i for i, k in enumerate(keys.tolist())}
            idx = np.searchsorted(gk, np.array(list(pos.keys()), np.uint64))
            idx = np.clip(idx, 0, gk.size - 1)
            for (k, i), j in zip(pos.items(), idx):
                if gk[j] == k:
                    assert gv[j].tobytes() == vals[i].tobytes()
            gs_, os_ = t.size(), o.size()
            assert abs(gs_ - os_) <= 0.001 * os_, (lam, gs_, os_)
        # find on the GPU's own state vs the oracle loaded with it
        gk, gs, gv, gb = export_state(t)
        ref = oracle.OracleTable(nb, dim, oracle.LFU, True)
        ref.load(gk, gs, gv, gb)
        q = np.concatenate([z.keys(rng, 20000), w.uniform_keys(rng, 20000, universe=1 << 32)])
        compare_find(t, ref, q)


@pytest.mark.parametrize("evicted_values", [True, False])
def test_tiered_values_in_host_memory(evicted_values):
    """Values past a small HBM budget live in pinned mapped host slices; the
    results are the same bit for bit. Host-memory rows are written after the
    probes, grouped by host region (phase I always; phase U too when no
    evicted values are asked for), and find copies host rows the same way."""
    rng = np.random.default_rng(1400)
    nb, dim = 128, 16
    slice_bytes = 8 * 128 * dim * 4                       # 8 buckets per slice
    t = hkv.Table(nb * 128, dim, hkv.LFU, hbm_value_budget_bytes=5 * slice_bytes,
                  slice_bytes=slice_bytes)
    assert t.hbm_value_slots == 5 * 8 * 128
    o = oracle.OracleTable(nb, dim, oracle.LFU)
    z = w.Zipf(0.99, 1 << 20)
    for _ in range(6):
        keys = z.keys(rng, 8000)
        vals = w.normal_values(rng, keys.size, dim)
        if evicted_values:
            compare_upsert(t, o, keys, vals)
        else:
            ost, oek, oes, _ = o.insert_or_assign(keys, vals)
            gst, gek, ges, _ = gpu_upsert(t, keys, vals, want_values=False)
            assert np.array_equal(gst, ost), "statuses differ"
            o_ord = np.argsort(oek, kind="stable")
            assert np.array_equal(gek, oek[o_ord]) and np.array_equal(ges, oes[o_ord])
        compare_find(t, o, z.keys(rng, 6000))
    same_state(export_state(t), o.export())
    compare_find(t, o, z.keys(rng, 10000))


def test_tiered_dual_bucket_invariants_and_last_value():
    """A dual-bucket table with most value rows in host memory, driven past
    lambda 1 with Zipf batches: phase I writes the rows of host-memory slots
    after the victim searches. The invariants hold, the size stays within
    0.1% of the oracle's, every resident key holds the last value written to
    it, and find on the GPU's own state matches the oracle loaded with it."""
    rng = np.random.default_rng(1450)
    nb, dim = 256, 32
    slice_bytes = 16 * 128 * dim * 4                      # 16 buckets per slice
    t = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True,
                  hbm_value_budget_bytes=3 * slice_bytes, slice_bytes=slice_bytes)
    assert t.hbm_value_slots == 3 * 16 * 128
    o = oracle.OracleTable(nb, dim, oracle.LFU, True)
    z = w.Zipf(1.05, 1 << 20)
    last = {}
    for b in range(10):
        # uniform keys past the capacity, then Zipf batches at lambda 1
        keys = w.uniform_keys(rng, 9000) if b < 6 else z.keys(rng, 12000)
        vals = w.normal_values(rng, keys.size, dim)
        # no evicted values asked for: phase U defers its host rows too
        gst, gek, ges, _ = gpu_upsert(t, keys, vals, want_values=False)
        o.insert_or_assign(keys, vals)
        for k, v in zip(keys.tolist(), vals):
            last[k] = v
        gk, gs, gv, gb = _check_batch_invariants(t, nb, keys, gst, gek, ges)
        assert abs(t.size() - o.size()) <= 0.001 * o.size()
    assert t.size() > 0.99 * t.capacity
    for k, v in zip(gk.tolist(), gv):
        assert v.tobytes() == last[k].tobytes(), "a resident key lost its last value"
    ref = oracle.OracleTable(nb, dim, oracle.LFU, True)
    ref.load(gk, gs, gv, gb)
    compare_find(t, ref, np.concatenate([z.keys(rng, 8000), w.uniform_keys(rng, 4000)]))


def test_streams_follow_the_triple_group_order():
    """An inserter on one stream and readers on others: each reader sees
    exactly the batches issued before it (the scheduler inserts the waits)."""
    rng = np.random.default_rng(1500)
    nb, dim = 256, 32
    t = hkv.Table(nb * 128, dim, hkv.LRU)
    o = oracle.OracleTable(nb, dim, oracle.LRU)
    streams = [torch.cuda.Stream() for _ in range(3)]
    pending = []
    for r in range(6):
        keys = w.uniform_keys(rng, 4096, distinct=True)
        vals = w.normal_values(rng, 4096, dim)
        kd, vd = dev(keys), dev(vals)
        torch.cuda.synchronize()
        with torch.cuda.stream(streams[r % 3]):
            t.insert_or_assign(kd, vd)
        o.insert_or_assign(keys, vals)
        q = np.concatenate([keys[:2000], w.uniform_keys(rng, 500)])
        qd = dev(q)
        torch.cuda.synchronize()
        with torch.cuda.stream(streams[(r + 1) % 3]):
            out, found, _ = t.find(qd)
        ov, of, _ = o.find(q)
        pending.append((streams[(r + 1) % 3], out, found, ov, of))
    torch.cuda.synchronize()
    for s, out, found, ov, of in pending:
        assert np.array_equal(host(found).astype(bool), of)
        assert np.array_equal(host(out)[of].view(np.uint32), ov[of].view(np.uint32))


def test_counters_account_for_every_key():
    rng = np.random.default_rng(1600)
    nb, dim = 64, 4
    t = hkv.Table(nb * 128, dim, hkv.LFU)
    keys = w.uniform_keys(rng, 12000, distinct=True)
    t.reset_counters()
    st, _, _, _ = gpu_upsert(t, keys, w.normal_values(rng, keys.size, dim))
    c = t.read_counters()
    assert c["updated"] == 0
    assert c["inserted"] + c["evicted"] + c["rejected"] >= keys.size
    t.find(dev(keys))
    c = t.read_counters()
    assert c["find_hit"] == int(np.sum(st == hkv.ST_INSERTED))
    assert c["find_hit"] + c["find_miss"] == keys.size


@pytest.mark.parametrize("policy,dim", [(hkv.LFU, 32), (hkv.LRU, 8), (hkv.CUSTOM, 3),
                                        (hkv.EPOCH_LFU, 4)])
def test_deterministic_dual_bucket_bit_exact(policy, dim):
    """Deterministic dual-bucket upsert runs phase I in batch order (waves of
    keys with disjoint candidate buckets) and so equals Algorithm 3 run key
    by key: statuses, evicted sets and the full state including the bucket
    of every key, bit for bit, from an empty table through lambda = 1 and
    well past it, with batches that mix resident and fresh keys."""
    rng = np.random.default_rng(9500 + policy * 10 + dim)
    nb = 256
    t = hkv.Table(nb * 128, dim, policy, dual_bucket=True, deterministic=True)
    o = oracle.OracleTable(nb, dim, policy, True)
    sizes = [1, 0, 5000, 9000, 7001, 12000, 3, 8192, 10000, 6000, 9000, 2047]
    for e, n in enumerate(sizes):
        t.set_epoch(e)
        o.set_epoch(e)
        resident = o.export()[0]
        k_old = rng.choice(resident, min(n // 3, resident.size), replace=False) if n else \
            np.zeros(0, np.uint64)
        k_new = w.uniform_keys(rng, n - k_old.size, distinct=True)
        keys = np.concatenate([k_old, k_new]).astype(np.uint64)
        assert np.unique(keys).size == keys.size
        rng.shuffle(keys)
        vals = w.normal_values(rng, keys.size, dim)
        sc = rng.integers(0, 50, keys.size, dtype=np.uint64) if policy == hkv.CUSTOM else None
        compare_upsert(t, o, keys, vals, sc, deterministic=True)
        same_state(export_state(t), o.export())
    assert o.size() == nb * 128  # filled, then evicting
    q = np.concatenate([o.export()[0][:3000], w.uniform_keys(rng, 3000)])
    compare_find(t, o, q)


def test_deterministic_dual_tables_refuse_the_graph_and_noalloc_paths():
    t = hkv.Table(128 * 16, 4, hkv.LRU, dual_bucket=True, deterministic=True)
    with pytest.raises(hkv.HKVError):
        hkv.Batch([t], [100])
    keys = torch.arange(1, 11, dtype=torch.int64, device="cuda")
    vals = torch.zeros((10, 4), device="cuda")
    with pytest.raises(hkv.HKVError):
        t.insert_or_assign_noalloc(keys, vals)


@pytest.mark.parametrize("dim,budget_slices", [(16, None), (3, None), (8, 1)])
def test_find_ptr_and_gather_bit_exact(dim, budget_slices):
    """find* returns the address of each hit's value row: gathering through
    the addresses gives exactly the oracle's rows, misses get NULL and keep
    their output rows, distinct keys get distinct addresses. With a one-slice
    HBM budget most rows live in mapped host memory."""
    rng = np.random.default_rng(9700 + dim)
    nb = 64
    kw = {}
    if budget_slices is not None:
        kw = dict(hbm_value_budget_bytes=8 * 128 * dim * 4, slice_bytes=8 * 128 * dim * 4)
    t = hkv.Table(nb * 128, dim, hkv.LFU, **kw)
    o = oracle.OracleTable(nb, dim, oracle.LFU)
    z = w.Zipf(1.05, 20000)
    for n in (6000, 9000, 3000):
        keys = z.keys(rng, n)
        vals = w.normal_values(rng, n, dim)
        compare_upsert(t, o, keys, vals)
    q = np.concatenate([z.keys(rng, 4000), w.uniform_keys(rng, 2000), np.zeros(0, np.uint64)])
    n = q.size
    found = torch.empty(n, dtype=torch.uint8, device="cuda")
    ptrs = t.find_ptr(dev(q), found=found)
    out = nan_filled(n, dim)
    hkv.gather_rows(ptrs, dim, out)
    torch.cuda.synchronize()
    ov = np.zeros((n, dim), np.uint32)
    ov[:] = NAN_BITS
    ov, of, _ = o.find(q, ov.view(np.float32))
    p = host(ptrs).view(np.uint64)
    gf = host(found).astype(bool)
    assert np.array_equal(gf, of), "hit masks differ"
    assert np.array_equal(p != 0, of), "NULL exactly for the misses"
    assert np.array_equal(host(out).view(np.uint32), ov.view(np.uint32)), "rows differ"
    hit_keys, first = np.unique(q[of], return_index=True)
    assert np.unique(p[of][first]).size == hit_keys.size, "distinct keys share an address"
    if dim % 4 == 0:
        assert np.all(p[of] % 16 == 0)


def test_export_batch_if_matches_filtered_export():
    rng = np.random.default_rng(9800)
    nb, dim = 64, 5
    t = hkv.Table(nb * 128, dim, hkv.CUSTOM)
    o = oracle.OracleTable(nb, dim, oracle.CUSTOM)
    for n in (5000, 7000, 4000):
        keys = w.uniform_keys(rng, n, distinct=True)
        compare_upsert(t, o, keys, w.normal_values(rng, n, dim),
                       rng.integers(0, 1000, n, dtype=np.uint64))
    ok, os_, ov, ob = o.export()
    cap = nb * 128
    for lo, hi in ((0, 2**64 - 1), (100, 499), (500, 500), (1000, 2000), (0, 0)):
        k = torch.empty(cap, dtype=torch.int64, device="cuda")
        s = torch.empty(cap, dtype=torch.int64, device="cuda")
        v = torch.empty((cap, dim), dtype=torch.float32, device="cuda")
        cnt, *_ = t.export_batch_if(lo, hi, keys=k, values=v, scores=s)
        torch.cuda.synchronize()
        c = int(cnt.item())
        gk, gs, gv = host(k[:c]), host(s[:c]), host(v[:c])
        order = np.argsort(gk, kind="stable")
        sel = (os_ >= lo) & (os_ <= hi)
        assert c == int(sel.sum()), (lo, hi)
        assert np.array_equal(gk[order], ok[sel])
        assert np.array_equal(gs[order], os_[sel])
        assert np.array_equal(gv[order].view(np.uint32), ov[sel].view(np.uint32))


@pytest.mark.parametrize("policy,dual,det,tiered", [(hkv.LFU, False, False, False),
                                                    (hkv.CUSTOM, False, False, False),
                                                    (hkv.LRU, True, True, False),
                                                    (hkv.LFU, False, False, True),
                                                    (hkv.LRU, True, True, True)])
def test_find_or_insert_bit_exact(policy, dual, det, tiered):
    """find_or_insert against the oracle's: returned rows, found flags and
    the full state after every batch (Zipf batches with duplicates, or
    distinct keys in deterministic dual-bucket mode), through the point
    where the table is full and refuses keys. Tiered: most value rows in
    host memory, where insert_or_assign defers its row writes; residents
    must keep their rows."""
    rng = np.random.default_rng(9900 + policy + 10 * dual)
    nb, dim = 32, 4
    budget = dict(hbm_value_budget_bytes=2 * 4 * 128 * dim * 4,
                  slice_bytes=4 * 128 * dim * 4) if tiered else {}
    t = hkv.Table(nb * 128, dim, policy, dual_bucket=dual, deterministic=det, **budget)
    if tiered:
        assert t.hbm_value_slots == 2 * 4 * 128
    o = oracle.OracleTable(nb, dim, policy, dual)
    z = w.Zipf(1.05, 12000)
    for n in (3000, 0, 1, 5000, 7000, 4096):
        keys = w.uniform_keys(rng, n, universe=12000, distinct=True) if det else z.keys(rng, n)
        vals = w.normal_values(rng, n, dim)
        sc = rng.integers(0, 40, n, dtype=np.uint64) if policy == hkv.CUSTOM else None
        orows, ofound = o.find_or_insert(keys, vals, sc)
        io = dev(vals.reshape(n, dim)) if n else torch.empty((0, dim), device="cuda")
        found = torch.empty(n, dtype=torch.uint8, device="cuda")
        t.find_or_insert(dev(keys), io, None if sc is None else dev(sc), found)
        torch.cuda.synchronize()
        assert np.array_equal(host(found), ofound)
        assert np.array_equal(host(io).view(np.uint32), orows.view(np.uint32))
        same_state(export_state(t), o.export())


def test_rows_from_page_locked_host_memory():
    """insert_or_assign and assign read their rows in place from mapped
    page-locked host memory: the same statuses, evicted sets and final state
    as the same batches from device memory, through fills, updates and the
    victim searches of full buckets (the key universe is 12x the capacity).
    Single-bucket mode, whose results do not depend on the schedule; the row
    paths are the same in dual mode."""
    rng = np.random.default_rng(9300)
    nb, dim = 32, 8
    a = hkv.Table(nb * 128, dim, hkv.LFU)
    b = hkv.Table(nb * 128, dim, hkv.LFU)
    z = w.Zipf(0.9, 12 * nb * 128)
    evicted = 0
    for rnd in range(6):
        n = 3000
        keys = z.keys(rng, n)
        vals = w.normal_values(rng, n, dim)
        outs = []
        for t, v in ((a, torch.from_numpy(vals.copy()).pin_memory()), (b, dev(vals))):
            st = torch.empty(n, dtype=torch.uint8, device="cuda")
            ek = torch.empty(n, dtype=torch.int64, device="cuda")
            ne = torch.zeros(1, dtype=torch.int64, device="cuda")
            t.insert_or_assign(dev(keys), v, None, st, ek, None, None, ne)
            t.sync()
            outs.append((host(st), np.sort(host(ek)[:int(ne.item())])))
        assert np.array_equal(outs[0][0], outs[1][0]), "statuses"
        assert np.array_equal(outs[0][1], outs[1][1]), "evicted keys"
        evicted += outs[0][1].size
        if rnd % 2:
            ak = z.keys(rng, 500)
            av = w.normal_values(rng, 500, dim)
            a.assign(dev(ak), torch.from_numpy(av.copy()).pin_memory())
            b.assign(dev(ak), dev(av))
    a.sync()
    b.sync()
    assert evicted > 0, "no victim search ran"
    same_state(export_state(a), export_state(b))


@pytest.mark.parametrize("dual,dim,tiered", [(False, 16, False), (True, 3, False),
                                             (True, 8, True)])
def test_find_without_digests_matches_the_oracle(dual, dim, tiered):
    """The digest ablation (hkv_find_full_keys: every key of a probed bucket
    compared, no digest line) returns exactly what find returns and what the
    oracle returns: rows, misses left untouched, found flags; with values
    NULL it is contains."""
    rng = np.random.default_rng(9950 + dim + 10 * dual)
    nb = 64
    budget = dict(hbm_value_budget_bytes=2 * 4 * 128 * dim * 4,
                  slice_bytes=4 * 128 * dim * 4) if tiered else {}
    t = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=dual, **budget)
    o = oracle.OracleTable(nb, dim, oracle.LFU, dual)
    z = w.Zipf(1.05, 20000)
    for n in (6000, 9000, 4000):
        keys = z.keys(rng, n)
        vals = w.normal_values(rng, n, dim)
        gpu_upsert(t, keys, vals)
        o.insert_or_assign(keys, vals)
    gk, gs, gv, gb = export_state(t)
    ref = oracle.OracleTable(nb, dim, oracle.LFU, dual)
    ref.load(gk, gs, gv, gb)
    q = np.concatenate([z.keys(rng, 5000), w.uniform_keys(rng, 2000)])
    n = q.size
    out = nan_filled(n, dim)
    found = torch.empty(n, dtype=torch.uint8, device="cuda")
    t.find_full_keys(dev(q), out, found)
    torch.cuda.synchronize()
    ov = np.zeros((n, dim), np.uint32)
    ov[:] = NAN_BITS
    ov, of, _ = ref.find(q, ov.view(np.float32))
    assert np.array_equal(host(found).astype(bool), of)
    assert np.array_equal(host(out).view(np.uint32), ov.view(np.uint32))
    _, only = t.find_full_keys(dev(q))
    assert np.array_equal(host(only).astype(bool), of)
    assert of.sum() > 0


def test_admission_burst_table9_bit_exact():
    """Table 9 (Exp 3d) on the GPU, scaled to a full 2^17-slot table: every
    bucket holds 128 keys with caller scores in [2, 1000); a burst of fresh
    keys with score 1 is refused whole and leaves the table as it was; the
    same burst with score 10^9 is admitted whole, each key displacing one of
    the originals. Statuses, evicted sets and states bit-exact against the
    oracle."""
    rng = np.random.default_rng(9970)
    nb, dim = 1 << 10, 2
    t = hkv.Table(nb * 128, dim, hkv.CUSTOM)
    o = oracle.OracleTable(nb, dim, oracle.CUSTOM)
    keys = w.uniform_keys(rng, nb * 128 * 3, distinct=True)
    b1, _, _ = oracle.map_keys(nb, False, keys)
    sel = np.concatenate([np.flatnonzero(b1 == b)[:128] for b in range(nb)])
    assert sel.size == nb * 128
    vals = w.normal_values(rng, sel.size, dim)
    sc = rng.integers(2, 1000, sel.size, dtype=np.uint64)
    compare_upsert(t, o, keys[sel], vals, sc)
    assert t.size() == nb * 128
    before = export_state(t)
    burst = w.uniform_keys(rng, 32768, distinct=True)
    bv = w.normal_values(rng, burst.size, dim)
    st = compare_upsert(t, o, burst, bv, np.full(burst.size, 1, np.uint64))
    assert np.all(st == hkv.ST_REJECTED)
    after = export_state(t)
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    st = compare_upsert(t, o, burst, bv, np.full(burst.size, 10**9, np.uint64))
    assert np.all(st == hkv.ST_INSERTED)
    same_state(export_state(t), o.export())
    assert host(t.contains(dev(burst))).all() and t.size() == nb * 128
