"""The single-table configuration at full size, in the launch configuration
bench.py times: 2^26 slots (2^19 buckets x 128), dim 32, LFU, dual-bucket,
filled with uniform keys over 2^32 to lambda ~ 1, then batches of 2^20
Zipf(1.05) keys (duplicates included) through hkv_insert_or_assign.

The oracle cannot replay 2^26-slot tables in seconds, so every check here is
a property that fixes the result at any size, computed from the table's own
state before and after each batch over all 2^26 slots (set operations as
sorts and binary searches in torch on the device; candidate buckets from the
oracle's key mapping): the structural invariants; statuses by residency at
batch start and end; the evicted output equal to the set of keys the batch
removed, with their scores at removal; LFU scores (old + multiplicity, or
multiplicity); admission (every refused or removed key below a full
candidate bucket's minimum); the last occurrence's value for every resident
key of the batch; and contains() on a sample against membership in the
exported state."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import host  # noqa: E402

NB = 1 << 19
DIM = 32
BATCH = 1 << 20
UNIVERSE = 1 << 32
SLOTS = 128


def export_kss(t):
    """(keys, scores, buckets) of every occupied slot as device int64
    tensors sorted by key (keys < 2^63 and LFU scores sort as signed)."""
    cap = t.capacity
    k = torch.empty(cap, dtype=torch.int64, device="cuda")
    s = torch.empty(cap, dtype=torch.int64, device="cuda")
    g = torch.empty(cap, dtype=torch.int64, device="cuda")
    cnt, *_ = t.export_batch(0, cap, keys=k, scores=s, slots=g)
    torch.cuda.synchronize()
    c = int(cnt.item())
    o = torch.argsort(k[:c])
    return k[:c][o], s[:c][o], g[:c][o] // SLOTS


def member(sorted_ref, q):
    """(q in sorted_ref, index of q in sorted_ref where present)."""
    j = torch.searchsorted(sorted_ref, q).clamp_(max=max(sorted_ref.numel() - 1, 0))
    return sorted_ref[j] == q, j


def buckets_of(keys_dev):
    b1, b2, _ = oracle.map_keys(NB, True, host(keys_dev))
    return (torch.from_numpy(b1.view(np.int64)).cuda(), torch.from_numpy(b2.view(np.int64)).cuda())


def sk_less(s1, k1, s2, k2):
    return (s1 < s2) | ((s1 == s2) & (k1 < k2))


def test_single_table_full_size_properties():
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.seed_for(2, 7))
    t = hkv.Table(NB * 128, DIM, hkv.LFU, dual_bucket=True)
    fill_vals = torch.randn((BATCH, DIM), device="cuda", generator=gen)
    for _ in range(200):
        if t.size() >= 0.999 * t.capacity:
            break
        t.insert_or_assign(w.uniform_keys_torch(gen, BATCH, UNIVERSE), fill_vals)
    assert t.size() >= 0.99 * t.capacity
    z = w.Zipf(1.05, UNIVERSE)
    for _ in range(2):
        kb, sb, _ = export_kss(t)
        keys = w.zipf_keys_torch(gen, z, BATCH)
        vals = torch.randn((BATCH, DIM), device="cuda", generator=gen)
        st = torch.empty(BATCH, dtype=torch.uint8, device="cuda")
        ek = torch.empty(BATCH, dtype=torch.int64, device="cuda")
        es = torch.empty(BATCH, dtype=torch.int64, device="cuda")
        ne = torch.zeros(1, dtype=torch.int64, device="cuda")
        t.insert_or_assign(keys, vals, None, st, ek, es, None, ne)
        t.sync()
        ka, sa, ba = export_kss(t)

        # structure: unique keys, each in a candidate bucket, <= 128 a bucket
        assert bool((ka[1:] > ka[:-1]).all()), "duplicate keys in the table"
        b1, b2 = buckets_of(ka)
        assert bool(((ba == b1) | (ba == b2)).all()), "entry outside its candidate buckets"
        counts = torch.bincount(ba, minlength=NB)
        assert int(counts.max()) <= SLOTS and int(counts.sum()) == t.size()

        # statuses from residency at batch start and end, the same for every
        # occurrence of a key
        uk, inv_idx, mult = torch.unique(keys, return_inverse=True, return_counts=True)
        pos = torch.arange(BATCH, device="cuda")
        last = torch.full_like(uk, -1).scatter_reduce_(0, inv_idx, pos, "amax")
        before, jb = member(kb, uk)
        after, ja = member(ka, uk)
        ust = st[last].long()
        assert bool(((ust == hkv.ST_UPDATED) == before).all())
        assert bool(((ust == hkv.ST_INSERTED) == (~before & after)).all())
        assert bool(((ust == hkv.ST_REJECTED) == (~before & ~after)).all())
        assert bool((st.long() == ust[inv_idx]).all()), "occurrences of a key disagree"

        # evicted output = exactly the keys the batch removed, with the score
        # each had when removed (old, or old + multiplicity if phase U
        # updated it first)
        m = int(ne.item())
        evk, o = torch.sort(ek[:m])
        evs = es[:m][o]
        still, _ = member(ka, kb)
        removed = kb[~still]
        assert torch.equal(evk, removed), "evicted output is not the removed set"
        _, jold = member(kb, evk)
        in_batch, ju = member(uk, evk)
        want_evs = sb[jold] + torch.where(in_batch, mult[ju], torch.zeros_like(mult[ju]))
        assert torch.equal(evs, want_evs), "evicted scores"

        # LFU scores of the batch's resident keys
        want = torch.where(before, sb[jb] + mult, mult)
        assert torch.equal(sa[ja][after], want[after]), "LFU scores"

        # admission: refused and removed keys sit below a full candidate
        # bucket's (score, key) minimum
        o = torch.sort(sa, stable=True)[1]          # keys already ascending
        o = o[torch.sort(ba[o], stable=True)[1]]    # -> (bucket, score, key)
        bs, ss, ks = ba[o], sa[o], ka[o]
        first = torch.ones_like(bs, dtype=torch.bool)
        first[1:] = bs[1:] != bs[:-1]
        big = torch.iinfo(torch.int64).max
        ms = torch.full((NB,), big, dtype=torch.int64, device="cuda")
        mk = torch.full((NB,), big, dtype=torch.int64, device="cuda")
        ms[bs[first]] = ss[first]
        mk[bs[first]] = ks[first]
        rej = ust == hkv.ST_REJECTED
        for k_, s_ in ((uk[rej], mult[rej]), (evk, evs)):
            c1, c2 = buckets_of(k_)
            ok1 = (counts[c1] == SLOTS) & sk_less(s_, k_, ms[c1], mk[c1])
            ok2 = (counts[c2] == SLOTS) & sk_less(s_, k_, ms[c2], mk[c2])
            assert bool((ok1 | ok2).all()), "refused or removed key above its buckets' minimum"

        # the last occurrence's value for every resident key of the batch
        q = uk[after]
        out = torch.empty((q.numel(), DIM), device="cuda")
        fnd = torch.empty(q.numel(), dtype=torch.uint8, device="cuda")
        t.find(q, out, fnd)
        torch.cuda.synchronize()
        assert bool(fnd.bool().all())
        assert torch.equal(out.view(torch.int32), vals[last[after]].view(torch.int32))

    # contains() on a sample against membership in the final state
    qs = torch.cat([w.zipf_keys_torch(gen, z, 1 << 18), w.uniform_keys_torch(gen, 1 << 18,
                                                                            UNIVERSE)])
    fnd = t.contains(qs)
    torch.cuda.synchronize()
    want, _ = member(ka, qs)
    assert torch.equal(fnd.bool(), want)
    t.close()
