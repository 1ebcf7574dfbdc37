"""Serving loop (hkv_serve_run): a trace of find / upsert requests with
Poisson arrivals, replayed through continuous batching and through the plain
one-request-at-a-time path on two identical sets of tables, and through the
CPU oracle in arrival order (each table's requests as a FIFO: Algorithms 1-2
per table, Sec. 3.2-3.3). Every request's result in the mix equals the
oracle's (bit for bit: found masks, found values, statuses) and the result
alone; the final table states equal the oracle's; batching really merged
requests, and the HBM admission budget is enforced."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, same_state  # noqa: E402

DIMS = (8, 16, 32, 64)
BUCKETS = (64, 32, 128, 16)


def tables_filled(seed, use_oracle=False):
    rng = np.random.default_rng(seed)
    ts = []
    for b, d in zip(BUCKETS, DIMS):
        k = w.uniform_keys(rng, b * 100, universe=60000)
        v = w.normal_values(rng, k.size, d)
        if use_oracle:
            t = oracle.OracleTable(b, d, oracle.LRU)
            t.insert_or_assign(k, v)
        else:
            t = hkv.Table(b * 128, d, hkv.LRU)
            t.insert_or_assign(dev(k), dev(v))
        ts.append(t)
    if not use_oracle:
        torch.cuda.synchronize()
    return ts


def oracle_replay(items, seed):
    """Each request's (found or status, rows) from the oracle, in arrival
    order, on oracle tables filled like tables_filled(seed)."""
    orc = tables_filled(seed, use_oracle=True)
    out = []
    for it in items:
        o = orc[it["table"]]
        keys = it["keys"].numpy().view(np.uint64)
        if it["op"] == hkv.OP_FIND:
            rows, found, _ = o.find(keys)
            out.append((found.astype(np.uint8), rows))
        else:
            st, _, _, _ = o.insert_or_assign(keys, it["values"].numpy())
            out.append((st, None))
    return orc, out


def trace(rng, n_req, rate):
    z = w.Zipf(1.1, 60000)
    t, items = 0.0, []
    for i in range(n_req):
        if i >= n_req // 4:  # a burst at t = 0, then Poisson arrivals
            t += rng.exponential(1.0 / rate)
        tab = int(rng.integers(0, len(DIMS)))
        n = int(np.clip(np.rint(np.exp(np.log(512) + rng.standard_normal())), 16, 4096))
        op = hkv.OP_FIND if rng.random() < 0.8 else hkv.OP_UPSERT
        keys = torch.from_numpy(z.keys(rng, n).view(np.int64)).pin_memory()
        if op == hkv.OP_FIND:
            vals = torch.zeros((n, DIMS[tab]), dtype=torch.float32).pin_memory()
        else:
            vals = torch.from_numpy(w.normal_values(rng, n, DIMS[tab])).pin_memory()
        flags = torch.zeros(n, dtype=torch.uint8).pin_memory()
        items.append(dict(arrival_s=t, table=tab, op=op, keys=keys, values=vals, flags=flags))
    return items


def clone_outputs(items):
    out = []
    for it in items:
        c = dict(it)
        if it["op"] == hkv.OP_FIND:
            c["values"] = torch.zeros_like(it["values"]).pin_memory()
        c["flags"] = torch.zeros_like(it["flags"]).pin_memory()
        out.append(c)
    return out


def test_each_request_is_the_same_alone_and_in_the_mix():
    rng = np.random.default_rng(9100)
    items = trace(rng, 600, rate=20000.0)
    mixed = tables_filled(9101)
    alone = tables_filled(9101)
    s_mix = hkv.Server(mixed, ring_keys=16384, max_inflight=3)
    s_alone = hkv.Server(alone, ring_keys=16384, max_inflight=1)
    items_alone = clone_outputs(items)
    res_mix = s_mix.run(hkv.make_requests(items), batched=True, use_graph=True)
    res_alone = s_alone.run(hkv.make_requests(items_alone), batched=False)
    orc, expect = oracle_replay(items, 9101)
    n_hits = 0
    for i, (a, b, (of, orows)) in enumerate(zip(items, items_alone, expect)):
        fa, fb = a["flags"].numpy(), b["flags"].numpy()
        assert np.array_equal(fa, of), f"request {i}: flags differ from the oracle"
        assert np.array_equal(fa, fb)
        if a["op"] == hkv.OP_FIND:
            m = fa.astype(bool)
            n_hits += int(m.sum())
            assert np.array_equal(a["values"].numpy()[m].view(np.uint32),
                                  orows[m].view(np.uint32)), f"request {i}: rows differ"
            assert np.array_equal(a["values"].numpy()[m].view(np.uint32),
                                  b["values"].numpy()[m].view(np.uint32))
        else:
            assert np.all(fa > 0)
    assert n_hits > 0
    for x, y, o in zip(mixed, alone, orc):
        same_state(export_state(x), o.export())
        same_state(export_state(y), o.export())
        assert x.get_step() == o.step
        o.close()
    rounds_mix = len({r.round for r in res_mix})
    rounds_alone = len({r.round for r in res_alone})
    assert rounds_alone == len(items)
    assert rounds_mix < len(items), rounds_mix
    # the burst queued at t = 0 is carried by far fewer rounds than requests
    burst = len(items) // 4
    assert len({r.round for r in list(res_mix)[:burst]}) < burst // 2
    for r, it in zip(res_mix, items):
        assert r.done_s >= r.admit_s >= it["arrival_s"] - 1e-6
    s_mix.close()
    s_alone.close()


def test_hbm_budget_is_enforced():
    ts = tables_filled(9200)
    with pytest.raises(hkv.HKVError) as e:
        hkv.Server(ts, ring_keys=1 << 16, hbm_budget_bytes=1 << 20)
    assert e.value.code == 4
    s = hkv.Server(ts, ring_keys=1 << 16, hbm_budget_bytes=8 << 30)
    assert 0 < s.hbm_bytes <= 8 << 30
    s.close()
