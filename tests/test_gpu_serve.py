"""Serving loop (hkv_serve_run): a trace of find / upsert requests with
Poisson arrivals, replayed through continuous batching and through the plain
one-request-at-a-time path on two identical sets of tables. Every request's
result is the same in the mix as alone (bit for bit: found masks, found
values, statuses), the final table states agree, batching really merged
requests, and the HBM admission budget is enforced."""
import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, same_state  # noqa: E402

DIMS = (8, 16, 32, 64)
BUCKETS = (64, 32, 128, 16)


def tables_filled(seed):
    rng = np.random.default_rng(seed)
    ts = []
    for b, d in zip(BUCKETS, DIMS):
        t = hkv.Table(b * 128, d, hkv.LRU)
        k = w.uniform_keys(rng, b * 100, universe=60000)
        t.insert_or_assign(dev(k), dev(w.normal_values(rng, k.size, d)))
        ts.append(t)
    torch.cuda.synchronize()
    return ts


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
    for a, b in zip(items, items_alone):
        fa, fb = a["flags"].numpy(), b["flags"].numpy()
        assert np.array_equal(fa, fb)
        if a["op"] == hkv.OP_FIND:
            m = fa.astype(bool)
            assert np.array_equal(a["values"].numpy()[m].view(np.uint32),
                                  b["values"].numpy()[m].view(np.uint32))
        else:
            assert np.all(fa > 0)
    for x, y in zip(mixed, alone):
        same_state(export_state(x), export_state(y))
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
