"""Batched multi-table rounds (hkv_batch_run) against the CPU oracle.

Each round gives every table at most one operation (Algorithms 1-2 applied
per table, Sec. 3.2-3.3). The oracle replays the same rounds in slot order
with one oracle table per CUDA table: a find reads the state at round start,
an upsert is insert_or_assign. Single-bucket tables make upsert
schedule-independent, so found masks, found rows, statuses and the final
state (key, score, value, bucket) must match bit for bit, round after round,
with the graph replayed across rounds of different sizes (including empty
rounds) and tables of different value widths. Plain per-table calls run
beside them as a second witness of the same history."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import NAN_BITS, dev, export_state, host, nan_filled, same_state  # noqa: E402

DIMS = (16, 32, 64, 8, 3, 128)
BUCKETS = (64, 128, 32, 256, 16, 32)
ORACLE_POLICY = {hkv.LRU: oracle.LRU, hkv.LFU: oracle.LFU, hkv.CUSTOM: oracle.CUSTOM}


def oracle_find_rows(o, keys, dim):
    ov = np.zeros((keys.size, dim), np.uint32)
    ov[:] = NAN_BITS
    rows, of, _ = o.find(keys, ov.view(np.float32))
    return rows.view(np.uint32), of


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("policy", [hkv.LRU, hkv.LFU, hkv.CUSTOM])
def test_batched_rounds_match_the_oracle(use_graph, policy):
    rng = np.random.default_rng(7000 + use_graph + 10 * policy)
    plain = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    batched = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    orc = [oracle.OracleTable(b, d, ORACLE_POLICY[policy]) for b, d in zip(BUCKETS, DIMS)]
    max_keys = [6000, 9000, 3000, 20000, 1500, 4000]
    batch = hkv.Batch(batched, max_keys)
    z = w.Zipf(1.05, 50000)
    n_find_hits = n_upserts = 0
    for rnd in range(14):
        ops, expect = [], []
        for i, (t, m) in enumerate(zip(plain, max_keys)):
            kind = rng.choice(["none", "find", "upsert"], p=[0.1, 0.5, 0.4])
            n = int(min(m, rng.lognormal(np.log(m / 4), 1.0))) if rnd else m
            if rnd % 5 == 3 and i == 0:
                n = 0
            if kind == "none":
                ops.append(None)
                expect.append(None)
                continue
            keys_h = z.keys(rng, n)
            keys = dev(keys_h)
            if kind == "find":
                out_p = nan_filled(n, t.dim)
                fnd_p = torch.empty(n, dtype=torch.uint8, device="cuda")
                t.find(keys, out_p, fnd_p)
                out_b = nan_filled(max(n, 1), t.dim)
                fnd_b = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                ops.append(dict(op=hkv.OP_FIND, keys=keys, values=out_b, flags=fnd_b, n=n))
                ov, of = oracle_find_rows(orc[i], keys_h, t.dim)
                n_find_hits += int(of.sum())
                expect.append(("find", out_p, fnd_p, out_b, fnd_b, n, ov, of))
            else:
                vals_h = w.normal_values(rng, n, t.dim)
                vals = dev(vals_h)
                sc_h = rng.integers(0, 1000, n, dtype=np.uint64) if policy == hkv.CUSTOM else None
                sc = dev(sc_h) if sc_h is not None else None
                st_p = torch.empty(n, dtype=torch.uint8, device="cuda")
                t.insert_or_assign(keys, vals, sc, st_p)
                st_b = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                ops.append(dict(op=hkv.OP_UPSERT, keys=keys, values=vals, flags=st_b, scores=sc,
                                n=n))
                ost, _, _, _ = orc[i].insert_or_assign(keys_h, vals_h, sc_h)
                n_upserts += n
                expect.append(("upsert", st_p, st_b, n, ost))
        batch.run(ops, use_graph=use_graph)
        torch.cuda.synchronize()
        for e in expect:
            if e is None:
                continue
            if e[0] == "find":
                _, out_p, fnd_p, out_b, fnd_b, n, ov, of = e
                gf = host(fnd_b)[:n].astype(bool)
                assert np.array_equal(gf, of), f"round {rnd}: hit mask differs from the oracle"
                assert np.array_equal(host(out_b)[:n].view(np.uint32), ov), \
                    f"round {rnd}: rows differ from the oracle (hits and untouched misses)"
                assert np.array_equal(host(fnd_p), host(fnd_b)[:n])
                assert np.array_equal(host(out_p).view(np.uint32), host(out_b)[:n].view(np.uint32))
            else:
                _, st_p, st_b, n, ost = e
                assert np.array_equal(host(st_b)[:n], ost), \
                    f"round {rnd}: statuses differ from the oracle"
                assert np.array_equal(host(st_p), host(st_b)[:n])
        for t, o in zip(batched, orc):
            assert t.get_step() == o.step
    assert n_find_hits > 0 and n_upserts > 0
    for a, b, o in zip(plain, batched, orc):
        a.sync()
        b.sync()
        same_state(export_state(b), o.export())
        same_state(export_state(a), o.export())
        assert a.get_step() == b.get_step() == o.step
    for o in orc:
        o.close()
    batch.close()


def test_batched_rounds_evict_like_the_oracle_at_full_load():
    """Tables driven past lambda = 1 within graph-replayed rounds: every round
    upserts fresh keys into full buckets, so admission and victim choice are
    exercised on every table; the state after each round equals the oracle's."""
    rng = np.random.default_rng(7100)
    dims, nbs = (8, 64, 24), (8, 4, 16)
    tabs = [hkv.Table(b * 128, d, hkv.LRU) for b, d in zip(nbs, dims)]
    orc = [oracle.OracleTable(b, d, oracle.LRU) for b, d in zip(nbs, dims)]
    batch = hkv.Batch(tabs, [3000] * 3)
    for rnd in range(8):
        ops, expect = [], []
        for i, (t, o) in enumerate(zip(tabs, orc)):
            n = int(rng.integers(200, 3000))
            k = w.uniform_keys(rng, n, universe=1 << 20)
            v = w.normal_values(rng, n, t.dim)
            st = torch.empty(n, dtype=torch.uint8, device="cuda")
            ops.append(dict(op=hkv.OP_UPSERT, keys=dev(k), values=dev(v), flags=st, n=n))
            ost, _, _, _ = o.insert_or_assign(k, v)
            expect.append((st, ost))
        batch.run(ops, use_graph=True)
        torch.cuda.synchronize()
        for t, o, (st, ost) in zip(tabs, orc, expect):
            assert np.array_equal(host(st), ost), f"round {rnd}: statuses differ"
            same_state(export_state(t), o.export())
    assert all(o.size() == o.capacity for o in orc)
    for o in orc:
        o.close()
    batch.close()


def test_batch_refuses_oversized_rounds_and_shared_tables():
    t = hkv.Table(128 * 8, 4)
    with pytest.raises(hkv.HKVError):
        hkv.Batch([t, t], [10, 10])
    b = hkv.Batch([t], [100])
    keys = torch.arange(1, 201, dtype=torch.int64, device="cuda")
    out = torch.empty((200, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(hkv.HKVError):
        b.run([dict(op=hkv.OP_FIND, keys=keys, values=out)])
    b.close()
