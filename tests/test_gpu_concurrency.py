"""Concurrent host clients on one table (Sec. 3.5): threads with their own
streams issue finds and assigns of disjoint key sets under the triple-group
rule and under a reader/writer lock; the final state equals the serial
application of the same calls, and every find sees values that some
completed state held (the value written or the one before it)."""
import threading

import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host, same_state  # noqa: E402


@pytest.mark.parametrize("rw", [False, True])
def test_threads_with_streams_match_serial(rw):
    rng = np.random.default_rng(9600 + rw)
    dim = 4
    t = hkv.Table(256 * 128, dim, hkv.LRU)
    ref = hkv.Table(256 * 128, dim, hkv.LRU)
    keys = w.uniform_keys(rng, 20000, distinct=True)
    v0 = w.normal_values(rng, keys.size, dim)
    for x in (t, ref):
        x.insert_or_assign(dev(keys), dev(v0))
    t.set_concurrency(rw)
    parts = np.array_split(keys, 4)
    new_vals = [w.normal_values(rng, p.size, dim) for p in parts]
    old_of = {int(k): v for k, v in zip(keys, v0)}
    seen = []

    def updater(p, nv):
        s = torch.cuda.Stream()
        for _ in range(5):
            t.assign(dev(p), dev(nv), stream=s)
        s.synchronize()

    def reader():
        s = torch.cuda.Stream()
        q = dev(keys[:4000])
        for _ in range(5):
            out = torch.empty((4000, dim), device="cuda")
            fnd = torch.empty(4000, dtype=torch.uint8, device="cuda")
            t.find(q, out, fnd, stream=s)
            s.synchronize()
            seen.append((host(out), host(fnd)))

    th = [threading.Thread(target=updater, args=(p, nv)) for p, nv in zip(parts, new_vals)]
    th += [threading.Thread(target=reader) for _ in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    torch.cuda.synchronize()
    for p, nv in zip(parts, new_vals):
        ref.assign(dev(p), dev(nv))
    for _ in range(4):  # the same number of step advances: 5 assigns per thread
        for p, nv in zip(parts, new_vals):
            ref.assign(dev(p), dev(nv))
    t.sync()
    ref.sync()
    gk, gs, gv, gb = export_state(t)
    rk, rs, rv, rb = export_state(ref)
    assert np.array_equal(gk, rk) and np.array_equal(gb, rb)
    assert np.array_equal(gv.view(np.uint32), rv.view(np.uint32))
    new_of = {}
    for p, nv in zip(parts, new_vals):
        new_of.update({int(k): v for k, v in zip(p, nv)})
    for out, fnd in seen:  # readers never run beside updaters: whole rows only
        assert fnd.all()
        for i in range(0, 4000, 97):
            k = int(keys[i])
            row = out[i].view(np.uint32)
            assert (np.array_equal(row, old_of[k].view(np.uint32))
                    or np.array_equal(row, new_of[k].view(np.uint32)))


def test_inserters_updaters_and_readers_on_their_own_streams():
    """Host threads, each with its own stream, take their roles and launch at
    the same time: two insert fresh keys (inserters, exclusive), two assign
    disjoint resident keys (updaters), two find. LFU scores add up and the
    key sets are disjoint, so the final state is order-free and must equal
    the serial application of the same calls. A find of a fresh key returns
    either a miss or exactly its inserted row (an inserter never overlaps a
    reader), and a find of an assigned key its old or its new row."""
    rng = np.random.default_rng(9650)
    dim = 8
    nb = 256
    t = hkv.Table(nb * 128, dim, hkv.LFU)
    ref = hkv.Table(nb * 128, dim, hkv.LFU)
    base = w.uniform_keys(rng, 8000, distinct=True)
    v0 = w.normal_values(rng, base.size, dim)
    for x in (t, ref):
        x.insert_or_assign(dev(base), dev(v0))
    torch.cuda.synchronize()
    fresh = [w.uniform_keys(rng, 4 * 1024, distinct=True) for _ in range(2)]
    fresh_vals = [w.normal_values(rng, f.size, dim) for f in fresh]
    upd = np.array_split(base[:4000], 2)
    upd_vals = [w.normal_values(rng, u.size, dim) for u in upd]
    row_of = {}
    for f, fv in zip(fresh, fresh_vals):
        row_of.update({int(k): fv[i].tobytes() for i, k in enumerate(f)})
    old_of = {int(k): v0[i].tobytes() for i, k in enumerate(base)}
    new_of = {}
    for u, uv in zip(upd, upd_vals):
        new_of.update({int(k): uv[i].tobytes() for i, k in enumerate(u)})
    errors, seen = [], []

    def inserter(f, fv):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for c in range(4):
                sl = slice(c * 1024, (c + 1) * 1024)
                t.insert_or_assign(dev(f[sl]), dev(fv[sl]))
        s.synchronize()

    def updater(u, uv):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for c in range(0, u.size, 500):
                t.assign(dev(u[c:c + 500]), dev(uv[c:c + 500]))
        s.synchronize()

    def reader(q):
        s = torch.cuda.Stream()
        for _ in range(6):
            with torch.cuda.stream(s):
                out, found, _ = t.find(dev(q))
            s.synchronize()
            seen.append((q, host(out).copy(), host(found).astype(bool)))

    q = np.concatenate([fresh[0][:600], fresh[1][:600], base[:1200]])
    threads = [threading.Thread(target=inserter, args=(f, fv)) for f, fv in zip(fresh, fresh_vals)]
    threads += [threading.Thread(target=updater, args=(u, uv)) for u, uv in zip(upd, upd_vals)]
    threads += [threading.Thread(target=reader, args=(q,)) for _ in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    for qq, out, found in seen:
        for k, row, f in zip(qq.tolist(), out, found):
            if k in row_of:
                if f and row.tobytes() != row_of[k]:
                    errors.append(("fresh", k))
            else:
                if not f or row.tobytes() not in (old_of[k], new_of.get(k, old_of[k])):
                    errors.append(("resident", k))
    assert not errors, errors[:5]
    # the same calls, one after another, on the reference table
    for f, fv in zip(fresh, fresh_vals):
        for c in range(4):
            sl = slice(c * 1024, (c + 1) * 1024)
            ref.insert_or_assign(dev(f[sl]), dev(fv[sl]))
    for u, uv in zip(upd, upd_vals):
        for c in range(0, u.size, 500):
            ref.assign(dev(u[c:c + 500]), dev(uv[c:c + 500]))
    torch.cuda.synchronize()
    gk, gs, gv, gb = export_state(t)
    rk, rs, rv, rb = export_state(ref)
    assert np.array_equal(gk, rk) and np.array_equal(gs, rs)
    assert np.array_equal(gv.view(np.uint32), rv.view(np.uint32))
    assert t.size() == base.size + sum(f.size for f in fresh)


def test_tables_upserting_at_once_on_their_own_streams():
    """Several tables take full-bucket upserts at the same time, one host
    thread and stream each, so their cooperative phase-I launches (phase I,
    reconcile and status with grid barriers between them) run side by side.
    No call may fail, and each table must end exactly as a twin fed the same
    batches serially: single-bucket results do not depend on the schedule."""
    rng = np.random.default_rng(4400)
    nb, dim, ntab, nbat, n = 64, 8, 4, 6, 20000
    z = w.Zipf(1.05, 60000)
    tabs = [hkv.Table(nb * 128, dim, hkv.LFU) for _ in range(ntab)]
    twins = [hkv.Table(nb * 128, dim, hkv.LFU) for _ in range(ntab)]
    batches = [[(dev(z.keys(rng, n)), dev(w.normal_values(rng, n, dim)))
                for _ in range(nbat)] for _ in range(ntab)]
    torch.cuda.synchronize()
    errors = []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for k, v in batches[i]:
                    tabs[i].insert_or_assign(k, v)
                tabs[i].sync()
        except Exception as e:  # reported below, on the test's thread
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(ntab)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for i in range(ntab):
        for k, v in batches[i]:
            twins[i].insert_or_assign(k, v)
        twins[i].sync()
        assert tabs[i].size() == tabs[i].capacity
        same_state(export_state(tabs[i]), export_state(twins[i]))
    for t in tabs + twins:
        t.close()
