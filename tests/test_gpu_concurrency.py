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
