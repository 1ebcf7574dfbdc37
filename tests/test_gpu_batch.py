"""Batched multi-table rounds (hkv_batch_run) against plain per-table calls:
the same inputs through both paths give bit-identical results and table
states, round after round, with the graph replayed across rounds of
different sizes (including empty rounds) and tables of different value
widths."""
import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import NAN_BITS, dev, export_state, host, nan_filled, same_state  # noqa: E402

DIMS = (16, 32, 64, 8, 3, 128)
BUCKETS = (64, 128, 32, 256, 16, 32)


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("policy", [hkv.LRU, hkv.CUSTOM])
def test_batched_rounds_match_plain_calls(use_graph, policy):
    rng = np.random.default_rng(7000 + use_graph + 10 * policy)
    plain = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    batched = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    max_keys = [6000, 9000, 3000, 20000, 1500, 4000]
    batch = hkv.Batch(batched, max_keys)
    z = w.Zipf(1.05, 50000)
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
            keys = dev(z.keys(rng, n))
            if kind == "find":
                out_p = nan_filled(n, t.dim)
                fnd_p = torch.empty(n, dtype=torch.uint8, device="cuda")
                t.find(keys, out_p, fnd_p)
                out_b = nan_filled(max(n, 1), t.dim)
                fnd_b = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                ops.append(dict(op=hkv.OP_FIND, keys=keys, values=out_b, flags=fnd_b, n=n))
                expect.append(("find", out_p, fnd_p, out_b, fnd_b, n))
            else:
                vals = dev(w.normal_values(rng, n, t.dim))
                sc = dev(rng.integers(0, 1000, n, dtype=np.uint64)) if policy == hkv.CUSTOM else None
                st_p = torch.empty(n, dtype=torch.uint8, device="cuda")
                t.insert_or_assign(keys, vals, sc, st_p)
                st_b = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                ops.append(dict(op=hkv.OP_UPSERT, keys=keys, values=vals, flags=st_b, scores=sc,
                                n=n))
                expect.append(("upsert", st_p, st_b, n))
        batch.run(ops, use_graph=use_graph)
        torch.cuda.synchronize()
        for e in expect:
            if e is None:
                continue
            if e[0] == "find":
                _, out_p, fnd_p, out_b, fnd_b, n = e
                assert np.array_equal(host(fnd_p), host(fnd_b)[:n])
                assert np.array_equal(host(out_p).view(np.uint32), host(out_b)[:n].view(np.uint32))
            else:
                _, st_p, st_b, n = e
                assert np.array_equal(host(st_p), host(st_b)[:n])
    for a, b in zip(plain, batched):
        a.sync()
        b.sync()
        same_state(export_state(b), export_state(a))
        assert a.get_step() == b.get_step()
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
    assert NAN_BITS
