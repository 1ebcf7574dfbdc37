"""Cache-quality streams (Sec. 5, Exp 3c and Exp 4) on the GPU against the
oracle run on the same stream at small scale: per batch, contains() then
insert_or_assign of Zipf(0.99) keys, five capacities of keys in all.
Single-bucket tables are bit-exact, so the hit counts of every batch and
the final top-N retention must be identical; a concurrent dual-bucket table
must land within a narrow band of the sequential one."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host  # noqa: E402

NB = 128
CAP = NB * 128
BATCH = 2048
UNIVERSE = 1 << 20


def run_stream(policy, dual, seed):
    rng = np.random.default_rng(seed)
    z = w.Zipf(0.99, UNIVERSE)
    t = hkv.Table(CAP, 1, policy, dual_bucket=dual)
    o = oracle.OracleTable(NB, 1, policy, dual)
    g_hits, o_hits = [], []
    for b in range(5 * CAP // BATCH):
        keys = z.keys(rng, BATCH)
        vals = np.zeros((BATCH, 1), np.float32)
        sc = np.full(BATCH, b, np.uint64) if policy == hkv.CUSTOM else None
        t.set_epoch(b)
        o.set_epoch(b)
        g_hits.append(int(host(t.contains(dev(keys))).sum()))
        o_hits.append(int(o.contains(keys).sum()))
        t.insert_or_assign(dev(keys), dev(vals), None if sc is None else dev(sc))
        o.insert_or_assign(keys, vals, sc)
    gk = export_state(t)[0]
    ok = o.export()[0]
    top = w.rank_to_key(np.arange(1, CAP + 1, dtype=np.uint64))
    return (np.array(g_hits), np.array(o_hits), np.isin(top, gk).mean(), np.isin(top, ok).mean())


@pytest.mark.parametrize("policy", [hkv.LRU, hkv.LFU, hkv.CUSTOM, hkv.EPOCH_LFU])
def test_single_bucket_quality_identical(policy):
    gh, oh, gret, oret = run_stream(policy, False, 5100 + policy)
    assert np.array_equal(gh, oh), "per-batch hit counts differ"
    assert gret == oret


def test_dual_bucket_quality_in_band():
    gh, oh, gret, oret = run_stream(hkv.LFU, True, 5200)
    gm, om = gh[2 * len(gh) // 5:].sum(), oh[2 * len(oh) // 5:].sum()
    assert abs(gm - om) <= 0.005 * om, (gm, om)
    assert abs(gret - oret) <= 0.005, (gret, oret)
