"""hkv_copy_state: a table copied from another holds the same state (keys,
scores, values, buckets, step, epoch), answers every later call as the
source would, and restores a saved state after the source has moved on
(the snapshot the benchmark restores between timed runs, so that each run
starts at the load factor it names). Checked against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host, same_state  # noqa: E402


def _upsert(t, keys, vals):
    st = torch.empty(keys.size, dtype=torch.uint8, device="cuda")
    t.insert_or_assign(dev(keys), dev(vals), status_out=st)
    t.sync()
    return host(st)


@pytest.mark.parametrize("budget_slices", [None, 1])
def test_copy_then_restore_single_bucket(budget_slices):
    rng = np.random.default_rng(8800 + (budget_slices or 0))
    nb, dim = 64, 8
    slice_bytes = 16 * 128 * dim * 4
    budget = 0 if budget_slices is None else budget_slices * slice_bytes
    mk = lambda: hkv.Table(nb * 128, dim, hkv.LFU, hbm_value_budget_bytes=budget,  # noqa: E731
                           slice_bytes=slice_bytes)
    a, snap = mk(), mk()
    o = oracle.OracleTable(nb, dim, oracle.LFU)
    z = w.Zipf(1.05, 30000)
    for _ in range(3):
        k = z.keys(rng, 6000)
        v = w.normal_values(rng, k.size, dim)
        assert np.array_equal(_upsert(a, k, v), o.insert_or_assign(k, v)[0])
    a.set_epoch(7)
    snap.copy_state_from(a)
    torch.cuda.synchronize()
    saved = o.export()
    same_state(export_state(snap), saved)
    assert snap.get_step() == a.get_step() == o.step
    # the source moves on; the copy answers as the oracle at the snapshot
    k = z.keys(rng, 8000)
    v = w.normal_values(rng, k.size, dim)
    _upsert(a, k, v)
    a.erase(dev(saved[0][:500]))
    a.sync()
    q = np.concatenate([saved[0][:3000], z.keys(rng, 3000)])
    out, found, _ = snap.find(dev(q))
    ov, of, _ = o.find(q)
    torch.cuda.synchronize()
    assert np.array_equal(host(found).astype(bool), of)
    assert np.array_equal(host(out)[of].view(np.uint32), ov[of].view(np.uint32))
    # restore the source from the copy, then both take the same batch
    a.copy_state_from(snap)
    torch.cuda.synchronize()
    same_state(export_state(a), saved)
    assert a.get_step() == o.step
    k = z.keys(rng, 7000)
    v = w.normal_values(rng, k.size, dim)
    ost = o.insert_or_assign(k, v)[0]
    assert np.array_equal(_upsert(a, k, v), ost)
    assert np.array_equal(_upsert(snap, k, v), ost)
    same_state(export_state(a), o.export())
    same_state(export_state(snap), o.export())
    assert a.size() == snap.size() == o.size()


def test_copy_dual_bucket_keeps_buckets_and_occupancy():
    """Dual-bucket tables: the copy holds every key in the same bucket, and
    its occupancy counters (read by phase D1 of Algorithm 3) equal the
    source's, so a deterministic batch gives the same result on both."""
    rng = np.random.default_rng(8900)
    nb, dim = 128, 4
    a = hkv.Table(nb * 128, dim, hkv.LRU, dual_bucket=True, deterministic=True)
    b = hkv.Table(nb * 128, dim, hkv.LRU, dual_bucket=True, deterministic=True)
    o = oracle.OracleTable(nb, dim, oracle.LRU, True)
    for n in (9000, 5000, 4000):
        k = w.uniform_keys(rng, n, distinct=True)
        v = w.normal_values(rng, n, dim)
        st = torch.empty(n, dtype=torch.uint8, device="cuda")
        a.insert_or_assign(dev(k), dev(v), status_out=st)
        o.insert_or_assign(k, v, deterministic=True)
    b.copy_state_from(a)
    torch.cuda.synchronize()
    same_state(export_state(b), o.export())
    k = w.uniform_keys(rng, 6000, distinct=True)
    v = w.normal_values(rng, k.size, dim)
    ost = o.insert_or_assign(k, v, deterministic=True)[0]
    assert np.array_equal(_upsert(b, k, v), ost)
    assert np.array_equal(_upsert(a, k, v), ost)
    same_state(export_state(b), o.export())
    same_state(export_state(a), o.export())


def test_copy_refuses_other_shapes():
    a = hkv.Table(128 * 16, 4, hkv.LRU)
    for other in (hkv.Table(128 * 32, 4, hkv.LRU), hkv.Table(128 * 16, 8, hkv.LRU),
                  hkv.Table(128 * 16, 4, hkv.LFU), hkv.Table(128 * 16, 4, hkv.LRU, True)):
        with pytest.raises(hkv.HKVError) as e:
            other.copy_state_from(a)
        assert e.value.code == 1
    with pytest.raises(hkv.HKVError):
        a.copy_state_from(a)
