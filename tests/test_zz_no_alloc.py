"""hkv_insert_or_assign_noalloc: the upsert for callers that cannot allocate
device memory (their device memory is reserved up front by a framework
allocator, or the call sits on a latency-critical path that must not risk an
allocation's synchronisation or an out-of-memory failure). It must give the
same results as hkv_insert_or_assign, bit for bit, call after call, while
working in the library's fixed 5 MiB device scratch array instead of pool
memory. This file is collected last so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host, same_state  # noqa: E402


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _outputs(n):
    return (torch.empty(n, dtype=torch.uint8, device="cuda"),
            torch.empty(n, dtype=torch.int64, device="cuda"),
            torch.empty(n, dtype=torch.int64, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"))


def _evicted(ek, es, ne):
    m = int(ne.item())
    k, s = host(ek[:m]), host(es[:m])
    o = np.argsort(k, kind="stable")
    return k[o], s[o]


@pytest.mark.parametrize("policy", [hkv.LFU, hkv.CUSTOM])
def test_noalloc_upsert_matches_pooled_upsert(policy):
    lib = hkv.load_library()
    rng = np.random.default_rng(4242 + policy)
    nb, dim = 64, 16
    pooled = hkv.Table(nb * 128, dim, policy)
    fixed = hkv.Table(nb * 128, dim, policy)
    seed = w.uniform_keys(rng, 9000, distinct=True)
    seed_v = dev(w.normal_values(rng, seed.size, dim))
    seed_s = dev(rng.integers(0, 50, seed.size, dtype=np.uint64))
    pooled.insert_or_assign(dev(seed), seed_v, seed_s)
    fixed.insert_or_assign(dev(seed), seed_v, seed_s)
    z = w.Zipf(1.05, 40000)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row on the same shared scratch array
    for n in (30000, hkv.NOALLOC_MAX_KEYS):
        keys = dev(z.keys(rng, n))
        vals = dev(w.normal_values(rng, n, dim))
        scores = dev(rng.integers(0, 60, n, dtype=np.uint64))
        st_a, ek_a, es_a, ne_a = _outputs(n)
        pooled.insert_or_assign(keys, vals, scores, st_a, ek_a, es_a, None, ne_a)
        st_b, ek_b, es_b, ne_b = _outputs(n)
        rc = lib.hkv_insert_or_assign_noalloc(fixed.handle, n, _p(keys), _p(vals), _p(scores),
                                              _p(st_b), _p(ek_b), _p(es_b), _p(ne_b), stream)
        assert rc == 0, lib.hkv_last_error()
        pooled.sync()
        fixed.sync()
        assert np.array_equal(host(st_a), host(st_b)), "statuses differ"
        ka, sa = _evicted(ek_a, es_a, ne_a)
        kb, sb = _evicted(ek_b, es_b, ne_b)
        assert np.array_equal(ka, kb) and np.array_equal(sa, sb), "evicted sets differ"
        assert ka.size > 0
        same_state(export_state(fixed), export_state(pooled))
    assert fixed.get_step() == pooled.get_step()


def test_noalloc_refuses_batches_above_its_limit():
    lib = hkv.load_library()
    t = hkv.Table(128 * 16, 4, hkv.LRU)
    n = hkv.NOALLOC_MAX_KEYS + 1
    keys = torch.arange(1, n + 1, dtype=torch.int64, device="cuda")
    vals = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    rc = lib.hkv_insert_or_assign_noalloc(t.handle, n, _p(keys), _p(vals), None, None, None,
                                          None, None,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"HKV_NOALLOC_MAX_KEYS" in lib.hkv_last_error()
    assert t.size() == 0


def test_noalloc_dual_bucket_keeps_the_invariants_and_the_pooled_count():
    """Dual-bucket tables (the single-table benchmark's mode) under the
    no-alloc call: concurrent phase D1 is order-dependent, so the check is
    every structural invariant after each of two calls in a row, and a
    retained count within 0.1% of the pooled call's on a twin table."""
    import oracle
    from tests import invariants as inv

    lib = hkv.load_library()
    rng = np.random.default_rng(4300)
    nb, dim = 256, 8
    pooled = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True)
    fixed = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True)
    seed = w.uniform_keys(rng, int(0.9 * nb * 128), distinct=True)
    seed_v = dev(w.normal_values(rng, seed.size, dim))
    pooled.insert_or_assign(dev(seed), seed_v)
    fixed.insert_or_assign(dev(seed), seed_v)
    z = w.Zipf(1.05, 1 << 20)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in (20000, hkv.NOALLOC_MAX_KEYS):
        keys = dev(z.keys(rng, n))
        vals = dev(w.normal_values(rng, n, dim))
        st_a, ek_a, es_a, ne_a = _outputs(n)
        pooled.insert_or_assign(keys, vals, None, st_a, ek_a, es_a, None, ne_a)
        st_b, ek_b, es_b, ne_b = _outputs(n)
        rc = lib.hkv_insert_or_assign_noalloc(fixed.handle, n, _p(keys), _p(vals), None,
                                              _p(st_b), _p(ek_b), _p(es_b), _p(ne_b), stream)
        assert rc == 0, lib.hkv_last_error()
        pooled.sync()
        fixed.sync()
        gk, gs, gv, gb = export_state(fixed)
        b1, b2, _ = oracle.map_keys(nb, True, gk)
        inv.check_state(gk, gs, gb, nb, b1, b2, fixed.capacity)
        st = host(st_b)
        assert np.all((st >= 1) & (st <= 3))
        kb, _ = _evicted(ek_b, es_b, ne_b)
        assert not np.any(np.isin(kb, gk)), "an evicted key is still resident"
        ins = np.unique(host(keys)[st == hkv.ST_INSERTED])
        assert np.all(np.isin(ins, gk)), "an inserted key is not resident"
        a, b = pooled.size(), fixed.size()
        assert abs(a - b) <= 0.001 * a, (a, b)


def test_noalloc_refuses_deterministic_dual_bucket_tables():
    lib = hkv.load_library()
    t = hkv.Table(128 * 16, 4, hkv.LRU, dual_bucket=True, deterministic=True)
    keys = torch.arange(1, 101, dtype=torch.int64, device="cuda")
    vals = torch.zeros((100, 4), dtype=torch.float32, device="cuda")
    rc = lib.hkv_insert_or_assign_noalloc(t.handle, 100, _p(keys), _p(vals), None, None, None,
                                          None, None,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"deterministic dual-bucket" in lib.hkv_last_error()
    assert t.size() == 0
