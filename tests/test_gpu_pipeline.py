"""Host-buffer pipeline (hkv_pipeline_*) against the device-buffer calls: the
same operations on twin tables, one set driven from host memory through the
pipeline and one through hkv_find / hkv_insert_or_assign on device buffers,
give identical found flags, rows, statuses and final table states, with
operations of several tables interleaved, page-locked and pageable host
buffers, and several pipeline depths. Rows of misses come back as zeros."""
import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host, same_state  # noqa: E402

DIMS = (32, 8, 3)
BUCKETS = (64, 32, 16)


def _host(a: np.ndarray, pinned: bool):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(a.copy())
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("depth,pinned,policy", [(3, True, hkv.LFU), (2, True, hkv.CUSTOM),
                                                 (4, False, hkv.LRU)])
def test_pipeline_matches_device_calls(depth, pinned, policy):
    rng = np.random.default_rng(8100 + depth)
    piped = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    plain = [hkv.Table(b * 128, d, policy) for b, d in zip(BUCKETS, DIMS)]
    max_keys = 5000
    pipe = hkv.Pipeline(max_keys, max(DIMS), depth)
    z = w.Zipf(1.05, 40000)
    pending = []
    for rnd in range(12):
        for ti, (tp, td) in enumerate(zip(piped, plain)):
            n = int(rng.integers(0, max_keys + 1)) if rnd % 4 else max_keys
            keys = z.keys(rng, n)
            if rng.random() < 0.5:
                kh = _host(keys, pinned)
                vh = torch.full((n, tp.dim), -7.0).pin_memory() if pinned else \
                    torch.full((n, tp.dim), -7.0)
                fh = torch.empty(n, dtype=torch.uint8)
                fh = fh.pin_memory() if pinned else fh
                pipe.find(tp, kh, vh, fh)
                vd = torch.zeros((max(n, 1), td.dim), device="cuda")
                fd = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                if n:
                    td.find(dev(keys), vd, fd)
                pending.append(("find", vh, fh, vd, fd, n))
            else:
                vals = w.normal_values(rng, n, tp.dim)
                sc = rng.integers(0, 1000, n, dtype=np.uint64) if policy == hkv.CUSTOM else None
                sh = torch.empty(n, dtype=torch.uint8)
                sh = sh.pin_memory() if pinned else sh
                pipe.insert_or_assign(tp, _host(keys, pinned), _host(vals, pinned),
                                      scores=None if sc is None else _host(sc, pinned), status=sh)
                sd = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
                if n:
                    td.insert_or_assign(dev(keys), dev(vals), None if sc is None else dev(sc),
                                        status_out=sd)
                pending.append(("upsert", sh, sd, n))
        if rnd % 3 == 2:  # several rounds in flight before each check
            pipe.sync()
            torch.cuda.synchronize()
            for e in pending:
                if e[0] == "find":
                    _, vh, fh, vd, fd, n = e
                    f = host(fd)[:n]
                    assert np.array_equal(fh.numpy(), f)
                    # hits carry the same rows bit for bit; misses are zeros
                    assert np.array_equal(vh.numpy().view(np.uint32), host(vd)[:n].view(np.uint32))
                else:
                    _, sh, sd, n = e
                    assert np.array_equal(sh.numpy(), host(sd)[:n])
            pending.clear()
    pipe.sync()
    for a, b in zip(piped, plain):
        a.sync()
        b.sync()
        same_state(export_state(a), export_state(b))
    pipe.close()


def test_pipeline_refuses_oversized_operations():
    t = hkv.Table(128 * 8, 16)
    pipe = hkv.Pipeline(100, 8, 2)
    keys = torch.arange(1, 11, dtype=torch.int64).pin_memory()
    vals = torch.zeros((10, 16)).pin_memory()
    with pytest.raises(hkv.HKVError):  # dim 16 > max_dim 8
        pipe.find(t, keys, vals)
    pipe2 = hkv.Pipeline(5, 16, 2)
    with pytest.raises(hkv.HKVError):  # 10 keys > max_keys 5
        pipe2.insert_or_assign(t, keys, vals)
    with pytest.raises(hkv.HKVError):
        hkv.Pipeline(100, 8, 1)  # depth below 2
    pipe.close()
    pipe2.close()


def test_pipeline_deterministic_dual_bit_exact():
    """Deterministic dual-bucket tables (ordered phase I) driven through the
    pipeline from page-locked buffers, with the rows of each batch's keys
    gathered after dedup, end in the same state, statuses and find results
    as the same batches through the device-buffer calls, bit for bit."""
    rng = np.random.default_rng(8200)
    nb, dim = 16, 8
    tp = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True, deterministic=True)
    td = hkv.Table(nb * 128, dim, hkv.LFU, dual_bucket=True, deterministic=True)
    pipe = hkv.Pipeline(3000, dim, 3)
    universe = 6 * nb * 128
    for rnd in range(6):
        n = 1500 + 200 * rnd
        keys = (rng.choice(universe, n, replace=False) + 1).astype(np.uint64)  # distinct
        vals = w.normal_values(rng, n, dim)
        sh = torch.empty(n, dtype=torch.uint8).pin_memory()
        pipe.insert_or_assign(tp, _host(keys, True), _host(vals, True), status=sh)
        sd = torch.empty(n, dtype=torch.uint8, device="cuda")
        td.insert_or_assign(dev(keys), dev(vals), status_out=sd)
        q = (rng.choice(universe, 1000, replace=False) + 1).astype(np.uint64)
        vh = torch.full((1000, dim), -7.0).pin_memory()
        fh = torch.empty(1000, dtype=torch.uint8).pin_memory()
        pipe.find(tp, _host(q, True), vh, fh)
        pipe.sync()
        torch.cuda.synchronize()
        assert np.array_equal(sh.numpy(), host(sd)), "statuses"
        vd = torch.zeros((1000, dim), device="cuda")
        fd = torch.empty(1000, dtype=torch.uint8, device="cuda")
        td.find(dev(q), vd, fd)
        torch.cuda.synchronize()
        assert np.array_equal(fh.numpy(), host(fd))
        assert np.array_equal(vh.numpy().view(np.uint32), host(vd).view(np.uint32))
    tp.sync()
    td.sync()
    same_state(export_state(tp), export_state(td))
    pipe.close()
