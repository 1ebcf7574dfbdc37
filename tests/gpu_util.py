"""Helpers of the GPU parity tests: numpy <-> CUDA tensors (64-bit keys as
int64 bit patterns) and a full read-back of a table's state through
hkv_export_batch."""
from __future__ import annotations

import numpy as np

NAN_BITS = 0x7FC00ABC  # a NaN payload that no stored value has


def dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t) -> np.ndarray:
    import torch
    a = t.detach().cpu().numpy()
    if t.dtype == torch.int64:
        a = a.view(np.uint64)
    return a


def nan_filled(n, dim):
    import torch
    return torch.full((n, dim), 0, dtype=torch.int32, device="cuda").fill_(NAN_BITS).view(torch.float32)


def export_state(table, slot_offset=0, n_slots=None):
    """(keys, scores, values, buckets) of every occupied slot, sorted by key."""
    import torch
    if n_slots is None:
        n_slots = table.capacity - slot_offset
    k = torch.empty(n_slots, dtype=torch.int64, device="cuda")
    s = torch.empty(n_slots, dtype=torch.int64, device="cuda")
    v = torch.empty((n_slots, table.dim), dtype=torch.float32, device="cuda")
    g = torch.empty(n_slots, dtype=torch.int64, device="cuda")
    cnt, *_ = table.export_batch(slot_offset, n_slots, k, v, s, g)
    torch.cuda.synchronize()
    c = int(cnt.item())
    keys, scores, vals, slots = host(k[:c]), host(s[:c]), host(v[:c]), host(g[:c])
    o = np.argsort(keys, kind="stable")
    return keys[o], scores[o], vals[o], slots[o] // 128


def same_state(gpu_state, oracle_state, check_buckets=True):
    gk, gs, gv, gb = gpu_state
    ok, os_, ov, ob = oracle_state
    assert gk.size == ok.size, (gk.size, ok.size)
    assert np.array_equal(gk, ok), "resident key sets differ"
    assert np.array_equal(gs, os_), "scores differ"
    assert np.array_equal(gv.view(np.uint32), ov.view(np.uint32)), "values differ"
    if check_buckets:
        assert np.array_equal(gb, ob), "buckets differ"
