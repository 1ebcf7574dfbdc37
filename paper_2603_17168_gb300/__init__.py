"""GB300-native cache-semantic GPU hash table (HierarchicalKV hot path,
arxiv 2603.17168): a thin ctypes binding of the C ABI in include/hkv.h.

Every step of find / insert_or_assign / assign / erase / size / export runs
in the CUDA library ``libhkv.so`` (built for sm_103a by
``python -m paper_2603_17168_gb300.build``). This module only marshals
arguments: it passes the device pointers of torch CUDA tensors and the
current torch stream. There is no CPU fallback: if the library is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhkv.so")

LRU, LFU, EPOCH_LRU, EPOCH_LFU, CUSTOM, CUSTOM_TS_FREQ = range(6)
ST_UPDATED, ST_INSERTED, ST_REJECTED = 1, 2, 3
COUNTER_NAMES = ("find_hit", "find_miss", "unique", "updated", "inserted", "evicted",
                 "rejected", "retries", "find_lines", "find_keys", "upd_lines", "upd_keys",
                 "ins_lines", "ins_score_lines", "ins_keys", "timeout_free", "timeout_evict",
                 "timeout_why", "timeout_key", "upd_claims", "upd_claim_lines")
KERNEL_NAMES = ("find", "dedup", "update", "insert", "reconcile", "status", "erase", "export",
                "size", "hostrows")
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "RESERVED_KEY", 3: "DUPLICATE_KEY", 4: "OOM",
                5: "CUDA", 6: "TIMEOUT", 7: "BUSY"}
SLOTS = 128
NOALLOC_MAX_KEYS = 65536

# Every C-ABI entry point declared in include/hkv.h with its ctypes signature.
_u64, _u32, _i32, _vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p
_P64 = ctypes.POINTER(ctypes.c_uint64)


class Options(ctypes.Structure):
    _fields_ = [("capacity", _u64), ("dim", _u32), ("policy", _i32), ("dual_bucket", _i32),
                ("deterministic", _i32), ("hbm_value_budget_bytes", _u64), ("slice_bytes", _u64)]


class BatchOp(ctypes.Structure):
    _fields_ = [("op", _i32), ("n", _u64), ("keys", _vp), ("values_in", _vp),
                ("values_out", _vp), ("flags", _vp), ("scores", _vp)]


OP_NONE, OP_FIND, OP_UPSERT = 0, 1, 2


class ServeRequest(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("table", _i32), ("op", _i32), ("n", _u64),
                ("keys", _vp), ("values_in", _vp), ("values_out", _vp), ("flags", _vp)]


class ServeResult(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("round", _u64)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("wall_s", "host_admit_s", "host_launch_s",
                                               "host_retire_s", "idle_s", "gpu_compute_s",
                                               "gpu_copy_out_s")] + \
               [(n, _u64) for n in ("requests", "direct_rounds", "batched_rounds",
                                    "loop_iterations", "h2d_bytes", "d2h_bytes")]

SIGNATURES = {
    "hkv_create": (_i32, [ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
    "hkv_destroy": (_i32, [_vp]),
    "hkv_capacity": (_u64, [_vp]),
    "hkv_num_buckets": (_u64, [_vp]),
    "hkv_dim": (_u32, [_vp]),
    "hkv_hbm_value_slots": (_u64, [_vp]),
    "hkv_find": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp, _vp]),
    "hkv_contains": (_i32, [_vp, _u64, _vp, _vp, _vp]),
    "hkv_insert_or_assign": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hkv_insert_or_assign_noalloc": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hkv_assign": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "hkv_erase": (_i32, [_vp, _u64, _vp, _vp]),
    "hkv_size": (_i32, [_vp, _P64, _vp]),
    "hkv_copy_state": (_i32, [_vp, _vp, _vp]),
    "hkv_export_batch": (_i32, [_vp, _u64, _u64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hkv_set_step": (_i32, [_vp, _u64]),
    "hkv_get_step": (_u64, [_vp]),
    "hkv_set_epoch": (_i32, [_vp, _u64]),
    "hkv_sync": (_i32, [_vp, _vp]),
    "hkv_read_counters": (_i32, [_vp, _P64, _vp]),
    "hkv_reset_counters": (_i32, [_vp, _vp]),
    "hkv_set_launch": (_i32, [_vp, _i32, _i32]),
    "hkv_set_value_vector": (_i32, [_vp, _i32]),
    "hkv_find_full_keys": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "hkv_host_memory_info": (_i32, [_vp, _P64, _P64, ctypes.POINTER(ctypes.c_int)]),
    "hkv_find_ptr": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "hkv_find_or_insert": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp, _vp]),
    "hkv_gather_rows": (_i32, [_vp, _u64, _u32, _vp, _vp]),
    "hkv_export_batch_if": (_i32, [_vp, _u64, _u64, _u64, _u64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hkv_set_l2_residency": (_i32, [_vp, _u64]),
    "hkv_set_concurrency": (_i32, [_vp, _i32]),
    "hkv_l2_residency": (_u64, [_vp]),
    "hkv_batch_create": (_i32, [_i32, ctypes.POINTER(_vp), _P64, ctypes.POINTER(_vp)]),
    "hkv_batch_run": (_i32, [_vp, ctypes.POINTER(BatchOp), _i32, _vp]),
    "hkv_batch_destroy": (_i32, [_vp]),
    "hkv_serve_create": (_i32, [ctypes.POINTER(_vp), _i32, _u64, _u64, _i32, ctypes.POINTER(_vp)]),
    "hkv_serve_hbm_bytes": (_u64, [_vp]),
    "hkv_serve_run": (_i32, [_vp, ctypes.POINTER(ServeRequest), _u64, _i32, _i32,
                             ctypes.POINTER(ServeResult), _vp]),
    "hkv_serve_destroy": (_i32, [_vp]),
    "hkv_serve_stats_get": (_i32, [_vp, ctypes.POINTER(ServeStats)]),
    "hkv_serve_profile": (_i32, [_vp, _i32]),
    "hkv_pipeline_create": (_i32, [_u64, _u32, _i32, ctypes.POINTER(_vp)]),
    "hkv_pipeline_find": (_i32, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "hkv_pipeline_insert_or_assign": (_i32, [_vp, _vp, _u64, _vp, _vp, _vp, _vp]),
    "hkv_pipeline_sync": (_i32, [_vp]),
    "hkv_pipeline_destroy": (_i32, [_vp]),
    "hkv_profile_enable": (_i32, [_vp, _i32]),
    "hkv_profile_read": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), _P64]),
    "hkv_measure_random_access": (_i32, [_u32, _i32, _u64, _u64, _i32,
                                          ctypes.POINTER(ctypes.c_double)]),
    "hkv_last_error": (ctypes.c_char_p, []),
}

_lib = None


class HKVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hkv error {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH):
    """Load libhkv.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_2603_17168_gb300.build` (nvcc, sm_103a)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise HKVError(rc, load_library().hkv_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _u64_types():
    import torch
    # 64-bit keys and scores: uint64 tensors, or int64 ones holding the same bits
    return (torch.uint64, torch.int64)


def _need(t, dtype, shape, name, pinned_ok=False):
    if t is None:
        return
    ok = t.dtype in dtype if isinstance(dtype, tuple) else t.dtype == dtype
    where = t.is_cuda or (pinned_ok and t.is_pinned())
    if not (where and ok and t.is_contiguous()):
        kind = "CUDA or page-locked host" if pinned_ok else "CUDA"
        raise ValueError(f"{name}: needs a contiguous {kind} tensor of {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")


class Table:
    """One hash table on the current CUDA device (see include/hkv.h)."""

    def __init__(self, capacity: int, dim: int, policy: int = LRU, dual_bucket: bool = False,
                 deterministic: bool = False, hbm_value_budget_bytes: int = 0,
                 slice_bytes: int = 0):
        L = load_library()
        o = Options(capacity, dim, policy, int(dual_bucket), int(deterministic),
                    hbm_value_budget_bytes, slice_bytes)
        h = ctypes.c_void_p()
        _check(L.hkv_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.dim = dim
        self.policy = policy
        self.dual_bucket = bool(dual_bucket)
        self.capacity = L.hkv_capacity(h)
        self.num_buckets = L.hkv_num_buckets(h)
        self.hbm_value_slots = L.hkv_hbm_value_slots(h)

    def close(self):
        if getattr(self, "_h", None):
            _check(load_library().hkv_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------- readers
    def find(self, keys, values_out=None, found=None, scores_out=None, stream=None):
        import torch
        n = keys.numel()
        if values_out is None:
            values_out = torch.zeros((n, self.dim), dtype=torch.float32, device=keys.device)
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        _need(keys, _u64_types(), (n,), "keys")
        _need(values_out, torch.float32, (n, self.dim), "values_out")
        _need(found, torch.uint8, (n,), "found")
        _need(scores_out, _u64_types(), (n,), "scores_out")
        _check(load_library().hkv_find(self._h, n, _ptr(keys), _ptr(values_out), _ptr(found),
                                       _ptr(scores_out), _stream(stream)))
        return values_out, found, scores_out

    def find_full_keys(self, keys, values_out=None, found=None, stream=None):
        """find without the digest line (the digest ablation,
        hkv_find_full_keys): same results as find()."""
        import torch
        n = keys.numel()
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        _need(keys, _u64_types(), (n,), "keys")
        _need(values_out, torch.float32, (n, self.dim), "values_out")
        _need(found, torch.uint8, (n,), "found")
        _check(load_library().hkv_find_full_keys(self._h, n, _ptr(keys), _ptr(values_out),
                                                 _ptr(found), _stream(stream)))
        return values_out, found

    def contains(self, keys, found=None, stream=None):
        import torch
        n = keys.numel()
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        _need(keys, _u64_types(), (n,), "keys")
        _need(found, torch.uint8, (n,), "found")
        _check(load_library().hkv_contains(self._h, n, _ptr(keys), _ptr(found), _stream(stream)))
        return found

    def find_ptr(self, keys, ptrs=None, found=None, stream=None):
        """find*: int64 tensor of value-row addresses (0 for misses), valid
        until the next mutating call; read rows with gather_rows."""
        import torch
        n = keys.numel()
        if ptrs is None:
            ptrs = torch.empty(n, dtype=torch.int64, device=keys.device)
        _need(keys, _u64_types(), (n,), "keys")
        _need(ptrs, torch.int64, (n,), "ptrs")
        _need(found, torch.uint8, (n,), "found")
        _check(load_library().hkv_find_ptr(self._h, n, _ptr(keys), _ptr(ptrs), _ptr(found),
                                           _stream(stream)))
        return ptrs

    def find_or_insert(self, keys, values_io, scores=None, found=None, stream=None):
        """Rows of values_io become the stored values of resident keys
        (missing keys are inserted with their rows first); returns found
        (1 = resident at call start) if given."""
        import torch
        n = keys.numel()
        _need(keys, _u64_types(), (n,), "keys")
        _need(values_io, torch.float32, (n, self.dim), "values_io")
        _need(scores, _u64_types(), (n,), "scores")
        _need(found, torch.uint8, (n,), "found")
        _check(load_library().hkv_find_or_insert(self._h, n, _ptr(keys), _ptr(values_io),
                                                 _ptr(scores), _ptr(found), _stream(stream)))
        return found

    def size(self, stream=None) -> int:
        out = ctypes.c_uint64()
        _check(load_library().hkv_size(self._h, ctypes.byref(out), _stream(stream)))
        return out.value

    def export_batch(self, slot_offset=0, n_slots=None, keys=None, values=None, scores=None,
                     slots=None, count=None, stream=None):
        """Occupied slots of [slot_offset, slot_offset + n_slots); returns
        (count tensor, keys, values, scores, slots), entries [:count] valid."""
        import torch
        if n_slots is None:
            n_slots = self.capacity - slot_offset
        dev = torch.device("cuda", torch.cuda.current_device())
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(load_library().hkv_export_batch(self._h, slot_offset, n_slots, _ptr(count),
                                               _ptr(keys), _ptr(values), _ptr(scores),
                                               _ptr(slots), _stream(stream)))
        return count, keys, values, scores, slots

    def export_batch_if(self, score_min, score_max, slot_offset=0, n_slots=None, keys=None,
                        values=None, scores=None, slots=None, count=None, stream=None):
        """export_batch restricted to scores in [score_min, score_max]."""
        import torch
        if n_slots is None:
            n_slots = self.capacity - slot_offset
        dev = torch.device("cuda", torch.cuda.current_device())
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(load_library().hkv_export_batch_if(
            self._h, slot_offset, n_slots, int(score_min), int(score_max), _ptr(count),
            _ptr(keys), _ptr(values), _ptr(scores), _ptr(slots), _stream(stream)))
        return count, keys, values, scores, slots

    # ------------------------------------------------------ updaters/inserters
    def insert_or_assign(self, keys, values, scores=None, status_out=None, evicted_keys=None,
                         evicted_scores=None, evicted_values=None, n_evicted=None, stream=None):
        import torch
        n = keys.numel()
        _need(keys, _u64_types(), (n,), "keys")
        # rows may also be page-locked host memory, read in place by the kernels
        _need(values, torch.float32, (n, self.dim), "values", pinned_ok=True)
        _need(scores, _u64_types(), (n,), "scores")
        _need(status_out, torch.uint8, (n,), "status_out")
        _need(evicted_keys, _u64_types(), None, "evicted_keys")
        _need(evicted_scores, _u64_types(), None, "evicted_scores")
        _need(evicted_values, torch.float32, None, "evicted_values")
        _need(n_evicted, _u64_types(), (1,), "n_evicted")
        for t in (evicted_keys, evicted_scores):
            if t is not None and t.numel() < n:
                raise ValueError("evicted outputs need room for n entries")
        if evicted_values is not None and evicted_values.numel() < n * self.dim:
            raise ValueError("evicted_values needs room for n rows")
        _check(load_library().hkv_insert_or_assign(
            self._h, n, _ptr(keys), _ptr(values), _ptr(scores), _ptr(status_out),
            _ptr(evicted_keys), _ptr(evicted_scores), _ptr(evicted_values), _ptr(n_evicted),
            _stream(stream)))
        return status_out

    def insert_or_assign_noalloc(self, keys, values, scores=None, status_out=None,
                                 evicted_keys=None, evicted_scores=None, n_evicted=None,
                                 stream=None):
        """insert_or_assign without any allocation inside the call (see
        hkv_insert_or_assign_noalloc in include/hkv.h): at most
        NOALLOC_MAX_KEYS keys, no evicted values."""
        import torch
        n = keys.numel()
        _need(keys, _u64_types(), (n,), "keys")
        # rows may also be page-locked host memory, read in place by the kernels
        _need(values, torch.float32, (n, self.dim), "values", pinned_ok=True)
        _need(scores, _u64_types(), (n,), "scores")
        _need(status_out, torch.uint8, (n,), "status_out")
        _need(evicted_keys, _u64_types(), None, "evicted_keys")
        _need(evicted_scores, _u64_types(), None, "evicted_scores")
        _need(n_evicted, _u64_types(), (1,), "n_evicted")
        _check(load_library().hkv_insert_or_assign_noalloc(
            self._h, n, _ptr(keys), _ptr(values), _ptr(scores), _ptr(status_out),
            _ptr(evicted_keys), _ptr(evicted_scores), _ptr(n_evicted), _stream(stream)))
        return status_out

    def assign(self, keys, values=None, scores=None, stream=None):
        import torch
        n = keys.numel()
        _need(keys, _u64_types(), (n,), "keys")
        # rows may also be page-locked host memory, read in place by the kernels
        _need(values, torch.float32, (n, self.dim), "values", pinned_ok=True)
        _need(scores, _u64_types(), (n,), "scores")
        _check(load_library().hkv_assign(self._h, n, _ptr(keys), _ptr(values), _ptr(scores),
                                         _stream(stream)))

    def erase(self, keys, stream=None):
        import torch
        _need(keys, _u64_types(), (keys.numel(),), "keys")
        _check(load_library().hkv_erase(self._h, keys.numel(), _ptr(keys), _stream(stream)))

    # ---------------------------------------------------------------- state
    def copy_state_from(self, src: "Table", stream=None):
        """Make this table a copy of `src` (same shape): see hkv_copy_state."""
        _check(load_library().hkv_copy_state(self.handle, src.handle, _stream(stream)))

    def set_step(self, step: int):
        _check(load_library().hkv_set_step(self._h, step))

    def get_step(self) -> int:
        return load_library().hkv_get_step(self._h)

    def set_epoch(self, epoch: int):
        _check(load_library().hkv_set_epoch(self._h, epoch))

    def sync(self, stream=None):
        _check(load_library().hkv_sync(self._h, _stream(stream)))

    def read_counters(self, stream=None) -> dict:
        arr = (ctypes.c_uint64 * len(COUNTER_NAMES))()
        _check(load_library().hkv_read_counters(self._h, arr, _stream(stream)))
        return dict(zip(COUNTER_NAMES, list(arr)))

    def reset_counters(self, stream=None):
        _check(load_library().hkv_reset_counters(self._h, _stream(stream)))

    def profile_enable(self, on: bool = True):
        _check(load_library().hkv_profile_enable(self._h, int(on)))

    def profile_read(self) -> dict:
        """{kernel: (total ms, launches)} since the last read."""
        ms = (ctypes.c_double * len(KERNEL_NAMES))()
        cnt = (ctypes.c_uint64 * len(KERNEL_NAMES))()
        _check(load_library().hkv_profile_read(self._h, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_NAMES) if cnt[i]}

    def set_launch(self, find_threads_per_key: int = 0, update_threads_per_key: int = 0):
        _check(load_library().hkv_set_launch(self._h, find_threads_per_key,
                                             update_threads_per_key))

    def host_memory_info(self) -> dict:
        """Host side of a tiered table: value bytes in host memory, the bytes
        of them huge pages backed at creation, one registered mapping or not
        (hkv_host_memory_info)."""
        hb, hu, one = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
        _check(load_library().hkv_host_memory_info(self._h, ctypes.byref(hb), ctypes.byref(hu),
                                                   ctypes.byref(one)))
        return {"host_bytes": hb.value, "huge_bytes": hu.value, "one_mapping": bool(one.value)}

    def set_value_vector(self, nbytes: int = 0):
        """Widest vector (16, 8 or 4 bytes; 0: default 16) of the value-row
        copies (hkv_set_value_vector)."""
        _check(load_library().hkv_set_value_vector(self._h, int(nbytes)))

    def set_concurrency(self, rw_lock: bool):
        """Triple-group rule (default) or a reader/writer lock (Exp 3e)."""
        _check(load_library().hkv_set_concurrency(self._h, 1 if rw_lock else 0))

    def set_l2_residency(self, digest_bytes: int):
        """Bytes of the digest array kept persisting in L2 (0: off)."""
        _check(load_library().hkv_set_l2_residency(self._h, int(digest_bytes)))

    @property
    def l2_residency(self) -> int:
        return int(load_library().hkv_l2_residency(self._h))


class Batch:
    """Batched multi-table rounds over a fixed set of tables (one slot each;
    see hkv_batch_run in include/hkv.h)."""

    def __init__(self, tables, max_keys):
        L = load_library()
        self.tables = list(tables)
        n = len(self.tables)
        arr = (_vp * n)(*[t.handle.value for t in self.tables])
        mk = (ctypes.c_uint64 * n)(*[int(m) for m in max_keys])
        h = ctypes.c_void_p()
        _check(L.hkv_batch_create(n, arr, mk, ctypes.byref(h)))
        self._h = h
        self.max_keys = list(max_keys)

    def close(self):
        if getattr(self, "_h", None):
            _check(load_library().hkv_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def make_ops(self, ops):
        """Pack a round's ops (see run) into the C array hkv_batch_run reads."""
        n = len(self.tables)
        arr = (BatchOp * n)()
        for i, o in enumerate(ops):
            if o is None:
                arr[i].op = OP_NONE
                continue
            keys = o["keys"]
            arr[i].op = o["op"]
            arr[i].n = int(o.get("n", keys.numel()))
            arr[i].keys = keys.data_ptr()
            vals = o.get("values")
            if o["op"] == OP_FIND:
                arr[i].values_out = vals.data_ptr()
            else:
                arr[i].values_in = vals.data_ptr()
            fl = o.get("flags")
            arr[i].flags = fl.data_ptr() if fl is not None else None
            sc = o.get("scores")
            arr[i].scores = sc.data_ptr() if sc is not None else None
        return arr

    def run_packed(self, arr, use_graph=True, stream=None):
        _check(load_library().hkv_batch_run(self._h, arr, int(use_graph), _stream(stream)))

    def run(self, ops, use_graph=True, stream=None):
        """ops: one entry per slot, None or a dict with keys op (OP_FIND /
        OP_UPSERT), keys, values (find: output rows; upsert: input rows),
        flags (found / status, optional for upsert), scores (optional), n
        (default keys.numel())."""
        n = len(self.tables)
        arr = (BatchOp * n)()
        for i, o in enumerate(ops):
            if o is None:
                arr[i].op = OP_NONE
                continue
            keys = o["keys"]
            cnt = int(o.get("n", keys.numel()))
            arr[i].op = o["op"]
            arr[i].n = cnt
            arr[i].keys = keys.data_ptr()
            vals = o.get("values")
            if o["op"] == OP_FIND:
                arr[i].values_out = vals.data_ptr()
            else:
                arr[i].values_in = vals.data_ptr()
            fl = o.get("flags")
            arr[i].flags = fl.data_ptr() if fl is not None else None
            sc = o.get("scores")
            arr[i].scores = sc.data_ptr() if sc is not None else None
        _check(load_library().hkv_batch_run(self._h, arr, int(use_graph), _stream(stream)))


def gather_rows(ptrs, dim, out, stream=None):
    """out[i] = the dim floats at address ptrs[i] (int64 device tensor, e.g.
    from Table.find_ptr); rows of zero addresses are left untouched."""
    _check(load_library().hkv_gather_rows(_ptr(ptrs), ptrs.numel(), int(dim), _ptr(out),
                                          _stream(stream)))
    return out


def measure_random_access(unit_bytes, write=False, buffer_bytes=8 << 30, accesses=64 << 20,
                          repeats=3):
    """Random accesses per second of `unit_bytes` units (8, 32 or 128) over a
    buffer far above L2 (see hkv_measure_random_access)."""
    out = ctypes.c_double()
    _check(load_library().hkv_measure_random_access(int(unit_bytes), int(bool(write)),
                                                     int(buffer_bytes), int(accesses),
                                                     int(repeats), ctypes.byref(out)))
    return out.value


class Pipeline:
    """Host-buffer pipeline (see hkv_pipeline_* in include/hkv.h): find and
    insert_or_assign on HOST tensors (page-locked for overlap), queued with
    their copies so that neighbouring operations' copies and kernels
    overlap. Results are in the host tensors after sync()."""

    def __init__(self, max_keys, max_dim, depth=3):
        h = ctypes.c_void_p()
        _check(load_library().hkv_pipeline_create(int(max_keys), int(max_dim), int(depth),
                                                   ctypes.byref(h)))
        self._h = h

    def find(self, table, keys, values, found=None, n=None):
        n = keys.numel() if n is None else int(n)
        _check(load_library().hkv_pipeline_find(self._h, table.handle, n, _ptr(keys),
                                                 _ptr(values), _ptr(found)))

    def insert_or_assign(self, table, keys, values, scores=None, status=None, n=None):
        n = keys.numel() if n is None else int(n)
        _check(load_library().hkv_pipeline_insert_or_assign(
            self._h, table.handle, n, _ptr(keys), _ptr(values), _ptr(scores), _ptr(status)))

    def sync(self):
        _check(load_library().hkv_pipeline_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _check(load_library().hkv_pipeline_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop with continuous batching (see hkv_serve_run in
    include/hkv.h). Requests are ServeRequest structs over pinned host
    buffers; run() replays them in real time and returns per-request
    (admit_s, done_s, round)."""

    def __init__(self, tables, ring_keys, hbm_budget_bytes=0, max_inflight=3):
        L = load_library()
        self.tables = list(tables)
        n = len(self.tables)
        arr = (_vp * n)(*[t.handle.value for t in self.tables])
        h = ctypes.c_void_p()
        _check(L.hkv_serve_create(arr, n, ring_keys, hbm_budget_bytes, max_inflight,
                                  ctypes.byref(h)))
        self._h = h
        self.hbm_bytes = L.hkv_serve_hbm_bytes(h)

    def close(self):
        if getattr(self, "_h", None):
            _check(load_library().hkv_serve_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, requests, batched=True, use_graph=True, stream=None):
        n = len(requests)
        res = (ServeResult * n)()
        _check(load_library().hkv_serve_run(self._h, requests, n, int(batched), int(use_graph),
                                            res, _stream(stream)))
        return res

    def profile(self, on: bool = True):
        """Time every round on the device in later runs (hkv_serve_profile)."""
        _check(load_library().hkv_serve_profile(self._h, int(on)))

    def stats(self) -> dict:
        """Where the last run() spent its time (hkv_serve_stats)."""
        st = ServeStats()
        _check(load_library().hkv_serve_stats_get(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServeStats._fields_}


def make_requests(items):
    """items: dicts with arrival_s, table, op, keys (pinned int64/uint64 CPU
    tensor), values (pinned float32 CPU tensor: input for upserts, output for
    finds), flags (pinned uint8 CPU tensor or None)."""
    arr = (ServeRequest * len(items))()
    for i, it in enumerate(items):
        r = arr[i]
        r.arrival_s = float(it["arrival_s"])
        r.table = int(it["table"])
        r.op = int(it["op"])
        r.n = int(it["keys"].numel())
        r.keys = it["keys"].data_ptr()
        if it["op"] == OP_FIND:
            r.values_out = it["values"].data_ptr()
        else:
            r.values_in = it["values"].data_ptr()
        fl = it.get("flags")
        r.flags = fl.data_ptr() if fl is not None else None
    return arr
