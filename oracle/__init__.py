"""CPU oracle of the HierarchicalKV hot path (arxiv 2603.17168), ctypes binding.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package; the library under
``paper_2603_17168_gb300`` never does. The arithmetic lives in
``hkv_oracle.c`` (plain single-threaded C, Algorithms 1-3 of the paper); this
module only compiles it and marshals numpy arrays.

Parity status of each function (pins are in tests/test_oracle_*.py):
  fmix64 / bucket / digest mapping  pinned (inverse permutation, avalanche,
                                    uniformity, first-eviction band)
  find / contains                   pinned (brute-force scan, Prop. 1 count)
  insert_or_assign, single bucket   pinned (closed-form top-S, permutation
                                    invariance, B = 1 top-k, Table 9 admission burst)
  insert_or_assign, dual bucket     pinned (Prop. 3 order statistic,
                                    first-eviction band of Table 11, invariants)
  assign / erase / export / load    pinned (brute-force model, round trip)
  score policies                    pinned (closed-form counts per policy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hkv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LRU, LFU, EPOCH_LRU, EPOCH_LFU, CUSTOM, CUSTOM_TS_FREQ = range(6)
ST_UPDATED, ST_INSERTED, ST_REJECTED = 1, 2, 3
OK, ERR_INVALID_ARG, ERR_RESERVED_KEY, ERR_DUPLICATE_KEY, ERR_OOM = range(5)
SLOTS = 128


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain gcc, -O2)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _u64p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u8p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f32p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        P64, P8, PF = ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_float)
        sig = {
            "ot_fmix64": (u64, [u64]),
            "ot_map_keys": (None, [u64, i32, u64, P64, P64, P64, P8]),
            "ot_create": (vp, [u64, u32, i32, i32]),
            "ot_destroy": (None, [vp]),
            "ot_set_step": (None, [vp, u64]),
            "ot_get_step": (u64, [vp]),
            "ot_set_epoch": (None, [vp, u64]),
            "ot_key_compares": (u64, [vp]),
            "ot_reset_key_compares": (None, [vp]),
            "ot_size": (u64, [vp]),
            "ot_bucket_count": (u32, [vp, u64]),
            "ot_find": (None, [vp, u64, P64, PF, P8, P64]),
            "ot_contains": (None, [vp, u64, P64, P8]),
            "ot_insert_or_assign": (i32, [vp, u64, P64, PF, P64, i32, P8, P64, P64, PF, P64]),
            "ot_insert_or_assign_topk": (i32, [vp, u64, P64, PF, P64, i32, P8, P64, P64, PF, P64]),
            "ot_assign": (i32, [vp, u64, P64, PF, P64]),
            "ot_find_or_insert": (i32, [vp, u64, P64, PF, P64, P8]),
            "ot_erase": (i32, [vp, u64, P64]),
            "ot_export": (u64, [vp, u64, P64, P64, PF, P64]),
            "ot_load": (i32, [vp, u64, P64, P64, PF, P64]),
            "ot_bucket_min": (i32, [vp, u64, P64, P64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def fmix64(keys: np.ndarray) -> np.ndarray:
    f = lib().ot_fmix64
    return np.array([f(int(k)) for k in np.asarray(keys, dtype=np.uint64)], dtype=np.uint64)


def map_keys(num_buckets: int, dual: bool, keys: np.ndarray):
    """(b1, b2, digest) per key, as the oracle maps them."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.size
    b1 = np.empty(n, np.uint64)
    b2 = np.empty(n, np.uint64)
    dg = np.empty(n, np.uint8)
    lib().ot_map_keys(num_buckets, int(dual), n, _u64p(keys), _u64p(b1), _u64p(b2), _u8p(dg))
    return b1, b2, dg


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code


class OracleTable:
    """One table of the oracle: ``num_buckets`` buckets of 128 slots."""

    def __init__(self, num_buckets: int, dim: int, policy: int = LRU, dual: bool = False):
        self.num_buckets, self.dim, self.policy, self.dual = num_buckets, dim, policy, dual
        self._h = lib().ot_create(num_buckets, dim, policy, int(dual))
        if not self._h:
            raise OracleError(ERR_INVALID_ARG)

    def close(self):
        if self._h:
            lib().ot_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def capacity(self) -> int:
        return self.num_buckets * SLOTS

    def set_step(self, s: int):
        lib().ot_set_step(self._h, s)

    @property
    def step(self) -> int:
        return lib().ot_get_step(self._h)

    def set_epoch(self, e: int):
        lib().ot_set_epoch(self._h, e)

    @property
    def key_compares(self) -> int:
        return lib().ot_key_compares(self._h)

    def reset_key_compares(self):
        lib().ot_reset_key_compares(self._h)

    def size(self) -> int:
        return lib().ot_size(self._h)

    def bucket_count(self, b: int) -> int:
        return lib().ot_bucket_count(self._h, b)

    def bucket_min(self, b: int):
        s, k = ctypes.c_uint64(), ctypes.c_uint64()
        if not lib().ot_bucket_min(self._h, b, ctypes.byref(s), ctypes.byref(k)):
            return None
        return s.value, k.value

    def find(self, keys, values_out=None):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = keys.size
        if values_out is None:
            values_out = np.zeros((n, self.dim), np.float32)
        found = np.zeros(n, np.uint8)
        scores = np.zeros(n, np.uint64)
        lib().ot_find(self._h, n, _u64p(keys), _f32p(values_out), _u8p(found), _u64p(scores))
        return values_out, found.astype(bool), scores

    def contains(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        found = np.zeros(keys.size, np.uint8)
        lib().ot_contains(self._h, keys.size, _u64p(keys), _u8p(found))
        return found.astype(bool)

    def _upsert(self, fn, keys, values, scores, deterministic):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = keys.size
        values = np.ascontiguousarray(values, dtype=np.float32).reshape(n, self.dim)
        scores = None if scores is None else np.ascontiguousarray(scores, dtype=np.uint64)
        status = np.zeros(n, np.uint8)
        ek = np.zeros(n, np.uint64)
        es = np.zeros(n, np.uint64)
        ev = np.zeros((n, self.dim), np.float32)
        ne = ctypes.c_uint64()
        rc = fn(self._h, n, _u64p(keys), _f32p(values), _u64p(scores), int(deterministic),
                _u8p(status), _u64p(ek), _u64p(es), _f32p(ev), ctypes.byref(ne))
        if rc:
            raise OracleError(rc)
        m = ne.value
        return status, ek[:m].copy(), es[:m].copy(), ev[:m].copy()

    def insert_or_assign(self, keys, values, scores=None, deterministic=False):
        """Returns (status[n], evicted_keys, evicted_scores, evicted_values)."""
        return self._upsert(lib().ot_insert_or_assign, keys, values, scores, deterministic)

    def find_or_insert(self, keys, values, scores=None):
        """find_or_insert of a batch: returns (rows, found). rows[i] is the
        key's value in the table afterwards, or values[i] if the table
        refused the key; found[i] = 1 iff it was resident at batch start."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = keys.size
        rows = np.ascontiguousarray(values, dtype=np.float32).reshape(n, self.dim).copy()
        scores = None if scores is None else np.ascontiguousarray(scores, dtype=np.uint64)
        found = np.zeros(n, np.uint8)
        rc = lib().ot_find_or_insert(self._h, n, _u64p(keys), _f32p(rows), _u64p(scores),
                                     _u8p(found))
        if rc:
            raise OracleError(rc)
        return rows, found

    def insert_or_assign_topk(self, keys, values, scores=None, deterministic=False):
        """Closed-form single-bucket formulation (per-bucket top-S)."""
        return self._upsert(lib().ot_insert_or_assign_topk, keys, values, scores, deterministic)

    def assign(self, keys, values, scores=None):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        values = np.ascontiguousarray(values, dtype=np.float32).reshape(keys.size, self.dim)
        scores = None if scores is None else np.ascontiguousarray(scores, dtype=np.uint64)
        rc = lib().ot_assign(self._h, keys.size, _u64p(keys), _f32p(values), _u64p(scores))
        if rc:
            raise OracleError(rc)

    def erase(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        rc = lib().ot_erase(self._h, keys.size, _u64p(keys))
        if rc:
            raise OracleError(rc)

    def export(self):
        """All entries: (keys, scores, values, buckets), sorted by key."""
        n = self.size()
        k = np.zeros(n, np.uint64)
        s = np.zeros(n, np.uint64)
        v = np.zeros((n, self.dim), np.float32)
        b = np.zeros(n, np.uint64)
        w = lib().ot_export(self._h, n, _u64p(k), _u64p(s), _f32p(v), _u64p(b))
        assert w == n
        o = np.argsort(k, kind="stable")
        return k[o], s[o], v[o], b[o]

    def load(self, keys, scores, values, buckets):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = keys.size
        scores = np.ascontiguousarray(scores, dtype=np.uint64)
        values = np.ascontiguousarray(values, dtype=np.float32).reshape(n, self.dim)
        buckets = np.ascontiguousarray(buckets, dtype=np.uint64)
        rc = lib().ot_load(self._h, n, _u64p(keys), _u64p(scores), _f32p(values), _u64p(buckets))
        if rc:
            raise OracleError(rc)
