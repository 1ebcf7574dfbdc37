"""Launch-shape autotuner for the probe kernels.

The probe kernels give a group of G lanes to each key (G in 1..32): each
lane scans 128/G digests of the key's line (the probe group width) and
copies 1/G of the value row, in vectors of V bytes (V in 4, 8, 16; the
widest the row addresses allow up to V). Small G packs more keys per warp
instruction (the kernels are issue-bound on hashing and compares); large G
copies wide value rows with fewer iterations per lane; narrow vectors cost
more instructions per row but are the only ones unaligned rows allow. The
best shape depends on the value width, the load factor and the batch size,
so it is measured, not guessed:

  find_tpk, vec_bytes  a joint search over (G, V), timed with find() over a
              sample of keys (a reader: the table is not modified); V is
              the one the find rows liked best, and applies to the update
              and insert phases too;
  update_tpk  timed through the update phase of assign() over keys that are
              absent from the table, so nothing is written (the probe
              alone: no row is copied, so V plays no part there).

Choices are cached per (GPU, dim, dual, policy, batch size class, load
factor class) in a JSON file (``$HKV_AUTOTUNE_CACHE``, default
``build/hkv_autotune.json`` under the repository root).
"""
from __future__ import annotations

import json
import os
import statistics

CANDIDATES = (1, 2, 4, 8, 16)
VECTORS = (16, 8, 4)
_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cache_path() -> str:
    return os.environ.get("HKV_AUTOTUNE_CACHE",
                          os.path.join(_ROOT, "build", "hkv_autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def cache_key(table, n: int, load: float) -> str:
    import torch
    name = torch.cuda.get_device_name()
    nclass = max(10, int(n).bit_length())
    return (f"{name}|dim={table.dim}|dual={int(table.dual_bucket)}|policy={table.policy}"
            f"|n=2^{nclass}|lambda={round(load, 1)}")


def _time(fn, repeats):
    import torch
    times = []
    for _ in range(repeats + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times[1:])


def tune(table, sample_keys, absent_keys=None, repeats=3, candidates=CANDIDATES,
         vectors=VECTORS, use_cache=True, apply=True):
    """Pick find threads-per-key and value-copy vector width jointly, and
    update threads-per-key, for `table` on this batch shape.

    sample_keys: a device tensor of keys shaped like the table's requests.
    absent_keys: keys that are not resident (default: sample_keys with bit 62
    flipped, keeping only those that contains() reports absent). assign()
    over them probes and writes nothing, though it advances the table step
    like any assign call.
    Returns {"find_tpk": G, "update_tpk": G, "vec_bytes": V, "find_ms": {...},
    "update_ms": {...}} with find_ms keyed "G/V".
    """
    import torch
    n = sample_keys.numel()
    load = table.size() / table.capacity
    key = cache_key(table, n, load)
    cache = _load() if use_cache else {}
    if key in cache and "vec_bytes" in cache[key]:
        choice = cache[key]
    else:
        out = torch.empty((n, table.dim), dtype=torch.float32, device=sample_keys.device)
        found = torch.empty(n, dtype=torch.uint8, device=sample_keys.device)
        if absent_keys is None:
            flipped = sample_keys ^ (1 << 62)
            absent_keys = flipped[table.contains(flipped) == 0].contiguous()
        find_ms, upd_ms = {}, {}
        for v in vectors:
            table.set_value_vector(v)
            for g in candidates:
                table.set_launch(find_threads_per_key=g)
                find_ms[f"{g}/{v}"] = _time(lambda: table.find(sample_keys, out, found), repeats)
        for g in candidates:
            table.set_launch(update_threads_per_key=g)
            upd_ms[g] = _time(lambda: table.assign(absent_keys), repeats)
        best = min(find_ms, key=find_ms.get)
        fg, fv = (int(x) for x in best.split("/"))
        choice = {"find_tpk": fg, "vec_bytes": fv,
                  "update_tpk": min(upd_ms, key=upd_ms.get),
                  "find_ms": find_ms, "update_ms": upd_ms}
        if use_cache:
            cache[key] = choice
            _save(cache)
    if apply:
        table.set_launch(find_threads_per_key=int(choice["find_tpk"]),
                         update_threads_per_key=int(choice["update_tpk"]))
        table.set_value_vector(int(choice["vec_bytes"]))
    return choice
