#!/usr/bin/env python
"""Throughput of the hash-table hot path on one GB300 (or N replicas).

Workload (the single-table configuration): one table per load factor
lambda in {0.50, 0.75, 0.90, 1.00}, each 2^26 slots (2^19 buckets x 128),
value dim 32 fp32, LFU scores, dual-bucket selection, pre-filled with
uniform keys over a 2^32-key universe; every step then runs, on each table,
one find and one insert_or_assign of 1,048,576 Zipf(1.05) keys over the same
universe through the plain one-batch-per-call path. A step is 8 calls and
8 Mi keys; value = keys processed / second (B-KV/s), summed over ranks.

`--impl reference` times the CPU oracle (oracle/, plain single-threaded C)
on a bounded, scaled sample of the same workload instead.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "find / insert_or_assign B-KV/s at λ 0.50–1.00 (% HBM roofline); served p50/p99"
UNIT = "B-KV/s"
LAMBDAS = (0.50, 0.75, 0.90, 1.00)
NB_LOG2 = 19
DIM = 32
BATCH = 1 << 20
UNIVERSE = 1 << 32
ALPHA = 1.05
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0


def single_workload(nb_log2=NB_LOG2, batch=BATCH, lambdas=LAMBDAS):
    """Name of the single-table workload at the given sizes (the headline
    configuration by default)."""
    lam = "/".join(f"{x:.2f}" for x in lambdas)
    n = f"2^{batch.bit_length() - 1}" if batch & (batch - 1) == 0 else str(batch)
    return (f"single table x{len(lambdas)} (lambda {lam}): 2^{nb_log2 + 7} slots "
            f"(2^{nb_log2} buckets x 128), dim {DIM} fp32, LFU, dual-bucket, uniform fill over "
            f"2^32, per step find + insert_or_assign of {n} Zipf(1.05) keys per table")


WORKLOAD = single_workload()


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--nb-log2", type=int, default=NB_LOG2, help="log2 buckets per table")
    p.add_argument("--batch", type=int, default=BATCH)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-depth", type=int, default=6, help="staging slots of the e2e pipeline")
    p.add_argument("--l2-residency", action="store_true",
                   help="keep each table's digest array persisting in L2 (hkv_set_l2_residency)")
    p.add_argument("--no-random-access", action="store_true",
                   help="skip the random-access ceiling measurement")
    p.add_argument("--find-tpk", type=int, default=0)
    p.add_argument("--update-tpk", type=int, default=0)
    p.add_argument("--workload", choices=("single", "multi", "serve", "tiered", "ordered",
                                          "quality", "concurrency", "apis"), default="single")
    p.add_argument("--quality-log2", type=int, default=27,
                   help="log2 slots of the cache-quality tables")
    p.add_argument("--tiered-shrink", type=int, default=0,
                   help="divide the tiered table and its HBM budget by 2^k (small runs)")
    p.add_argument("--serve-budget-gib", type=float, default=120.0)
    p.add_argument("--serve-pool", type=int, default=512)
    p.add_argument("--serve-peak-requests", type=int, default=4096)
    p.add_argument("--serve-seconds", type=float, default=3.0)
    p.add_argument("--serve-warm-seconds", type=float, default=0.5,
                   help="untimed run of each path at each offered load before its measured "
                        "run (the batched loop captures a graph per new combination of "
                        "busy tables, once)")
    p.add_argument("--no-served", action="store_true",
                   help="single-table workload: skip the short serving-loop record")
    p.add_argument("--served-seconds", type=float, default=2.0,
                   help="seconds per offered load of the serving record in the default run")
    p.add_argument("--multi-lambda", type=float, default=1.0)
    p.add_argument("--multi-shrink", type=int, default=0,
                   help="divide the multi-table slot counts by 2^k (small runs)")
    p.add_argument("--lambdas", type=str, default=",".join(str(x) for x in LAMBDAS),
                   help="comma-separated load factors (a subset, for profiling runs)")
    a = p.parse_args(argv)
    a.lambdas = tuple(float(x) for x in a.lambdas.split(","))
    return a


# ------------------------------------------------------------- distribution

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max_sum(ms: float, units: float, world: int, device=None):
    """Max of elapsed ms and sum of units over ranks (replicas only)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        self.dev = device_index
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def mark(self, name):
        self.marks.append((name, time.time()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        def active(x):
            return x.lower() in ("active", "0x1") or x.lower().startswith("active")
        win = [p for (t, p) in self.samples if t0 - 0.25 <= t <= t1 + 0.25]
        if not win:
            win = [p for (_, p) in self.samples]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        sm = [float(p[1]) for p in win if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in win if p[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for p in win for n, v in zip(names, p[5:9]) if active(v)})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(win),
                "power_w_max": max((float(p[3]) for p in win
                                    if p[3].replace(".", "").isdigit()), default=None)}


# ----------------------------------------------------------------- roofline

def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# Sources of the kernels the single-table workload launches and of the
# table layout they read: a committed traffic capture is valid while these
# are unchanged.
KERNEL_SOURCES = ("hkv_common.cuh", "hkv_find.cu", "hkv_internal.h", "hkv_table.cu",
                  "hkv_upsert.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_17168_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload_key):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken from the current kernel sources on this workload; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload_key, {}).get(kernel)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def kernel_bytes(kind: str, c: dict, n_calls: int, batch: int, dim: int) -> float:
    """Algorithmic bytes a kernel kind had to move, from the device counters.
    Coalesced streams count their exact bytes; each scattered scalar access
    counts one 32-byte sector; a digest line is 128 B, a bucket's (key, score)
    run 2 KiB, a value row 4*dim B (read and write counted separately)."""
    D = 4 * dim
    S = 32
    if kind == "find":
        return (n_calls * batch * 9 + 128 * c["find_lines"] + S * c["find_keys"]
                + 2 * D * c["find_hit"])
    u = c["unique"]
    uc = c.get("upd_claims", 0)
    if kind == "update":
        # probe + in-place update of residents, and the free-slot claims made
        # here: two occupancy counters read and one incremented, the key CAS,
        # digest, score and status writes, the 32-B digest sectors scanned,
        # the input row read and the value row written
        deferred = u - c["updated"] - uc
        return (u * (4 + 8 + 1 + S) + 128 * c["upd_lines"] + S * c["upd_keys"]
                + c["updated"] * (2 * D + 2 * S + S) + deferred * 8
                + S * c.get("upd_claim_lines", 0) + uc * (9 * S + 2 * D))
    if kind == "insert":
        ins = c["inserted"] - uc
        nm = ins + c["evicted"] + c["rejected"]
        # per search: the miss record, status and victim; one 2 KiB (key,
        # score) run per candidate bucket per try; the slot written
        return (nm * (4 * 4 + S + S) + 128 * c["ins_lines"] + 2048 * c["ins_score_lines"]
                + (ins + c["evicted"]) * (3 * S + 2 * D) + c["evicted"] * S)
    if kind == "dedup":
        return n_calls * batch * (8 + 4) + u * 2 * S
    if kind == "status":
        return n_calls * batch * (4 + 1 + S)
    if kind == "reconcile":
        return c["evicted"] * (16 + S)
    return 0.0


def kind_bytes(kind: str, launched: set, c: dict, n_calls: int, batch: int, dim: int) -> float:
    """Algorithmic bytes of one kernel kind's launches. On the plain upsert
    path one cooperative launch runs phase I, reconcile and status (profiled
    as insert; reconcile and status then have no launches of their own), or,
    after the host-row pass of tiered tables, reconcile and status (profiled
    as status): such a kind carries the bytes of every pass it ran."""
    b = kernel_bytes(kind, c, n_calls, batch, dim)
    if kind == "status" and "reconcile" not in launched:
        b += kernel_bytes("reconcile", c, n_calls, batch, dim)
    if kind == "insert" and "status" not in launched and "reconcile" not in launched:
        b += (kernel_bytes("reconcile", c, n_calls, batch, dim)
              + kernel_bytes("status", c, n_calls, batch, dim))
    return b


RANDOM_KINDS = ("line_reads", "sector_reads", "line_writes", "sector_writes")


def kernel_random_accesses(kind: str, c: dict, n_calls: int, batch: int, dim: int):
    """Scattered DRAM accesses of a probe kernel from the device counters,
    {line_reads, sector_reads, line_writes, sector_writes} (128-B lines,
    32-B sectors), plus the bytes it streams in order (batch keys, flags,
    output rows written by batch index). L2-resident scratch (the dedup
    table, the occupancy counters) is not counted."""
    D = 4 * dim
    uc = c.get("upd_claims", 0)
    if kind == "find":
        return {"line_reads": c["find_lines"] + c["find_hit"], "sector_reads": c["find_keys"],
                "line_writes": 0, "sector_writes": 0,
                "stream_bytes": n_calls * batch * 9 + D * c["find_hit"]}
    if kind == "update":
        u = c["unique"]
        # probe lines and key confirms; an update reads its input row and
        # its score sector and writes the value row and the score; a claim
        # reads its input row and the key sector (CAS) and writes the value
        # row and the key, score and digest sectors
        return {"line_reads": c["upd_lines"] + c["updated"] + uc,
                "sector_reads": c["upd_keys"] + c["updated"] + uc,
                "line_writes": c["updated"] + uc,
                "sector_writes": c["updated"] + 3 * uc,
                "stream_bytes": u * 13 + (u - c["updated"] - uc) * 8}
    return None


def measure_random_ceiling():
    """Random-access rates of this GPU's HBM (accesses/s) over an 8 GiB
    buffer: 128-B line and 32-B sector reads and writes."""
    import paper_2603_17168_gb300 as hkv
    return {"line_reads": hkv.measure_random_access(128),
            "sector_reads": hkv.measure_random_access(32),
            "line_writes": hkv.measure_random_access(128, write=True),
            "sector_writes": hkv.measure_random_access(32, write=True)}


# -------------------------------------------------------------------- ours

def fill_table(t, lam, gen, dim, batch_fill=1 << 20, max_batches=400):
    """Insert fresh uniform keys over the universe until the table holds
    lam * capacity keys (0.999 * capacity for lam >= 1). Batches that cannot
    overshoot (each adds at most batch_fill keys) run without a size check;
    the last one is cut to the keys still missing, so a table below the
    first-eviction load lands within a few keys of its target."""
    import torch
    from paper_2603_17168_gb300 import workloads as w
    cap = t.capacity
    target = lam * cap if lam < 1.0 else 0.999 * cap
    vals = torch.randn((batch_fill, dim), device="cuda", generator=gen)
    blind = max(0, int((target - t.size()) / batch_fill * 0.98))
    for b in range(max_batches):
        k = w.uniform_keys_torch(gen, batch_fill, UNIVERSE)
        if b >= blind:
            size = t.size()
            if size >= target:
                break
            need = int(target - size)
            if need < batch_fill and lam < 1.0:
                k = k[:max(need, 1)].contiguous()
        t.insert_or_assign(k, vals[:k.numel()])
    return t.size() / cap


def op_bytes(op: str, c: dict, n_calls: int, batch: int, dim: int) -> float:
    """Algorithmic bytes of one operation kind over n_calls batches: find is
    its kernel's bytes; insert_or_assign is the bytes of its update and
    insert kernels (probe, in-place update, claims, victim searches) plus each
    input key read and each status byte written once. The dedup pre-pass and
    the reconcile / status bookkeeping are not the method's work and are left
    out."""
    if op == "find":
        return kernel_bytes("find", c, n_calls, batch, dim)
    return (kernel_bytes("update", c, n_calls, batch, dim)
            + kernel_bytes("insert", c, n_calls, batch, dim) + n_calls * batch * (8 + 1))


SEG_STEPS = 3        # steps per timed segment; every table is restored before each
CONTROL_RUNS = 5     # runs of the uniform-key control per load factor (median)


def spread(xs):
    """(max - min) / mean of a list of positive numbers."""
    xs = [x for x in xs if x]
    return round((max(xs) - min(xs)) / (sum(xs) / len(xs)), 4) if xs else None


def run_ours(args):
    """The single-table workload. Tables are filled to just below their load
    factor, take the W warm-up steps, are topped up to the load factor with
    fresh uniform keys, and are then saved to device snapshots
    (hkv_copy_state). The K timed steps run in segments of SEG_STEPS steps;
    before each segment every table is restored from its snapshot, outside
    the timed brackets, so each segment starts at the load factor it names
    (the paper's median-of-runs methodology, Sec. 5.1). Two more passes
    repeat the same segments on the same restored states and batches: one
    with an event around every call (the per-lambda rates), one with the
    library's per-kernel events (kernel times and counters), kept apart
    because the kernel events lengthen every call; the uniform-key control
    runs CONTROL_RUNS times per table from the snapshot."""
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    nb = 1 << args.nb_log2
    batch = args.batch
    steps, warm = args.steps, args.warmup
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(2, rank))

    nvtx = torch.cuda.nvtx
    lambdas = args.lambdas
    ceiling = None if args.no_random_access else measure_random_ceiling()
    tables = []
    nvtx.range_push("fill")
    for lam in lambdas:
        t = hkv.Table(nb * 128, DIM, hkv.LFU, dual_bucket=True)
        t.set_launch(args.find_tpk, args.update_tpk)
        if args.l2_residency:
            t.set_l2_residency(nb * 128)
        # below the load factor by more than the warm-up steps add (each
        # Zipf batch brings about 0.4% of the capacity in new keys)
        pre = lam - min(0.2, 0.006 * warm + 0.01) if lam < 1.0 else lam
        fill_table(t, max(0.0, pre), gen, DIM)
        tables.append(t)
    nvtx.range_pop()

    z = w.Zipf(ALPHA, UNIVERSE)
    nbat = warm + steps
    fk = [w.zipf_keys_torch(gen, z, batch) for _ in range(nbat)]
    uk = [w.zipf_keys_torch(gen, z, batch) for _ in range(nbat)]
    uv = [torch.randn((batch, DIM), device=dev, generator=gen) for _ in range(nbat)]
    out_v = torch.empty((batch, DIM), device=dev)
    out_f = torch.empty(batch, dtype=torch.uint8, device=dev)
    out_s = torch.empty(batch, dtype=torch.uint8, device=dev)

    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in tables]
          for _ in range(nbat)]

    def step(i, per_op=False):
        for li, t in enumerate(tables):
            if per_op:
                ev[i][li][0].record()
            t.find(fk[i], out_v, out_f)
            if per_op:
                ev[i][li][1].record()
            t.insert_or_assign(uk[i], uv[i], status_out=out_s)
            if per_op:
                ev[i][li][2].record()

    nvtx.range_push("warmup")
    for i in range(warm):
        step(i)
    torch.cuda.synchronize()
    nvtx.range_pop()
    # top up to the load factor, then save every table's state
    lam_fill = [fill_table(t, lam, gen, DIM) for lam, t in zip(lambdas, tables)]
    snaps = []
    for t in tables:
        s = hkv.Table(nb * 128, DIM, hkv.LFU, dual_bucket=True)
        s.copy_state_from(t)
        snaps.append(s)
    torch.cuda.synchronize()

    def restore(which=None):
        for li, (t, s) in enumerate(zip(tables, snaps)):
            if which is None or li == which:
                t.copy_state_from(s)

    def lams():
        return [t.size() / t.capacity for t in tables]

    segments = []
    i = warm
    while i < warm + steps:
        segments.append(range(i, min(i + SEG_STEPS, warm + steps)))
        i += SEG_STEPS

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.6)

    # headline pass: the calls alone, no per-operation events or kernel
    # profiling in the stream; restores between segments, outside the timing
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms_local, lam_end = 0.0, [0.0] * len(tables)
    t_wall0 = time.time()
    nvtx.range_push("timed")
    for seg in segments:
        restore()
        barrier(world)
        torch.cuda.synchronize()
        e0.record()
        for i in seg:
            step(i)
        e1.record()
        e1.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        ms_local += e0.elapsed_time(e1)
        lam_end = [max(a, b) for a, b in zip(lam_end, lams())]
    nvtx.range_pop()
    t_wall1 = time.time()
    units_local = float(steps * len(tables) * 2 * batch)
    ms, units = reduce_max_sum(ms_local, units_local, world, dev)

    # per-operation pass: the same segments on the same restored states and
    # batches, with an event around every call (the per-lambda rates; the
    # library's kernel events stay off, since they lengthen every call)
    nvtx.range_push("per_op")
    for seg in segments:
        restore()
        for i in seg:
            step(i, per_op=True)
    torch.cuda.synchronize()
    nvtx.range_pop()
    op_ms = {i: [(ev[i][li][0].elapsed_time(ev[i][li][1]), ev[i][li][1].elapsed_time(ev[i][li][2]))
                 for li in range(len(tables))] for seg in segments for i in seg}
    # profiled pass: the same again with the library's kernel events (the
    # per-kernel device times) and its counters
    for t in tables:
        t.sync()
        t.reset_counters()
        t.profile_read()
        t.profile_enable(True)
    nvtx.range_push("profiled")
    for seg in segments:
        restore()
        for i in seg:
            step(i)
    torch.cuda.synchronize()
    nvtx.range_pop()
    for t in tables:
        t.profile_enable(False)
        t.sync()
    peak, peak_src = load_peak()

    per_lambda = []
    for li, (lam, t) in enumerate(zip(lambdas, tables)):
        f_seg = [len(seg) * batch / sum(op_ms[i][li][0] for i in seg) / 1e6 for seg in segments]
        u_seg = [len(seg) * batch / sum(op_ms[i][li][1] for i in seg) / 1e6 for seg in segments]
        f_ms = sum(op_ms[i][li][0] for seg in segments for i in seg)
        u_ms = sum(op_ms[i][li][1] for seg in segments for i in seg)
        c = t.read_counters()
        fb = op_bytes("find", c, steps, batch, DIM)
        ub = op_bytes("upsert", c, steps, batch, DIM)
        per_lambda.append({
            "lambda_target": lam, "lambda_start": round(lam_fill[li], 4),
            "lambda_end": round(lam_end[li], 4),
            "find_bkvs": round(statistics.median(f_seg), 4),
            "upsert_bkvs": round(statistics.median(u_seg), 4),
            "find_frac": round(fb / (f_ms * 1e6) / peak, 4),
            "upsert_frac": round(ub / (u_ms * 1e6) / peak, 4),
            "find_bytes_per_key": round(fb / (steps * batch), 1),
            "upsert_bytes_per_key": round(ub / (steps * batch), 1),
            "find_hit_rate": round(c["find_hit"] / max(1, c["find_hit"] + c["find_miss"]), 4),
            "upsert_unique": c["unique"], "updated": c["updated"], "inserted": c["inserted"],
            "evicted": c["evicted"], "rejected": c["rejected"], "retries": c["retries"],
            "_counters": c})

    # kernel-level roofline: device time per kernel kind from the library's
    # event brackets on the launching stream, bytes from the counters
    kinds = {}
    for li, t in enumerate(tables):
        prof = t.profile_read()
        c = per_lambda[li]["_counters"]
        per_lambda[li]["kernel_ms"] = {k: round(v[0], 4) for k, v in prof.items()}
        for kind, (kms, launches) in prof.items():
            e = kinds.setdefault(kind, {"ms": 0.0, "launches": 0, "bytes": 0.0, "ra": None})
            e["ms"] += kms
            e["launches"] += launches
            e["bytes"] += kind_bytes(kind, set(prof), c, steps, batch, DIM)
            ra = kernel_random_accesses(kind, c, steps, batch, DIM)
            if ra is not None:
                acc = e["ra"] or dict.fromkeys(ra, 0)
                e["ra"] = {k: acc[k] + ra[k] for k in ra}
    for kind, e in kinds.items():
        e["ra_frac"] = None
        if ceiling and e["ra"] and e["ms"] > 0:
            e["ra_bound_ms"] = 1e3 * (sum(e["ra"][k] / ceiling[k] for k in RANDOM_KINDS)
                                      + e["ra"]["stream_bytes"] / (peak * 1e9))
            e["ra_frac"] = e["ra_bound_ms"] / e["ms"]
    for kind, e in kinds.items():
        e["gbs"] = e["bytes"] / (e["ms"] * 1e6) if e["ms"] > 0 else None
        e["frac_measured"] = e["gbs"] / peak if e["gbs"] else None
        e["share"] = e["ms"] / sum(x["ms"] for x in kinds.values())
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    wkey = f"single_nb{args.nb_log2}_b{batch}_l{'-'.join(str(x) for x in lambdas)}"
    traffic = traffic_for(dom, wkey)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(d["gbs"], 1), "peak": peak,
                "unit": "GB/s", "frac": round(d["gbs"] / peak, 4),
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy, burst)",
                "frac_of_nominal_8tbs": round(d["gbs"] / NOMINAL_HBM_GBS, 4),
                "algorithmic_bytes_per_launch": round(d["bytes"] / d["launches"]),
                "avg_launch_ms": round(d["ms"] / d["launches"], 5),
                "traffic": traffic}
    if d.get("ra_frac") is not None:
        n_l = d["launches"]
        roofline["random_access"] = {
            "note": "the same kernel against the random-access rate of this GPU's HBM, "
                    "measured in this run (hkv_measure_random_access, 8 GiB buffer): each "
                    "scattered 128-B line or 32-B sector access per launch (device counters) "
                    "costed at the measured rate of its kind, plus the bytes streamed in order "
                    "at the copy peak; frac = that bound / the measured launch time",
            "ceiling": {k: round(v / 1e9, 2) for k, v in ceiling.items()},
            "ceiling_unit": "G accesses/s",
            "per_launch": {k: round(v / n_l) for k, v in d["ra"].items()},
            "bound_ms_per_launch": round(d["ra_bound_ms"] / n_l, 5),
            "frac": round(d["ra_frac"], 4)}
    gpu_launches = sum(e["launches"] for e in kinds.values())
    for e in per_lambda:
        e.pop("_counters")

    # uniform-key control per load factor (the paper's load-factor sweep
    # uses uniform keys, Sec. 5.2): from the snapshot, CONTROL_RUNS runs of
    # one find and one insert_or_assign, each batch half keys sampled
    # uniformly from the residents and half fresh uniform keys
    ctl_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)]
              for _ in range(CONTROL_RUNS)]
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    res_keys = torch.empty(nb * 128, dtype=torch.int64, device=dev)
    for li, t in enumerate(tables):
        restore(li)
        t.export_batch(0, nb * 128, res_keys, None, None, None, cnt)
        n_res = int(cnt.item())

        def control_batch():
            half = batch // 2
            pick = torch.randint(0, max(n_res, 1), (half,), device=dev, generator=gen)
            k = torch.cat([res_keys[pick], w.uniform_keys_torch(gen, batch - half, UNIVERSE)])
            return k[torch.randperm(batch, device=dev, generator=gen)].contiguous()

        ck = [(control_batch(), control_batch()) for _ in range(CONTROL_RUNS)]
        t.sync()
        t.reset_counters()
        lam_c = 0.0
        for r, (kf, ku) in enumerate(ck):
            restore(li)
            ctl_ev[r][0].record()
            t.find(kf, out_v, out_f)
            ctl_ev[r][1].record()
            t.insert_or_assign(ku, uv[r % nbat], status_out=out_s)
            ctl_ev[r][2].record()
            lam_c = max(lam_c, t.size() / t.capacity)
        torch.cuda.synchronize()
        c = t.read_counters()
        f_ms = [e[0].elapsed_time(e[1]) for e in ctl_ev]
        u_ms = [e[1].elapsed_time(e[2]) for e in ctl_ev]
        fb = op_bytes("find", c, CONTROL_RUNS, batch, DIM)
        ub = op_bytes("upsert", c, CONTROL_RUNS, batch, DIM)
        per_lambda[li]["uniform"] = {
            "find_bkvs": round(batch / statistics.median(f_ms) / 1e6, 4),
            "upsert_bkvs": round(batch / statistics.median(u_ms) / 1e6, 4),
            "find_frac": round(fb / (sum(f_ms) * 1e6) / peak, 4),
            "upsert_frac": round(ub / (sum(u_ms) * 1e6) / peak, 4),
            "find_hit_rate": round(c["find_hit"] / max(1, c["find_hit"] + c["find_miss"]), 4),
            "lambda_end": round(lam_c, 4),
            "evicted": c["evicted"], "rejected": c["rejected"]}
    del res_keys
    spreads = {"zipf": {op: spread([e[f"{op}_frac"] for e in per_lambda])
                        for op in ("find", "upsert")},
               "uniform": {op: spread([e["uniform"][f"{op}_frac"] for e in per_lambda])
                           for op in ("find", "upsert")},
               "definition": "(max - min) / mean over the load factors of each operation's "
                             "fraction of the measured copy peak"}

    # find* (pointer-returning find) on the snapshot states and the same
    # batches: value copy left out, as in the paper's find* numbers
    restore()
    ptrs = torch.empty(batch, dtype=torch.int64, device=dev)
    for li, t in enumerate(tables):
        t.find_ptr(fk[0], ptrs, out_f)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for i in range(warm, warm + steps):
            t.find_ptr(fk[i], ptrs, out_f)
        b.record()
        b.synchronize()
        per_lambda[li]["find_ptr_bkvs"] = round(steps * batch / a.elapsed_time(b) / 1e6, 4)

    # end to end through the public API: pinned host inputs copied in and
    # results copied out inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(tables, restore, segments, fk, uk, uv, batch, world, dev, args.e2e_depth)
    clk = clocks.summary(t_wall0, t_wall1)
    clocks.stop()

    result = None
    if rank == 0:
        value = units / (ms * 1e-3) / 1e9
        # digests, (key, score) pairs and fp32 values per slot; per table and
        # step the find's keys and rows out, the upsert's keys and rows in
        table_gib = nb * 128 * (1 + 16 + 4 * DIM) / 2**30
        step_gib = len(lambdas) * 2 * batch * (8 + 4 * DIM) / 2**30
        result = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": round(ms / steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded uniform fill + Zipf(1.05) request keys over 2^32, N(0,1) fp32 values)",
            "config": {"workload": single_workload(args.nb_log2, batch, lambdas),
                       "buckets_per_table": nb, "slots_per_table": nb * 128,
                       "dim": DIM, "batch": batch, "policy": "LFU", "dual_bucket": True,
                       "lambdas": list(lambdas), "parallelism": f"replicas x{world}",
                       "held_lambda": f"every table restored from a device snapshot "
                                      f"(hkv_copy_state) before each segment of {SEG_STEPS} "
                                      f"timed steps, outside the timed brackets; value = keys "
                                      f"of all {steps} steps / summed segment times",
                       "l2": f"no flush: each table is {table_gib:.1f} GiB and a step's "
                             f"inputs {step_gib:.2f} GiB, both far above the 129 MB L2",
                       "launch": {"find_tpk": args.find_tpk or "default",
                                  "update_tpk": args.update_tpk or "default"},
                       "l2_residency_bytes": [t.l2_residency for t in tables]},
            "per_lambda": per_lambda, "spread": spreads,
            "kernels": {k: {"ms": round(v["ms"], 4), "launches": v["launches"],
                            "share": round(v["share"], 4),
                            "gbs": round(v["gbs"], 1) if v["gbs"] else None,
                            "frac_measured": round(v["frac_measured"], 4) if v["frac_measured"] else None,
                            "frac_random_access": round(v["ra_frac"], 4) if v["ra_frac"] else None}
                        for k, v in sorted(kinds.items(), key=lambda kv: -kv[1]["ms"])},
            "roofline": roofline, "gpu_launches": gpu_launches, "clocks": clk, "e2e": e2e,
        }
    for t in tables + snaps:
        t.close()
    return result


def run_e2e(tables, restore, segments, fk, uk, uv, batch, world, dev, depth=3):
    """The same steps end to end through the library's host-buffer pipeline
    (hkv_pipeline_*): every step's keys and rows start in page-locked host
    memory and every result (find rows and flags, upsert statuses) ends
    there; the copies of neighbouring operations overlap the kernels. Keys,
    find rows and flags and statuses cross the link whole; an upsert sends
    the rows of its distinct keys only (gathered after dedup), so those
    bytes come from the tables' own counters over the timed steps. The
    segments and restores are those of the device-timed pass."""
    import torch
    import paper_2603_17168_gb300 as hkv
    pin = lambda x: x.cpu().pin_memory()  # noqa: E731
    steps = sum(len(seg) for seg in segments)
    first = segments[0][0]
    fk_h = {i: pin(fk[i]) for seg in segments for i in seg}
    uk_h = {i: pin(uk[i]) for seg in segments for i in seg}
    uv_h = {i: pin(uv[i]) for seg in segments for i in seg}
    # one result buffer per table: the pipeline writes them in call order
    ov_h = [torch.empty((batch, DIM)).pin_memory() for _ in tables]
    of_h = [torch.empty(batch, dtype=torch.uint8).pin_memory() for _ in tables]
    os_h = [torch.empty(batch, dtype=torch.uint8).pin_memory() for _ in tables]
    pipe = hkv.Pipeline(batch, DIM, depth=depth)
    h2d = d2h = 0

    def step(i, count):
        nonlocal h2d, d2h
        for j, t in enumerate(tables):
            pipe.find(t, fk_h[i], ov_h[j], of_h[j])
            pipe.insert_or_assign(t, uk_h[i], uv_h[i], status=os_h[j])
            if count:
                h2d += fk_h[i].numel() * 8 + uk_h[i].numel() * 8
                d2h += ov_h[j].numel() * 4 + of_h[j].numel() + os_h[j].numel()

    restore()
    step(first, False)   # the pipeline's first use, untimed
    pipe.sync()
    for t in tables:
        t.reset_counters()
    secs = 0.0
    for seg in segments:
        restore()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in seg:
            step(i, True)
        pipe.sync()
        secs += time.perf_counter() - t0
        barrier(world)
    pipe.close()
    for t in tables:
        h2d += t.read_counters()["unique"] * DIM * 4
    ms, units = reduce_max_sum(secs * 1e3, float(steps * len(tables) * 2 * batch), world, dev)
    return {"value": round(units / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps,
            "ms_per_step": round(ms / steps, 4),
            "path": "hkv_pipeline_find / hkv_pipeline_insert_or_assign on page-locked host "
                    f"buffers, {depth} staging slots; upsert rows of distinct keys only; "
                    "tables restored between segments as in the device-timed pass"}


# -------------------------------------------------------------- the oracle

SAMPLE_NB = 1 << 13        # 2^20 slots per table: 1/64 of the GPU tables
SAMPLE_OPS = 1 << 16       # keys per find and per upsert call: 1/16 of a batch


def oracle_tables(seed):
    import oracle
    from paper_2603_17168_gb300 import workloads as w
    rng = np.random.default_rng(seed)
    tabs = []
    for lam in LAMBDAS:
        t = oracle.OracleTable(SAMPLE_NB, DIM, oracle.LFU, True)
        cap = t.capacity
        target = lam * cap if lam < 1.0 else 0.999 * cap
        vals = w.normal_values(rng, 1 << 16, DIM)
        for _ in range(200):
            size = t.size()
            if size >= target:
                break
            n = int(min(1 << 16, max(1, target - size))) if lam < 1.0 else 1 << 16
            t.insert_or_assign(w.uniform_keys(rng, n, universe=UNIVERSE), vals[:n])
        tabs.append(t)
    return tabs, rng


def _step_inputs(step_seed, z):
    """One step's find keys, upsert keys and upsert rows of the oracle sample
    (a seeded draw, so that every process draws the same ones)."""
    from paper_2603_17168_gb300 import workloads as w
    rng = np.random.default_rng(step_seed)
    return z.keys(rng, SAMPLE_OPS), z.keys(rng, SAMPLE_OPS), w.normal_values(rng, SAMPLE_OPS, DIM)


_FIND_WORKER = {}


def _find_worker_init(seed):
    from paper_2603_17168_gb300 import workloads as w
    _FIND_WORKER["tabs"], _ = oracle_tables(seed)
    _FIND_WORKER["z"] = w.Zipf(ALPHA, UNIVERSE)


def _find_worker(task):
    """One process's share of a step's finds on its own copy of the sample
    tables (built from the same seed, so the same state); returns seconds."""
    step_seed, part, parts = task
    fk, _, _ = _step_inputs(step_seed, _FIND_WORKER["z"])
    chunk = fk[part * fk.size // parts:(part + 1) * fk.size // parts]
    t0 = time.perf_counter()
    for t in _FIND_WORKER["tabs"]:
        t.find(chunk)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleBaseline:
    """The oracle timed on the host cores, with threads where the semantics
    allow: a step's find over every core (one process per core, each with its
    own copy of the sample tables; a step's find time is its slowest
    process's), its dual-bucket insert_or_assign on one core (Algorithm 3 is
    order-dependent). Like the GPU pass, every step starts from the tables'
    state after filling: the upsert's tables are reloaded from a saved export
    after each step, outside the timing."""

    def __init__(self, seed):
        import multiprocessing as mp
        import concurrent.futures as cf
        from paper_2603_17168_gb300 import workloads as w
        self.cores = host_cores()
        # spawn, not fork: a forked child of a process that has used the GPU hangs
        self.pool = cf.ProcessPoolExecutor(self.cores, mp_context=mp.get_context("spawn"),
                                           initializer=_find_worker_init, initargs=(seed,))
        warm = [self.pool.submit(_find_worker, (1, p, self.cores)) for p in range(self.cores)]
        self.tabs, _ = oracle_tables(seed)
        self.saved = [t.export() for t in self.tabs]
        self.z = w.Zipf(ALPHA, UNIVERSE)
        for f in warm:
            f.result()

    def reload(self):
        import oracle
        for i, (t, st) in enumerate(zip(self.tabs, self.saved)):
            fresh = oracle.OracleTable(t.num_buckets, t.dim, t.policy, t.dual)
            fresh.load(*st)
            t.close()
            self.tabs[i] = fresh

    def step(self, step_seed):
        """(find seconds, upsert seconds, keys) of one step."""
        parts = self.cores
        fut = [self.pool.submit(_find_worker, (step_seed, p, parts)) for p in range(parts)]
        _, uk, uv = _step_inputs(step_seed, self.z)
        f_s = max(f.result() for f in fut)
        t0 = time.perf_counter()
        for t in self.tabs:
            t.insert_or_assign(uk, uv)
        u_s = time.perf_counter() - t0
        self.reload()
        return f_s, u_s, 2 * SAMPLE_OPS * len(self.tabs)

    def close(self):
        self.pool.shutdown()
        for t in self.tabs:
            t.close()


ORACLE_SAMPLE = (f"oracle (plain C) on 4 dual-bucket LFU tables of 2^20 slots (1/64 scale) at "
                 f"lambda 0.50/0.75/0.90/1.00, per step one find and one insert_or_assign of "
                 f"{SAMPLE_OPS} Zipf(1.05) keys each; find split over one process per host core, "
                 f"insert_or_assign on one core (order-dependent dual-bucket semantics); every "
                 f"step from the filled state; fill time excluded")


def tiny_whole_run_seconds():
    """The tiny configuration run whole by the oracle on one core: 512
    buckets x 128, dim 8, LRU, deterministic single-bucket, 16 batches of
    4,096 distinct uniform keys, then 4,096 finds (2,048 resident keys and
    2,048 fresh ones)."""
    import oracle
    from paper_2603_17168_gb300 import workloads as w
    rng = np.random.default_rng(w.seed_for(1))
    batches = [w.uniform_keys(rng, 4096, distinct=True) for _ in range(16)]
    vals = [w.normal_values(rng, 4096, 8) for _ in range(16)]
    t0 = time.perf_counter()
    t = oracle.OracleTable(512, 8, oracle.LRU)
    for k, v in zip(batches, vals):
        t.insert_or_assign(k, v, deterministic=True)
    res = t.export()[0]
    q = np.concatenate([rng.choice(res, 2048, replace=False), w.uniform_keys(rng, 2048)])
    t.find(q)
    secs = time.perf_counter() - t0
    t.close()
    return secs


def time_oracle(steps, warmup=1):
    from paper_2603_17168_gb300 import workloads as w
    base = OracleBaseline(w.seed_for(2, 99))
    try:
        for i in range(warmup):
            base.step(w.seed_for(2, 1000 + i))
        f_s = u_s = units = 0
        for i in range(steps):
            a, b, u = base.step(w.seed_for(2, 2000 + i))
            f_s += a
            u_s += b
            units += u
    finally:
        base.close()
    secs = f_s + u_s
    return {"value": round(units / secs / 1e9, 6), "unit": UNIT, "cores": base.cores,
            "kind": "oracle", "secs": secs,
            "find_bkvs": round(units / 2 / f_s / 1e9, 6),
            "upsert_bkvs": round(units / 2 / u_s / 1e9, 6),
            "sample": ORACLE_SAMPLE + f", {steps} timed steps ({secs:.1f} s of timed work)"}


def cpu_baseline(steps=24):
    r = time_oracle(steps)
    r.pop("secs")
    r["cfg1_s"] = round(tiny_whole_run_seconds(), 4)
    r["cfg1_note"] = "the tiny configuration's whole run (16 upsert batches and the finds), 1 core"
    return r


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    r = time_oracle(args.steps, args.warmup)
    secs = r.pop("secs")
    value = r["value"]
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle sample, see cpu_baseline)"},
            "cpu_baseline": r,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ----------------------------------------------------- multi-table workload

MULTI_WORKLOAD = ("8 tables of 2^22-2^25 slots, dims {16, 32, 64, 64, 128, 128, 256, 8} fp32, LRU, "
                  "single-bucket, pre-filled with uniform keys; per round and table a batch of "
                  "lognormal size (median 32K, sigma 1, clipped to 1K-512K) of Zipf(1.05) keys "
                  "over 2^32, find w.p. 0.8 else insert_or_assign")


def run_multi(args):
    """Batched multi-table rounds vs plain per-table calls on the same rounds."""
    import ctypes

    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import autotune
    from paper_2603_17168_gb300 import workloads as w

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(3, rank))
    rng = np.random.default_rng(w.seed_for(3, 100 + rank))
    maxn, pools = 524288, 3
    shrink = args.multi_shrink
    tables = []
    for slots, dim in zip(w.MULTI_SLOTS, w.MULTI_DIMS):
        t = hkv.Table(slots >> shrink, dim, hkv.LRU)
        fill_table(t, args.multi_lambda, gen, dim)
        tables.append(t)
    z = w.Zipf(ALPHA, UNIVERSE)
    pk = [[w.zipf_keys_torch(gen, z, maxn) for _ in range(pools)] for _ in tables]
    pv = [[torch.randn((maxn, t.dim), device=dev, generator=gen) for _ in range(pools)]
          for t in tables]
    outs = [torch.empty((maxn, t.dim), device=dev) for t in tables]
    flags = [torch.empty(maxn, dtype=torch.uint8, device=dev) for _ in tables]
    tuned = {}
    for i, t in enumerate(tables):
        c = autotune.tune(t, pk[i][0][:32768].contiguous())
        tuned[f"dim{t.dim}_slot{i}"] = {"find_tpk": c["find_tpk"], "update_tpk": c["update_tpk"]}
    batch = hkv.Batch(tables, [maxn] * len(tables))
    L = hkv.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    nround = args.warmup + args.steps
    rounds = []
    for r in range(nround):
        ops = []
        for i, t in enumerate(tables):
            n = int(np.clip(np.rint(np.exp(np.log(32768) + rng.standard_normal())), 1024, maxn))
            op = hkv.OP_FIND if rng.random() < 0.8 else hkv.OP_UPSERT
            p = r % pools
            off = int(rng.integers(0, maxn - n + 1))
            keys = pk[i][p][off:off + n]
            vals = outs[i][:n] if op == hkv.OP_FIND else pv[i][p][off:off + n]
            ops.append(dict(op=op, keys=keys, values=vals, flags=flags[i][:n], n=n))
        rounds.append(ops)
    keys_timed = sum(o["n"] for ops in rounds[args.warmup:] for o in ops)
    packed = [batch.make_ops(ops) for ops in rounds]
    plain_args = []
    for ops in rounds:
        calls = []
        for t, o in zip(tables, ops):
            kp, vp, fp = (ctypes.c_void_p(o["keys"].data_ptr()), ctypes.c_void_p(o["values"].data_ptr()),
                          ctypes.c_void_p(o["flags"].data_ptr()))
            if o["op"] == hkv.OP_FIND:
                calls.append((L.hkv_find, (t.handle, o["n"], kp, vp, fp, None, stream)))
            else:
                calls.append((L.hkv_insert_or_assign,
                              (t.handle, o["n"], kp, vp, None, fp, None, None, None, None, stream)))
        plain_args.append(calls)

    def plain(r):
        for fn, a in plain_args[r]:
            fn(*a)

    def graph(r):
        batch.run_packed(packed[r], True)

    def direct(r):
        batch.run_packed(packed[r], False)

    res = {}
    for name, fn in (("plain", plain), ("graph", graph), ("multistream", direct)):
        for r in range(args.warmup):
            fn(r)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record()
        for r in range(args.warmup, nround):
            fn(r)
        e1.record()
        host_ms = (time.perf_counter() - h0) * 1e3
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ms, units = reduce_max_sum(ms, float(keys_timed), world, dev)
        res[name] = {"bkvs": round(units / (ms * 1e-3) / 1e9, 4),
                     "ms_per_round": round(ms / args.steps, 4),
                     "host_issue_ms_per_round": round(host_ms / args.steps, 4)}
    for t in tables:
        t.sync()
    batch.close()
    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": res["graph"]["bkvs"], "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": res["graph"]["ms_per_round"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
               "config": {"workload": MULTI_WORKLOAD, "lambda": args.multi_lambda,
                          "slots_shift": shrink, "rounds_timed": args.steps,
                          "keys_per_round_mean": round(keys_timed / args.steps),
                          "step": "one round: 8 tables, one operation each"},
               "paths": res, "speedup_graph_vs_plain": round(res["graph"]["bkvs"] / res["plain"]["bkvs"], 3),
               "autotune": tuned}
    for t in tables:
        t.close()
    return out


# ------------------------------------------------------------ tiered table

TIERED_WORKLOAD = ("tiered: one table of 2^28 slots, dim 128 fp32 (128 GiB of values) with a 48 GiB "
                   "HBM value budget and the rest in pinned mapped host memory, TS_FREQ scores "
                   "(timestamp = batch number), pre-filled to lambda 1.0; per step find then "
                   "insert_or_assign of the same 2^20 Zipf(0.99) keys over 2^34")


def run_tiered(args):
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(4, rank))
    sh = args.tiered_shrink
    slots, dim = w.TIERED["slots"] >> sh, w.TIERED["dim"]
    budget = w.TIERED["hbm_value_bytes"] >> sh
    t0 = time.time()
    t = hkv.Table(slots, dim, hkv.CUSTOM_TS_FREQ, hbm_value_budget_bytes=budget)
    create_s = time.time() - t0
    host_mem = t.host_memory_info()
    batch = args.batch
    t.set_epoch(1)
    t1 = time.time()
    lam = fill_table(t, 1.0, gen, dim)
    fill_s = time.time() - t1
    z = w.Zipf(w.TIERED["zipf_alpha"], w.TIERED["universe"])
    nbat = args.warmup + args.steps
    keys = [w.zipf_keys_torch(gen, z, batch) for _ in range(nbat)]
    vals = [torch.randn((batch, dim), device=dev, generator=gen) for _ in range(nbat)]
    out = torch.empty((batch, dim), device=dev)
    found = torch.empty(batch, dtype=torch.uint8, device=dev)
    st = torch.empty(batch, dtype=torch.uint8, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nbat)]

    def step(i):
        t.set_epoch(2 + i)
        ev[i][0].record()
        t.find(keys[i], out, found)
        ev[i][1].record()
        t.insert_or_assign(keys[i], vals[i], status_out=st)
        ev[i][2].record()

    if args.find_tpk or args.update_tpk:
        t.set_launch(args.find_tpk, args.update_tpk)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    t.reset_counters()
    # the library's kernel events stay on in the timed pass: a step takes
    # milliseconds, against microseconds of event recording
    t.sync()
    t.profile_read()
    t.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.warmup, nbat):
        step(i)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    t.profile_enable(False)
    t.sync()
    kernel_ms = {k: round(v[0] / args.steps, 3) for k, v in t.profile_read().items()}
    c = t.read_counters()
    f_ms = sum(ev[i][0].elapsed_time(ev[i][1]) for i in range(args.warmup, nbat))
    u_ms = sum(ev[i][1].elapsed_time(ev[i][2]) for i in range(args.warmup, nbat))
    attempted = c["inserted"] + c["evicted"] + c["rejected"]
    # find* (value-row addresses, no copy: the paper's hybrid headline) and
    # find* followed by a gather of the rows, over the same batches on the
    # final state
    ptrs = torch.empty(batch, dtype=torch.int64, device=dev)
    fp = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t.find_ptr(keys[0], ptrs, found)
    fp[0].record()
    for i in range(args.warmup, nbat):
        t.find_ptr(keys[i], ptrs, found)
    fp[1].record()
    for i in range(args.warmup, nbat):
        t.find_ptr(keys[i], ptrs, found)
        hkv.gather_rows(ptrs, dim, out)
    fp[2].record()
    fp[2].synchronize()
    find_ptr_bkvs = args.steps * batch / fp[0].elapsed_time(fp[1]) / 1e6
    find_ptr_gather_bkvs = args.steps * batch / fp[1].elapsed_time(fp[2]) / 1e6

    # host link reference: pinned host -> device copy bandwidth (copy engine)
    h = torch.empty(1 << 28, dtype=torch.uint8).pin_memory()
    d = torch.empty(1 << 28, dtype=torch.uint8, device=dev)
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        d.copy_(h, non_blocking=True)
    b.record()
    b.synchronize()
    h2d_gbs = 5 * (1 << 28) / (a.elapsed_time(b) * 1e6)
    hbm_frac = t.hbm_value_slots / t.capacity
    res = {"metric": METRIC, "value": round(2 * args.steps * batch / (ms * 1e-3) / 1e9, 4),
           "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": TIERED_WORKLOAD, "slots": slots, "dim": dim,
                      "hbm_value_budget_gib": round(budget / (1 << 30), 2),
                      "host_value_gib": round((t.capacity - t.hbm_value_slots) * dim * 4 / (1 << 30), 2),
                      "value_slots_in_hbm_frac": round(hbm_frac, 4), "batch": batch,
                      "create_s": round(create_s, 1), "fill_s": round(fill_s, 1),
                      "host_huge_page_frac": round(host_mem["huge_bytes"] /
                                                   max(1, host_mem["host_bytes"]), 4),
                      "host_one_mapping": host_mem["one_mapping"],
                      "lambda_fill": round(lam, 4)},
           "find_bkvs": round(args.steps * batch / f_ms / 1e6, 4),
           "upsert_bkvs": round(args.steps * batch / u_ms / 1e6, 4),
           "find_ptr_bkvs": round(find_ptr_bkvs, 4),
           "find_ptr_gather_bkvs": round(find_ptr_gather_bkvs, 4),
           "kernel_ms_per_step": kernel_ms,
           "launch": {"find_tpk": args.find_tpk or "default",
                      "update_tpk": args.update_tpk or "default"},
           "find_hit_rate": round(c["find_hit"] / max(1, c["find_hit"] + c["find_miss"]), 4),
           "eviction_rate": round(c["evicted"] / max(1, attempted), 4),
           "rejection_rate": round(c["rejected"] / max(1, attempted), 4),
           "host_value_bytes_per_step_est": int((1 - hbm_frac) * 4 * dim * (c["find_hit"] + c["updated"]
                                                 + c["inserted"] + c["evicted"]) / args.steps),
           "h2d_copy_gbs_reference": round(h2d_gbs, 1)}
    t.close()
    return res


# ----------------------------------------------------------- serving loop

SERVE_WORKLOAD = ("serving: the 8 multi-table tables (LRU, pre-filled to lambda 1.0) behind the "
                  "continuous-batching loop; requests find (0.8) / insert_or_assign (0.2), "
                  "lognormal sizes (median 4096, sigma 1.5, clipped to 256-262144) of Zipf(1.1) "
                  "keys over 2^32 on a uniformly chosen table, Poisson arrivals; inputs from and "
                  "results to pinned host memory")


def _latency_stats(items, res, stats=None):
    lat = np.array([(r.done_s - it["arrival_s"]) * 1e3 for r, it in zip(res, items)])
    span = max(r.done_s for r in res) - min(it["arrival_s"] for it in items)
    keys = sum(int(it["keys"].numel()) for it in items)
    out = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
           "p99_ms": round(float(np.percentile(lat, 99)), 3),
           "p999_ms": round(float(np.percentile(lat, 99.9)), 3),
           "max_ms": round(float(lat.max()), 3),
           "bkvs": round(keys / span / 1e9, 4), "requests": len(items),
           "rounds": len({r.round for r in res})}
    if stats:
        # where the run's time went: host loop phases, device busy time, and
        # the host link's load (bytes each way over the run's wall time)
        w_s = max(stats["wall_s"], 1e-9)
        out["breakdown"] = {
            "wall_s": round(stats["wall_s"], 3),
            "host_admit_s": round(stats["host_admit_s"], 3),
            "host_launch_s": round(stats["host_launch_s"], 3),
            "host_retire_s": round(stats["host_retire_s"], 3),
            "host_idle_s": round(stats["idle_s"], 3),
            "gpu_compute_s": round(stats["gpu_compute_s"], 3),
            "gpu_copy_out_s": round(stats["gpu_copy_out_s"], 3),
            "direct_rounds": stats["direct_rounds"], "batched_rounds": stats["batched_rounds"],
            "h2d_gbs": round(stats["h2d_bytes"] / w_s / 1e9, 2),
            "d2h_gbs": round(stats["d2h_bytes"] / w_s / 1e9, 2)}
    return out


def measure_link(nbytes=1 << 28, reps=5):
    """Host link bandwidth between page-locked host memory and HBM, in GB/s:
    host to device, device to host, and both at once (two streams), best of
    `reps` copies of nbytes each way, timed with CUDA events."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = {"h2d": 0.0, "d2h": 0.0, "both": 0.0}
    for _ in range(reps):
        for kind in best:
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if kind in ("h2d", "both"):
                s1.wait_event(a)
                with torch.cuda.stream(s1):
                    d_a.copy_(h_in, non_blocking=True)
            if kind in ("d2h", "both"):
                s2.wait_event(a)
                with torch.cuda.stream(s2):
                    h_out.copy_(d_b, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s1)
            torch.cuda.current_stream().wait_stream(s2)
            b.record()
            b.synchronize()
            moved = nbytes * (2 if kind == "both" else 1)
            best[kind] = max(best[kind], moved / (a.elapsed_time(b) * 1e-3) / 1e9)
    return {k: round(v, 1) for k, v in best.items()}


def run_serve(args):
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import autotune
    from paper_2603_17168_gb300 import workloads as w

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.seed_for(5, rank))
    rng = np.random.default_rng(w.seed_for(5, 100 + rank))
    shrink = args.multi_shrink
    tables = []
    for slots, dim in zip(w.MULTI_SLOTS, w.MULTI_DIMS):
        t = hkv.Table(slots >> shrink, dim, hkv.LRU)
        fill_table(t, 1.0, gen, dim)
        autotune.tune(t, w.zipf_keys_torch(gen, w.Zipf(1.1, UNIVERSE), 4096))
        tables.append(t)
    budget = int(args.serve_budget_gib * (1 << 30))
    srv = hkv.Server(tables, ring_keys=1 << 20, hbm_budget_bytes=budget, max_inflight=3)
    server_gib = srv.hbm_bytes / (1 << 30)
    z = w.Zipf(1.1, UNIVERSE)
    pool = []
    for _ in range(args.serve_pool):
        tab = int(rng.integers(0, len(tables)))
        n = int(np.clip(np.rint(np.exp(np.log(4096) + 1.5 * rng.standard_normal())), 256, 262144))
        op = hkv.OP_FIND if rng.random() < 0.8 else hkv.OP_UPSERT
        dim = tables[tab].dim
        keys = torch.from_numpy(z.keys(rng, n).view(np.int64)).pin_memory()
        vals = (torch.empty((n, dim), dtype=torch.float32).pin_memory() if op == hkv.OP_FIND else
                torch.from_numpy(w.normal_values(rng, n, dim)).pin_memory())
        flags = torch.empty(n, dtype=torch.uint8).pin_memory()
        pool.append(dict(table=tab, op=op, keys=keys, values=vals, flags=flags))
    mean_n = float(np.mean([p["keys"].numel() for p in pool]))
    # bytes each request moves over the host link, per key of the pool
    keys_total = sum(p["keys"].numel() for p in pool)
    h2d_pk = sum(p["keys"].numel() * 8 + (p["values"].numel() * 4 if p["op"] == hkv.OP_UPSERT
                                          else 0) for p in pool) / keys_total
    d2h_pk = sum(p["keys"].numel() + (p["values"].numel() * 4 if p["op"] == hkv.OP_FIND else 0)
                 for p in pool) / keys_total
    link = measure_link()
    link_bound = min(link["h2d"] * 1e9 / h2d_pk, link["d2h"] * 1e9 / d2h_pk,
                     link["both"] * 1e9 / (h2d_pk + d2h_pk)) / 1e9

    def make(n_req, rate):
        items, t = [], 0.0
        for i in range(n_req):
            if rate:
                t += rng.exponential(1.0 / rate)
            it = dict(pool[i % len(pool)])
            it["arrival_s"] = t
            items.append(it)
        return items

    def run(items, reqs, batched):
        res = srv.run(reqs, batched=batched)
        return _latency_stats(items, res, srv.stats())

    # warm the graphs and the pipeline
    warm = make(min(256, len(pool)), 0)
    srv.run(hkv.make_requests(warm), batched=True)
    srv.run(hkv.make_requests(warm[:64]), batched=False)
    # peak: closed loop, every request queued at t = 0
    peak_items = make(args.serve_peak_requests, 0)
    peak_reqs = hkv.make_requests(peak_items)
    peak_b = run(peak_items, peak_reqs, True)
    peak_p = run(peak_items, peak_reqs, False)
    peak_keys_s = peak_b["bkvs"] * 1e9
    # the same closed loops with every round timed on the device, for the
    # breakdown only (the timing events cost host time of their own)
    srv.profile(True)
    srv.run(peak_reqs, batched=True)
    peak_b["profiled"] = _latency_stats(peak_items, srv.run(peak_reqs, batched=True),
                                        srv.stats())["breakdown"]
    srv.run(peak_reqs, batched=False)
    peak_p["profiled"] = _latency_stats(peak_items, srv.run(peak_reqs, batched=False),
                                        srv.stats())["breakdown"]
    srv.profile(False)
    served = {}
    for frac in (0.25, 0.50, 0.90):
        rate = frac * peak_keys_s / mean_n
        if args.serve_warm_seconds > 0:
            # steady state: the round combinations this load produces are
            # captured before its measured runs
            warm = make(max(64, int(rate * args.serve_warm_seconds)), rate)
            warm_reqs = hkv.make_requests(warm)
            srv.run(warm_reqs, batched=True)
            srv.run(warm_reqs, batched=False)
        n_req = max(64, int(rate * args.serve_seconds))
        items = make(n_req, rate)
        reqs = hkv.make_requests(items)
        served[f"{int(frac * 100)}%"] = {
            "offered_bkvs": round(frac * peak_keys_s / 1e9, 4),
            "batched": run(items, reqs, True),
            "plain": run(items, reqs, False)}
    srv.close()
    for t in tables:
        t.close()
    return {"metric": METRIC, "value": peak_b["bkvs"], "unit": UNIT, "n_gpus": world,
            "steps": args.serve_peak_requests, "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": SERVE_WORKLOAD, "slots_shift": shrink,
                       "hbm_budget_gib": args.serve_budget_gib,
                       "server_hbm_gib": round(server_gib, 2),
                       "ring_keys_per_table": 1 << 20, "max_inflight_rounds": 3,
                       "request_pool": len(pool), "mean_request_keys": round(mean_n),
                       "seconds_per_load": args.serve_seconds,
                       "warm_seconds_per_load": args.serve_warm_seconds,
                       "link_bytes_per_key": {"h2d": round(h2d_pk, 1), "d2h": round(d2h_pk, 1)},
                       "link_gbs": link,
                       "link_bound_bkvs": round(link_bound, 4),
                       "step": "a request; value = closed-loop peak of the batched loop"},
            "peak": {"batched": peak_b, "plain": peak_p}, "served": served}


def served_record(args):
    """The serving workload's latency half of the metric in the default run:
    the same server, tables and request pool as --workload serve, with
    args.served_seconds per offered load (the full record uses 60 s). It runs
    as its own process, as a server would, so nothing the single-table run
    left in this process (its contexts' memory, threads, pinned buffers)
    shares the host with the loop."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve",
           "--serve-seconds", str(args.served_seconds),
           "--serve-warm-seconds", str(args.serve_warm_seconds),
           "--serve-budget-gib", str(args.serve_budget_gib),
           "--serve-pool", str(args.serve_pool),
           "--serve-peak-requests", str(args.serve_peak_requests),
           "--multi-shrink", str(args.multi_shrink)]
    env = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE"):
        env.pop(k, None)
    out = subprocess.run(cmd, stdout=subprocess.PIPE, env=env, text=True, check=True).stdout
    r = json.loads([x for x in out.splitlines() if x.startswith("{")][-1])
    keep = ("p50_ms", "p99_ms", "bkvs", "requests")
    return {"workload": r["config"]["workload"],
            "process": "own (bench.py --workload serve)",
            "seconds_per_load": args.served_seconds,
            "warm_seconds_per_load": args.serve_warm_seconds,
            "link_bound_bkvs": r["config"]["link_bound_bkvs"],
            "peak_bkvs": {"batched": r["peak"]["batched"]["bkvs"],
                          "plain": r["peak"]["plain"]["bkvs"]},
            "loads": {k: {"offered_bkvs": v["offered_bkvs"],
                          "batched": {x: v["batched"][x] for x in keep},
                          "plain": {x: v["plain"][x] for x in keep}}
                      for k, v in r["served"].items()}}


def run_apis(args):
    """Every API by value width and load factor, and find by capacity (the
    paper's per-API load-factor sweep over its Configs A-C, Sec. 5.2, and its
    capacity scaling, Sec. 5.3). Tables of 2^27 slots (the paper's 128 M),
    LRU, dual-bucket, dims 8 / 32 / 64, filled with uniform keys over 2^32;
    each call takes 2^20 keys, half resident (sampled from the table) and
    half fresh uniform keys, as in the paper's uniform-key sweep. Per load
    factor the readers run first (find, find*, contains), then assign of
    resident keys (updates in place), then insert_or_assign of fresh and
    resident keys (the only call that moves lambda; its drift is reported).
    find_no_digest / contains_no_digest are the digest ablation (Sec. 5.4,
    Exp 3a): the same calls comparing every key of a probed bucket instead
    of reading its digest line first.
    Capacity sweep: find at lambda 0.5, dim 32, 2^24 .. 2^29 slots. Times
    are the median of `reps` calls, CUDA events on the launching stream."""
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(6))
    batch, reps = args.batch, max(3, args.steps)

    def med_ms(fn, inputs):
        fn(inputs[0])
        torch.cuda.synchronize()
        ts = []
        for x in inputs:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(x)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def mixed_batches(t, n_batches):
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        res = torch.empty(t.capacity, dtype=torch.int64, device=dev)
        t.export_batch(0, t.capacity, res, None, None, None, cnt)
        n_res = int(cnt.item())
        out = []
        for _ in range(n_batches):
            half = batch // 2
            pick = torch.randint(0, max(1, n_res), (half,), device=dev, generator=gen)
            k = torch.cat([res[pick], w.uniform_keys_torch(gen, batch - half, UNIVERSE)])
            out.append(k[torch.randperm(batch, device=dev, generator=gen)].contiguous())
        del res
        return out, n_res

    rate = lambda ms: round(batch / ms / 1e6, 4)  # noqa: E731
    per_dim = {}
    for dim in (8, 32, 64):
        t = hkv.Table(1 << 27, dim, hkv.LRU, dual_bucket=True)
        rows = {}
        for lam in (0.5, 1.0):
            lam_fill = fill_table(t, lam, gen, dim)
            ks, _ = mixed_batches(t, reps)
            vals = torch.randn((batch, dim), device=dev, generator=gen)
            out = torch.empty((batch, dim), device=dev)
            fl = torch.empty(batch, dtype=torch.uint8, device=dev)
            ptrs = torch.empty(batch, dtype=torch.int64, device=dev)
            r = {"lambda_fill": round(lam_fill, 4),
                 "find": rate(med_ms(lambda k: t.find(k, out, fl), ks)),
                 "find_ptr": rate(med_ms(lambda k: t.find_ptr(k, ptrs, fl), ks)),
                 "contains": rate(med_ms(lambda k: t.contains(k, fl), ks)),
                 # the digest ablation (Exp 3a): every key of a probed bucket compared
                 "find_no_digest": rate(med_ms(lambda k: t.find_full_keys(k, out, fl), ks)),
                 "contains_no_digest": rate(med_ms(lambda k: t.find_full_keys(k, None, fl),
                                                   ks)),
                 "assign": rate(med_ms(lambda k: t.assign(k, vals), ks)),
                 "insert_or_assign": rate(med_ms(lambda k: t.insert_or_assign(k, vals), ks))}
            r["lambda_end"] = round(t.size() / t.capacity, 4)
            rows[str(lam)] = r
        per_dim[str(dim)] = rows
        t.close()
    capacity = {}
    for log2 in (24, 26, 28, 29):
        t = hkv.Table(1 << log2, 32, hkv.LRU, dual_bucket=True)
        fill_table(t, 0.5, gen, 32)
        ks, _ = mixed_batches(t, reps)
        out = torch.empty((batch, 32), device=dev)
        fl = torch.empty(batch, dtype=torch.uint8, device=dev)
        capacity[f"2^{log2}"] = rate(med_ms(lambda k: t.find(k, out, fl), ks))
        t.close()
    cv = list(capacity.values())
    return {"metric": "B-KV/s per API by value width and load factor; find by capacity",
            "value": per_dim["32"]["0.5"]["find"], "unit": UNIT, "n_gpus": 1, "steps": reps,
            "warmup": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "2^27 slots, LRU, dual-bucket, dims 8/32/64, uniform fill "
                                   "over 2^32, 2^20-key calls half resident / half fresh; "
                                   "capacity sweep 2^24..2^29 slots at dim 32, lambda 0.5",
                       "batch": batch},
            "per_dim": per_dim, "capacity_find": capacity,
            "capacity_find_spread": round((max(cv) - min(cv)) / statistics.mean(cv), 4)}


def distinct_keys_torch(gen, n, universe, dev):
    """n distinct keys of uniform ranks in [1, universe], in random order."""
    import torch
    from paper_2603_17168_gb300 import workloads as w
    r = torch.unique(torch.randint(1, universe + 1, (n + n // 8 + 1024,), dtype=torch.int64,
                                   device=dev, generator=gen))[:n]
    return w.rank_to_key_torch(r[torch.randperm(r.numel(), device=dev, generator=gen)])


def run_ordered(args):
    """Deterministic dual-bucket upsert (ordered phase I) against the
    concurrent mode on twin tables of the single-table shape, fed the same
    duplicate-free batches (deterministic mode refuses duplicates): half the
    keys of each batch come from the previous batch, half are fresh."""
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(6))
    nb, batch = 1 << args.nb_log2, args.batch
    res = {}
    for lam in (0.5, 1.0):
        tabs = {m: hkv.Table(nb * 128, DIM, hkv.LFU, dual_bucket=True, deterministic=(m == "ordered"))
                for m in ("ordered", "concurrent")}
        target = lam * nb * 128 if lam < 1 else 0.999 * nb * 128
        vals = torch.randn((batch, DIM), device=dev, generator=gen)
        for _ in range(400):
            if tabs["concurrent"].size() >= target:
                break
            k = distinct_keys_torch(gen, batch, UNIVERSE, dev)
            for t in tabs.values():
                t.insert_or_assign(k, vals[:k.numel()])
        nbat = args.warmup + args.steps
        prev = distinct_keys_torch(gen, batch, UNIVERSE, dev)
        batches = []
        for _ in range(nbat):
            fresh = distinct_keys_torch(gen, batch, UNIVERSE, dev)
            k = torch.unique(torch.cat([prev[:batch // 2], fresh[:batch // 2]]))
            k = k[torch.randperm(k.numel(), device=dev, generator=gen)]
            batches.append(k)
            prev = k
        st = torch.empty(batch, dtype=torch.uint8, device=dev)
        row = {"lambda_fill": round(tabs["concurrent"].size() / (nb * 128), 4)}
        for m, t in tabs.items():
            for i in range(args.warmup):
                t.insert_or_assign(batches[i], vals[:batches[i].numel()],
                                   status_out=st[:batches[i].numel()])
            torch.cuda.synchronize()
            t.reset_counters()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            nk = 0
            for i in range(args.warmup, nbat):
                t.insert_or_assign(batches[i], vals[:batches[i].numel()],
                                   status_out=st[:batches[i].numel()])
                nk += batches[i].numel()
            b.record()
            b.synchronize()
            c = t.read_counters()
            row[m] = {"upsert_bkvs": round(nk / a.elapsed_time(b) / 1e6, 4),
                      "updated": c["updated"], "inserted": c["inserted"],
                      "evicted": c["evicted"], "rejected": c["rejected"]}
        row["ordered_over_concurrent"] = round(row["ordered"]["upsert_bkvs"]
                                               / row["concurrent"]["upsert_bkvs"], 4)
        res[str(lam)] = row
        for t in tabs.values():
            t.close()
    return {"metric": "insert_or_assign B-KV/s, deterministic (ordered phase I) vs concurrent "
                      "dual-bucket", "value": res["1.0"]["ordered"]["upsert_bkvs"],
            "unit": "B-KV/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"ordered: twin tables of {nb * 128} slots, dim {DIM}, LFU, "
                                   f"dual-bucket; batches of {batch} distinct keys, half from "
                                   "the previous batch, half fresh uniform over 2^32"},
            "per_lambda": res}


def quality_stream(t, policy_custom, z, gen, batch, n_batches, measure_from,
                   track_first_eviction=False, keep=None):
    """Sustained ingestion: per batch, look the keys up (contains), then
    insert_or_assign them (scores = batch number for HKV_CUSTOM; the epoch
    advances every batch). Returns (hits, lookups) over batches >=
    measure_from and the load factor at the first eviction; `keep`, if
    given, receives every batch's keys (for the stream's frequencies)."""
    import torch
    from paper_2603_17168_gb300 import workloads as w
    dev = torch.device("cuda", 0)
    vals = torch.zeros((batch, 1), device=dev)
    hits = torch.zeros((), dtype=torch.int64, device=dev)
    looked = 0
    first_ev = None
    for b in range(n_batches):
        keys = w.zipf_keys_torch(gen, z, batch)
        if keep is not None:
            keep[b * batch:(b + 1) * batch] = keys
        t.set_epoch(b)
        if b >= measure_from:
            hits += t.contains(keys).sum()
            looked += batch
        sc = torch.full((batch,), b, dtype=torch.int64, device=dev) if policy_custom else None
        t.insert_or_assign(keys, vals, sc)
        if track_first_eviction and first_ev is None:
            c = t.read_counters()
            if c["evicted"] + c["rejected"] > 0:
                first_ev = t.size() / t.capacity
    return int(hits.item()), looked, first_ev


def run_quality(args):
    """Cache quality under sustained Zipf ingestion (Sec. 5: Exp 3c, Exp 4).
    Hit rate by policy and alpha: single-bucket tables of 2^quality_log2
    slots, batches of 2^20 Zipf(alpha) keys over a universe of 2^30 and of
    2^32 keys; the first two capacities of keys fill the table and reach
    steady state, the hit rate is taken over the next three (5 x capacity in
    all). Single vs dual bucket at alpha 0.99 under LFU (universe 2^30): the
    load factor at the first eviction, the hit rate, and top-N retention: the
    fraction of the N = capacity keys seen most often in the stream (ties by
    the larger key, as the table breaks them) resident at the end."""
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cap = 1 << args.quality_log2
    batch = 1 << 20
    per_cap = max(1, cap // batch)
    n_batches, measure_from = 5 * per_cap, 2 * per_cap
    policies = (("LRU", hkv.LRU), ("LFU", hkv.LFU), ("EPOCH_LRU", hkv.EPOCH_LRU),
                ("EPOCH_LFU", hkv.EPOCH_LFU), ("CUSTOM", hkv.CUSTOM))
    alphas = (0.5, 0.75, 0.99, 1.25)
    hit_rate = {}
    for ulog in (30, 32):
        for alpha in alphas:
            z = w.Zipf(alpha, 1 << ulog)
            for name, pol in policies:
                gen = torch.Generator(device=dev)
                gen.manual_seed(w.seed_for(7) + int(alpha * 100) + ulog)  # one stream per (u, a)
                t = hkv.Table(cap, 1, pol)
                h, n, _ = quality_stream(t, pol == hkv.CUSTOM, z, gen, batch, n_batches,
                                         measure_from)
                hit_rate.setdefault(f"universe_2^{ulog}", {}).setdefault(name, {})[str(alpha)] = \
                    round(100.0 * h / n, 2)
                t.close()
    z = w.Zipf(0.99, 1 << 30)
    bucket = {}
    for dual in (False, True):
        gen = torch.Generator(device=dev)
        gen.manual_seed(w.seed_for(7) + 99)
        t = hkv.Table(cap, 1, hkv.LFU, dual_bucket=dual)
        seen = torch.empty(n_batches * batch, dtype=torch.int64, device=dev)
        h, n, first = quality_stream(t, False, z, gen, batch, n_batches, measure_from,
                                     track_first_eviction=True, keep=seen)
        k = torch.empty(cap, dtype=torch.int64, device=dev)
        cnt, *_ = t.export_batch(0, cap, keys=k)
        torch.cuda.synchronize()
        resident = torch.sort(k[:int(cnt.item())])[0]
        uk, counts = torch.unique(seen, return_counts=True)
        del seen
        # the N keys seen most often, ties by the larger key: order by
        # (count, key) descending
        o = torch.sort(uk, descending=True, stable=True)[1]
        o = o[torch.sort(counts[o], descending=True, stable=True)[1]]
        ideal = uk[o[:cap]]
        j = torch.searchsorted(resident, ideal).clamp_(max=max(resident.numel() - 1, 0))
        retained = int((resident[j] == ideal).sum().item())
        bucket["dual" if dual else "single"] = {
            "first_eviction_lambda": round(first, 4) if first is not None else None,
            "top_n_retention_pct": round(100.0 * retained / min(cap, ideal.numel()), 2),
            "hit_rate_pct": round(100.0 * h / n, 2)}
        t.close()
    return {"metric": "cache hit rate (%) by policy and Zipf alpha; single vs dual bucket",
            "value": hit_rate["universe_2^30"]["LFU"]["0.99"],
            "unit": "% hit rate (LFU, alpha 0.99, universe 2^30)",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"quality: {cap} slots, dim 1, batches of {batch} Zipf(alpha) "
                                   "keys over 2^30 and 2^32; per batch contains() then "
                                   "insert_or_assign; 2 capacities of warm-up, hit rate over the "
                                   "next 3; HKV_CUSTOM scores = batch number; epoch = batch "
                                   "number; top-N = the capacity keys seen most often",
                       "capacity": cap, "batch": batch},
            "hit_rate_pct": hit_rate, "single_vs_dual_alpha_0.99_lfu_universe_2^30": bucket}


def run_concurrency(args):
    """Concurrency ablation (Sec. 5, Exp 3e): host client threads, each with
    its own CUDA stream, issue 200 batches of 2^16 keys of one role (find,
    assign, or insert_or_assign of fresh keys) against one table (2^24 slots,
    dim 16, LRU, filled to lambda 0.75), under the triple-group rule and
    under a reader/writer lock (hkv_set_concurrency). Throughput = all keys
    / wall time from the start barrier to the last stream's completion."""
    import threading
    import torch
    import paper_2603_17168_gb300 as hkv
    from paper_2603_17168_gb300 import workloads as w
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cap, dim, batch, nbat, pool = 1 << 24, 16, 1 << 16, 200, 8
    mixes = {"1U": (0, 1, 0), "2U": (0, 2, 0), "4U": (0, 4, 0), "10U": (0, 10, 0),
             "4F/5U/1I": (4, 5, 1), "4F/2U/4I": (4, 2, 4), "8F/1U/1I": (8, 1, 1)}
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed_for(8))
    res = {}
    for mix, (nf, nu, ni) in mixes.items():
        row = {}
        for mode in ("triple_group", "rw_lock"):
            t = hkv.Table(cap, dim, hkv.LRU)
            fill = torch.randn((1 << 20, dim), device=dev, generator=gen)
            while t.size() < 0.75 * cap:
                t.insert_or_assign(w.uniform_keys_torch(gen, 1 << 20, 1 << 40), fill)
            k = torch.empty(cap, dtype=torch.int64, device=dev)
            cnt, *_ = t.export_batch(0, cap, keys=k)
            torch.cuda.synchronize()
            resident = k[:int(cnt.item())]
            t.set_concurrency(mode == "rw_lock")
            roles = ["F"] * nf + ["U"] * nu + ["I"] * ni
            work = []
            for r in roles:
                if r == "I":
                    keys = [w.uniform_keys_torch(gen, batch, 1 << 40) for _ in range(pool)]
                else:
                    keys = [resident[torch.randint(0, resident.numel(), (batch,), device=dev,
                                                   generator=gen)] for _ in range(pool)]
                vals = [torch.randn((batch, dim), device=dev, generator=gen) for _ in range(pool)]
                out = torch.empty((batch, dim), device=dev)
                work.append((r, keys, vals, out, torch.cuda.Stream()))
            torch.cuda.synchronize()
            start = threading.Barrier(len(work) + 1)

            def client(r, keys, vals, out, s):
                start.wait()
                for i in range(nbat):
                    if r == "F":
                        t.find(keys[i % pool], out, stream=s)
                    elif r == "U":
                        t.assign(keys[i % pool], vals[i % pool], stream=s)
                    else:
                        t.insert_or_assign(keys[i % pool], vals[i % pool], stream=s)
                s.synchronize()

            th = [threading.Thread(target=client, args=wk) for wk in work]
            for x in th:
                x.start()
            start.wait()
            t0 = time.perf_counter()
            for x in th:
                x.join()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            row[mode] = round(len(work) * nbat * batch / dt / 1e9, 4)
            t.close()
        row["triple_over_rw"] = round(row["triple_group"] / row["rw_lock"], 3)
        res[mix] = row
    return {"metric": "B-KV/s under concurrent host clients: triple-group vs reader/writer lock",
            "value": res["10U"]["triple_group"], "unit": "B-KV/s (10 updater threads)",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"concurrency: one table of {cap} slots, dim {dim}, LRU, "
                                   f"lambda 0.75; client threads with their own streams, {nbat} "
                                   f"batches of {batch} keys each (F find, U assign of resident "
                                   "keys, I insert_or_assign of fresh keys)"},
            "mixes": res}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        res = run_reference(args)
    elif args.workload == "multi":
        import __graft_entry__ as g
        g.build()
        res = run_multi(args)
    elif args.workload == "tiered":
        import __graft_entry__ as g
        g.build()
        res = run_tiered(args)
    elif args.workload == "serve":
        import __graft_entry__ as g
        g.build()
        res = run_serve(args)
    elif args.workload == "ordered":
        import __graft_entry__ as g
        g.build()
        res = run_ordered(args)
    elif args.workload == "quality":
        import __graft_entry__ as g
        g.build()
        res = run_quality(args)
    elif args.workload == "apis":
        import __graft_entry__ as g
        g.build()
        res = run_apis(args)
    elif args.workload == "concurrency":
        import __graft_entry__ as g
        g.build()
        res = run_concurrency(args)
    else:
        import __graft_entry__ as g
        g.build()
        res = run_ours(args)
        rank, world, _ = dist_env()
        if res is not None and rank == 0:
            res["cpu_baseline"] = None if (args.no_cpu_baseline or world > 1) else cpu_baseline()
            if not args.no_served and world == 1:
                res["served"] = served_record(args)
    if res is not None:
        print(json.dumps(res), flush=True)
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
