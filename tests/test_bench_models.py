"""Properties of bench.py's measurement models (CPU only): the algorithmic
byte counts and scattered-access counts it derives from the device counters,
and the workload name it reports. These feed `roofline` and `kernels` in the
bench line, so they are checked against what each kernel must move, not
re-derived formula by formula."""
import bench

ZERO = {k: 0 for k in ("find_hit", "find_miss", "unique", "updated", "inserted", "evicted",
                       "rejected", "retries", "find_lines", "find_keys", "upd_lines", "upd_keys",
                       "ins_lines", "ins_score_lines", "ins_keys", "upd_claims",
                       "upd_claim_lines")}


def counters(**kw):
    c = dict(ZERO)
    c.update(kw)
    return c


def test_find_bytes_count_lines_keys_and_hit_rows():
    n, dim = 1000, 32
    base = bench.kernel_bytes("find", counters(find_lines=n), 1, n, dim)
    # every key reads its 8-byte key, writes its found flag, reads one line
    assert base == n * 9 + 128 * n
    # a hit adds its row read from the table and written to the output
    hits = bench.kernel_bytes("find", counters(find_lines=n, find_hit=10), 1, n, dim)
    assert hits - base == 10 * 2 * 4 * dim
    # a confirmed key read is one 32-byte sector
    keys = bench.kernel_bytes("find", counters(find_lines=n, find_keys=7), 1, n, dim)
    assert keys - base == 7 * 32


def test_phase_i_moves_nothing_without_deferred_keys():
    c = counters(unique=500, updated=300, inserted=200, upd_claims=200, upd_lines=500)
    assert bench.kernel_bytes("insert", c, 1, 1000, 32) == 0
    assert bench.kernel_bytes("reconcile", c, 1, 1000, 32) == 0


def test_update_rows_scale_with_dim_per_update_and_claim():
    c = counters(unique=500, updated=300, inserted=200, upd_claims=200, upd_lines=500)
    b32 = bench.kernel_bytes("update", c, 1, 1000, 32)
    b64 = bench.kernel_bytes("update", c, 1, 1000, 64)
    # each update and each claim reads one input row and writes one table row
    assert b64 - b32 == (300 + 200) * 2 * 4 * 32


def test_victim_searches_count_two_kib_per_pair_run():
    c0 = counters(unique=100, updated=0, inserted=0, evicted=50, rejected=50)
    c1 = counters(unique=100, updated=0, inserted=0, evicted=50, rejected=50, ins_score_lines=3)
    assert bench.kernel_bytes("insert", c1, 1, 100, 8) - bench.kernel_bytes("insert", c0, 1, 100, 8) \
        == 3 * 2048


def test_random_access_model_counts_rows_as_lines():
    c = counters(find_lines=100, find_hit=40, find_keys=60)
    ra = bench.kernel_random_accesses("find", c, 1, 100, 32)
    assert ra["line_reads"] == 100 + 40 and ra["sector_reads"] == 60
    assert ra["line_writes"] == 0 and ra["sector_writes"] == 0
    assert ra["stream_bytes"] == 100 * 9 + 40 * 128
    u = counters(unique=10, updated=4, upd_claims=5, upd_lines=10, upd_keys=3)
    ru = bench.kernel_random_accesses("update", u, 1, 10, 32)
    # updates and claims each read an input row and write a table row
    assert ru["line_reads"] == 10 + 4 + 5 and ru["line_writes"] == 4 + 5
    assert ru["sector_writes"] == 4 + 3 * 5
    assert bench.kernel_random_accesses("dedup", u, 1, 10, 32) is None


def test_workload_name_follows_the_sizes():
    assert bench.single_workload() == bench.WORKLOAD
    assert "2^26 slots (2^19 buckets x 128)" in bench.WORKLOAD
    assert "2^20 Zipf(1.05)" in bench.WORKLOAD
    small = bench.single_workload(17, 1 << 18, (0.5,))
    assert small.startswith("single table x1 (lambda 0.50): 2^24 slots (2^17 buckets x 128)")
    assert "2^18 Zipf(1.05)" in small
    assert "3000 Zipf" in bench.single_workload(17, 3000, (0.5, 1.0))


def test_upsert_op_bytes_leave_out_dedup_and_bookkeeping():
    c = counters(unique=500, updated=300, inserted=200, upd_claims=200, upd_lines=500,
                 evicted=5, rejected=3)
    n = 1000
    ob = bench.op_bytes("upsert", c, 1, n, 32)
    # the update and insert kernels' work plus one key read and one status
    # byte per input key; dedup, reconcile and status kernels are not counted
    assert ob == (bench.kernel_bytes("update", c, 1, n, 32)
                  + bench.kernel_bytes("insert", c, 1, n, 32) + n * 9)
    assert bench.op_bytes("find", c, 1, n, 32) == bench.kernel_bytes("find", c, 1, n, 32)


def test_spread_is_range_over_mean():
    assert bench.spread([0.5, 0.5, 0.5]) == 0.0
    assert bench.spread([0.4, 0.6]) == 0.4
    assert bench.spread([None, 0.3, 0.3]) == 0.0
    assert bench.spread([]) is None


def test_oracle_baseline_splits_find_over_cores_and_times_the_tiny_run():
    """The CPU baseline's find work is split over processes that each rebuild
    the same sample tables; two steps of it run here on the host."""
    r = bench.time_oracle(steps=1, warmup=0)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
    assert r["find_bkvs"] > 0 and r["upsert_bkvs"] > 0
    assert 0 < bench.tiny_whole_run_seconds() < 60


def test_fused_launches_carry_the_passes_they_ran():
    n, dim = 1000, 32
    c = counters(unique=800, inserted=500, evicted=300, rejected=20, ins_score_lines=600)
    ins = bench.kernel_bytes("insert", c, 1, n, dim)
    rec = bench.kernel_bytes("reconcile", c, 1, n, dim)
    st = bench.kernel_bytes("status", c, 1, n, dim)
    assert rec > 0 and st > 0
    # phase I, reconcile and status in one launch, profiled as insert
    assert bench.kind_bytes("insert", {"insert", "update"}, c, 1, n, dim) == ins + rec + st
    # reconcile and status in one launch after a separate phase I
    assert bench.kind_bytes("insert", {"insert", "status"}, c, 1, n, dim) == ins
    assert bench.kind_bytes("status", {"insert", "status"}, c, 1, n, dim) == st + rec
    # every pass in its own launch
    every = {"insert", "reconcile", "status"}
    assert bench.kind_bytes("status", every, c, 1, n, dim) == st
    assert bench.kind_bytes("insert", every, c, 1, n, dim) == ins
