/*
 * hkv.h - C ABI of a GB300-native (sm_103a) cache-semantic GPU hash table:
 * the data-parallel hot path of HierarchicalKV (arxiv 2603.17168).
 *
 * A table is a power-of-two number B of buckets of S = 128 slots. Each
 * bucket keeps, in HBM, a 128-byte line of 8-bit digests (one per slot) and
 * a 2 KiB run of 128 (uint64 key, uint64 score) pairs, each pair one
 * 16-byte unit; values (dim fp32 each) live in a separate arena addressed by
 * (bucket, slot), spilling past an HBM budget into pinned host memory
 * (Sec. 3.2, Fig. 4; Sec. 3.6; Sec. 4.2).
 *
 * Conventions for every call below:
 *  - Array arguments are DEVICE pointers (or pinned, mapped host pointers
 *    that the device can read) owned by the caller; the library never frees
 *    or retains them after the call's work completes on `stream`.
 *    Value arrays are row-major [n][dim] fp32.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) unless stated otherwise. Outputs are valid once the
 *    stream reaches the call's completion point.
 *  - Each call takes its role of the triple-group protocol (Sec. 3.5,
 *    Table 4) on the table: find, contains, size and export are readers;
 *    assign is an updater; insert_or_assign and erase are inserters.
 *    Readers run concurrently with readers, updaters with updaters, and
 *    every other pair is serialised. The library enforces this across
 *    streams with CUDA events; calls on one stream are ordered anyway.
 *  - Errors are returned as hkv_status; no C++ exception crosses the ABI.
 *    Errors found on the device (a reserved key, a duplicate key in
 *    deterministic mode, a bounded wait that ran out) are latched in the
 *    table and returned by the next hkv_sync / hkv_size call; the batch that
 *    raised them leaves the table unchanged, except HKV_ERR_TIMEOUT.
 *    hkv_last_error() gives a message for the calling thread's last error.
 *  - Keys >= 2^63 are reserved (2^64-1 marks an empty slot, 2^64-2 a locked
 *    one) and may not be inserted.
 */
#ifndef HKV_H
#define HKV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hkv_table_s *hkv_table_t; /* opaque; owned by the library */
typedef void *hkv_stream_t;              /* a cudaStream_t */

typedef enum {
  HKV_OK = 0,
  HKV_ERR_INVALID_ARG = 1,
  HKV_ERR_RESERVED_KEY = 2,
  HKV_ERR_DUPLICATE_KEY = 3, /* deterministic mode only */
  HKV_ERR_OOM = 4,
  HKV_ERR_CUDA = 5,
  HKV_ERR_TIMEOUT = 6,
  HKV_ERR_BUSY = 7
} hkv_status;

/* Score policies (Sec. 3.3, "Scoring policies"; Table 8, cache hit rate by policy). The paper names
 * them without formulas; this library defines, per insert_or_assign or
 * assign call (the table step advances by one at the start of each):
 *   HKV_LRU            score = step, for new and updated keys;
 *   HKV_LFU            new: m (multiplicity of the key in the batch);
 *                      hit: old + m, saturating at 2^64-1;
 *   HKV_EPOCH_LRU      (epoch << 32) | (step & 0xFFFFFFFF);
 *   HKV_EPOCH_LFU      (epoch << 32) | count, count as LFU saturating at 2^32-1;
 *   HKV_CUSTOM         the caller's score of the key's last occurrence;
 *   HKV_CUSTOM_TS_FREQ (epoch << 16) | count, count saturating at 2^16-1,
 *                      the epoch being the caller's timestamp. */
typedef enum {
  HKV_LRU = 0,
  HKV_LFU = 1,
  HKV_EPOCH_LRU = 2,
  HKV_EPOCH_LFU = 3,
  HKV_CUSTOM = 4,
  HKV_CUSTOM_TS_FREQ = 5
} hkv_policy;

/* Per-key result of insert_or_assign (Algorithm 2's outcomes, decided for
 * the batch as a whole): UPDATED = resident at batch start, value and score
 * rewritten; INSERTED = new and resident at batch end; REJECTED = new and not
 * resident at batch end (refused by admission control, or displaced again by
 * a higher-scoring key of the same batch). Every occurrence of a key in the
 * batch gets the same status. */
enum { HKV_ST_UPDATED = 1, HKV_ST_INSERTED = 2, HKV_ST_REJECTED = 3 };

typedef struct {
  uint64_t capacity;       /* slots wanted; rounded up to 128 * 2^k, >= 128 */
  uint32_t dim;            /* fp32 elements per value, >= 1 */
  int32_t policy;          /* hkv_policy */
  int32_t dual_bucket;     /* 1: two candidate buckets per key (Sec. 3.4) */
  int32_t deterministic;   /* 1: a batch holding a key twice is refused with
                              HKV_ERR_DUPLICATE_KEY. With dual_bucket, phase
                              I then runs key by key in batch order (in
                              waves of keys with disjoint buckets), so the
                              table equals sequential Algorithm 3 bit for
                              bit; hkv_insert_or_assign returns once phase
                              I is done, and the no-alloc, batch and serve
                              paths refuse such tables */
  uint64_t hbm_value_budget_bytes; /* value bytes kept in HBM; the rest go to
                                      pinned mapped host memory. 0 = all HBM */
  uint64_t slice_bytes;    /* value slice size (Sec. 4.2); 0 = 1 GiB. Rounded
                              to a power-of-two number of buckets */
} hkv_options;

/* Create a table on the current CUDA device (Sec. 4.2: bucket arrays in HBM,
 * value slices in HBM up to the budget, then pinned mapped host memory).
 * Synchronous. All slots start empty; step = epoch = 0. */
hkv_status hkv_create(const hkv_options *opts, hkv_table_t *out);

/* Free everything the table owns. Synchronous: waits for the table's
 * outstanding work. */
hkv_status hkv_destroy(hkv_table_t t);

/* Table geometry. */
uint64_t hkv_capacity(hkv_table_t t);    /* B * 128 */
uint64_t hkv_num_buckets(hkv_table_t t); /* B */
uint32_t hkv_dim(hkv_table_t t);
uint64_t hkv_hbm_value_slots(hkv_table_t t);
/* Host side of a tiered table (a diagnostic): value bytes in host memory,
 * how many of them transparent huge pages backed when the table was created
 * (scattered host rows are bound by the device's address translation, so
 * the page size matters), and whether the host slices are one registered
 * mapping (1) or cudaHostAlloc slices (0). */
hkv_status hkv_host_memory_info(hkv_table_t t, uint64_t *host_bytes, uint64_t *huge_bytes,
                                int *one_mapping); /* slots whose values sit in HBM */

/* find (reader; Algorithm 1): for each keys[i], probe its bucket(s) through
 * the digest line and copy the value of a hit to values_out[i]
 * ([n][dim]), set found[i] = 1 and scores_out[i] = its score. A miss leaves
 * values_out[i] and scores_out[i] untouched and sets found[i] = 0.
 * found and scores_out may be NULL. Scores are never modified. */
hkv_status hkv_find(hkv_table_t t, uint64_t n, const uint64_t *keys, float *values_out,
                    uint8_t *found, uint64_t *scores_out, hkv_stream_t stream);

/* find* (reader; the pointer-returning find of Sec. 5.2 and Sec. 5.3): the
 * probe of hkv_find, but a hit writes the address of its value row to
 * ptrs_out[i] instead of copying the row, and a miss writes NULL. ptrs_out
 * is a DEVICE array of n pointers; each is a device pointer into an HBM
 * value slice or the device-mapped address of a host slice (position-based
 * addressing, Sec. 3.6), 16-byte aligned when dim % 4 == 0. found may be
 * NULL. An address stays valid until the next call that mutates the table
 * (insert_or_assign, assign, erase) or destroys it. */
hkv_status hkv_find_ptr(hkv_table_t t, uint64_t n, const uint64_t *keys, const float **ptrs_out,
                        uint8_t *found, hkv_stream_t stream);

/* Gather rows through pointers, the companion of find*: out[i] ([n][dim],
 * DEVICE) = the dim floats at ptrs[i] (DEVICE array of n pointers); a NULL
 * pointer leaves out[i] untouched. On the current device; asynchronous. */
hkv_status hkv_gather_rows(const float *const *ptrs, uint64_t n, uint32_t dim, float *out,
                           hkv_stream_t stream);

/* contains (reader; Sec. 3.5): found[i] = 1 iff keys[i] is resident. */
hkv_status hkv_contains(hkv_table_t t, uint64_t n, const uint64_t *keys, uint8_t *found,
                        hkv_stream_t stream);

/* Digest ablation (Sec. 5.4, Exp 3a; a measurement hook): hkv_find (or, with
 * values_out NULL, hkv_contains) without the digest line. A warp reads each
 * probed bucket's 2 KiB run of (key, score) pairs and compares every key;
 * results (rows, found flags) are identical to hkv_find's, the bytes moved
 * per probed bucket are 2 KiB instead of 128 B plus one key sector per
 * digest match. Same arguments, roles and errors as hkv_find; tables with
 * host-memory slices are read in place (no region ordering). */
hkv_status hkv_find_full_keys(hkv_table_t t, uint64_t n, const uint64_t *keys,
                              float *values_out, uint8_t *found, hkv_stream_t stream);

/* insert_or_assign (inserter; Algorithms 2 and 3): upsert a batch.
 * Duplicate keys collapse to one entry: the value of the last occurrence,
 * and multiplicity m for the LFU-type policies. Keys resident at batch start
 * are updated in place; the other keys are inserted into a free slot of
 * their bucket (dual mode: of the less occupied candidate), or, when full,
 * replace the minimum-(score, key) entry if their (score, key) is larger
 * (dual mode: the minimum over both candidates), else are rejected.
 *   values     [n][dim], required: device memory, or page-locked host memory
 *              mapped into the device's address space (cudaHostAlloc /
 *              cudaHostRegister), which the kernels then read in place
 *              (slower: each stored row crosses the host link while the
 *              kernels wait).
 *   scores     [n], required iff policy == HKV_CUSTOM, else ignored (NULL ok).
 *   status_out [n] HKV_ST_*, may be NULL.
 *   evicted_keys / evicted_scores / evicted_values ([n], [n], [n][dim]), may
 *              be NULL: the entries resident at batch start that the batch
 *              displaced, compacted in unspecified order; their number is
 *              written to *n_evicted (a DEVICE uint64, may be NULL).
 * In single-bucket mode the resulting table state, statuses and evicted
 * set are a function of the state and the batch alone (the largest 128
 * (score, key) pairs per bucket); in dual mode they depend on the order in
 * which concurrent keys claim slots. */
hkv_status hkv_insert_or_assign(hkv_table_t t, uint64_t n, const uint64_t *keys,
                                const float *values, const uint64_t *scores,
                                uint8_t *status_out, uint64_t *evicted_keys,
                                uint64_t *evicted_scores, float *evicted_values,
                                uint64_t *n_evicted, hkv_stream_t stream);

/* insert_or_assign for callers that cannot allocate device memory. The
 * paper has no counterpart; this library adds it. hkv_insert_or_assign takes
 * its per-call scratch (about 75 bytes per key) from a stream-ordered pool,
 * which may allocate. A process whose device memory is all reserved up front
 * by its framework's allocator, or a latency-critical path that must not
 * meet an allocation's possible synchronisation or out-of-memory failure,
 * can call this variant instead: it runs the same kernels with the same
 * results (except that evicted values are not returned) in one fixed
 * scratch array of 5 MiB that lives in the library's device image, and it
 * allocates no memory (no cudaMalloc, cudaFree or pool allocation). Like
 * every call it records a CUDA event for cross-stream ordering, reusing the
 * table's event objects.
 *   n           at most HKV_NOALLOC_MAX_KEYS; larger batches are refused
 *               with HKV_ERR_INVALID_ARG (split them, or use the pooled call).
 *   the table's device must be current.
 * Every GPU that loads the library holds the 5 MiB array until the process
 * exits. Each call looks up the array's device address in the current
 * context (cudaGetSymbolAddress); the first lookup on a device may load the
 * library's device code there, so make the first call on each device before
 * any stream capture.
 * All calls on a device share the one array, and each call overwrites it:
 * calls that can overlap on that GPU (issued on different streams, even for
 * different tables) race and must be ordered by the caller.
 * Deterministic dual-bucket tables are refused with HKV_ERR_INVALID_ARG
 * (their ordered waves need pool scratch; use hkv_insert_or_assign). Other
 * arguments and results are as in hkv_insert_or_assign. */
#define HKV_NOALLOC_MAX_KEYS 65536u
hkv_status hkv_insert_or_assign_noalloc(hkv_table_t t, uint64_t n, const uint64_t *keys,
                                        const float *values, const uint64_t *scores,
                                        uint8_t *status_out, uint64_t *evicted_keys,
                                        uint64_t *evicted_scores, uint64_t *n_evicted,
                                        hkv_stream_t stream);

/* find_or_insert (inserter; the cold-start primitive of Sec. 4.1): a key
 * resident at call start keeps its value and has its score updated as by
 * hkv_insert_or_assign; every other key is inserted with the row of its last
 * occurrence in values_io ([n][dim], DEVICE) under the rules of
 * hkv_insert_or_assign (free slot, else admission against the minimum).
 * Then every row of values_io whose key is resident becomes the stored
 * value; rows of keys the table refused keep the caller's values.
 * found_out[i] (nullable) = 1 iff keys[i] was resident at call start.
 * Errors as in hkv_insert_or_assign. */
hkv_status hkv_find_or_insert(hkv_table_t t, uint64_t n, const uint64_t *keys, float *values_io,
                              const uint64_t *scores, uint8_t *found_out, hkv_stream_t stream);

/* assign (updater; Sec. 3.5): for each resident key, overwrite its value
 * (last occurrence wins) and score per the policy; HKV_CUSTOM takes scores[]
 * when given, else keeps the old score. Missing keys are ignored; the bucket
 * structure never changes. values may be NULL (scores only); like the
 * rows of hkv_insert_or_assign they may be device memory or mapped
 * page-locked host memory. */
hkv_status hkv_assign(hkv_table_t t, uint64_t n, const uint64_t *keys, const float *values,
                      const uint64_t *scores, hkv_stream_t stream);

/* erase (inserter; Sec. 3.5): remove each resident key; missing keys are
 * ignored. An emptied slot needs no tombstone (no probe chains). */
hkv_status hkv_erase(hkv_table_t t, uint64_t n, const uint64_t *keys, hkv_stream_t stream);

/* size (reader): number of resident keys, written to *out (HOST). Synchronises
 * `stream` and returns any latched device error. */
hkv_status hkv_size(hkv_table_t t, uint64_t *out, hkv_stream_t stream);

/* export_batch (reader; Sec. 4.1, export_batch_if without a predicate): scan
 * slots [slot_offset, slot_offset + n_slots) in global slot order (slot =
 * bucket * 128 + position) and write each occupied one, compacted in
 * unspecified order, to keys / values / scores / slots (each may be NULL;
 * room for n_slots entries). The number written goes to *count_out, a DEVICE
 * uint64. */
hkv_status hkv_export_batch(hkv_table_t t, uint64_t slot_offset, uint64_t n_slots,
                            uint64_t *count_out, uint64_t *keys, float *values,
                            uint64_t *scores, uint64_t *slots, hkv_stream_t stream);

/* export_batch_if (reader; Sec. 4.1): hkv_export_batch restricted to the
 * occupied slots whose score lies in [score_min, score_max] (inclusive). */
hkv_status hkv_export_batch_if(hkv_table_t t, uint64_t slot_offset, uint64_t n_slots,
                               uint64_t score_min, uint64_t score_max, uint64_t *count_out,
                               uint64_t *keys, float *values, uint64_t *scores, uint64_t *slots,
                               hkv_stream_t stream);

/* copy_state (inserter on dst, reader on src): make dst a copy of src -
 * digests, (key, score) pairs, per-bucket occupancy, every value slice, and
 * the host-side step and epoch - with stream-ordered device-to-device
 * copies on `stream` (host slices copied host to host). The paper has no
 * such call: its evaluation reports the median of repeated runs from one
 * table state (Sec. 5.1), and this is how a caller restores that state
 * between runs, or keeps a checkpoint of a table on the device.
 *   dst, src  distinct tables created with the same capacity, dim, policy,
 *             dual_bucket, deterministic, value budget and slice size, on
 *             the same device; otherwise HKV_ERR_INVALID_ARG and nothing
 *             is copied.
 * Counters, profiling records, launch shapes and the L2 window of dst are
 * kept. Cost: one read and one write of each table's bytes. */
hkv_status hkv_copy_state(hkv_table_t dst, hkv_table_t src, hkv_stream_t stream);

/* Step and epoch used by the score policies (see hkv_policy). Host-side
 * state: apply to calls issued after this one. */
hkv_status hkv_set_step(hkv_table_t t, uint64_t step);
uint64_t hkv_get_step(hkv_table_t t);
hkv_status hkv_set_epoch(hkv_table_t t, uint64_t epoch);

/* Wait for `stream` and return (and clear) the table's latched device error. */
hkv_status hkv_sync(hkv_table_t t, hkv_stream_t stream);

/* Outcome and traffic counters accumulated on the device by the kernels
 * since the last reset, copied to out[HKV_COUNTER_COUNT] (HOST);
 * synchronises `stream`. The traffic counters (digest lines, full-key reads,
 * score lines) give the bytes each kernel had to move for its inputs. */
enum {
  HKV_CNT_FIND_HIT = 0,
  HKV_CNT_FIND_MISS = 1,
  HKV_CNT_UNIQUE = 2,      /* distinct keys of upsert / assign batches */
  HKV_CNT_UPDATED = 3,
  HKV_CNT_INSERTED = 4,    /* claimed a free slot (either phase) */
  HKV_CNT_EVICTED = 5,     /* replaced a minimum entry */
  HKV_CNT_REJECTED = 6,    /* refused by admission */
  HKV_CNT_RETRIES = 7,     /* slot-claim retries after a lost race */
  HKV_CNT_FIND_LINES = 8,  /* 128-B digest lines read by find / contains */
  HKV_CNT_FIND_KEYS = 9,   /* full keys read by find / contains */
  HKV_CNT_UPD_LINES = 10,  /* digest lines read by the update phase */
  HKV_CNT_UPD_KEYS = 11,   /* full keys read by the update phase */
  HKV_CNT_INS_LINES = 12,  /* digest lines read by the insert phase (0: free
                              slots are claimed in the update phase) */
  HKV_CNT_INS_SCORES = 13, /* 2-KiB (key, score) pair runs read by victim
                              searches (one per candidate bucket per try) */
  HKV_CNT_INS_KEYS = 14,   /* 0: victim searches read keys with the pairs */
  HKV_CNT_TIMEOUT_FREE = 15,   /* free-slot claims that ran out of attempts */
  HKV_CNT_TIMEOUT_EVICT = 16,  /* victim searches that ran out of attempts */
  HKV_CNT_TIMEOUT_WHY = 17,    /* last such search's last failure: 1 a locked
                                  candidate, 2 no candidate, 3 lost the
                                  (key, score) CAS, 5 lost a free-slot
                                  CAS */
  HKV_CNT_TIMEOUT_KEY = 18,    /* its key */
  HKV_CNT_UPD_CLAIMS = 19,     /* free-slot claims made by the update phase
                                  (included in HKV_CNT_INSERTED) */
  HKV_CNT_UPD_CLAIM_LINES = 20, /* 32-byte digest sectors those claims read */
  HKV_COUNTER_COUNT = 21
};
hkv_status hkv_read_counters(hkv_table_t t, uint64_t *out, hkv_stream_t stream);
hkv_status hkv_reset_counters(hkv_table_t t, hkv_stream_t stream);

/* Launch shape of the probe kernels: threads per key (1, 2, 4, 8, 16 or 32)
 * for find/contains, and for the update phase of insert_or_assign/assign.
 * 0 keeps the current choice. The autotuner in the Python package sets
 * these; defaults follow the value width. */
hkv_status hkv_set_launch(hkv_table_t t, int find_threads_per_key, int update_threads_per_key);

/* Widest vector the value-row copies of find, the update phase and the
 * insert phase use: 16, 8 or 4 bytes (0 restores the default, 16). A call
 * whose row addresses do not allow it (16 bytes: dim % 4 == 0 and 16-byte
 * aligned rows; 8 bytes: dim even and 8-byte aligned rows) takes the widest
 * width they allow below it. Results do not depend on it. The autotuner
 * sets it with the threads per key. */
hkv_status hkv_set_value_vector(hkv_table_t t, int bytes);

/* Concurrency rule between calls on different streams (Sec. 3.5, Table 4).
 * HKV_CC_TRIPLE_GROUP (default): readers run beside readers and updaters
 * beside updaters, every other pair is ordered. HKV_CC_RW_LOCK: the
 * conventional reader/writer lock of the paper's Exp 3e, where updaters
 * are writers and are ordered among themselves as well. Applies to calls
 * issued afterwards. */
enum { HKV_CC_TRIPLE_GROUP = 0, HKV_CC_RW_LOCK = 1 };
hkv_status hkv_set_concurrency(hkv_table_t t, int mode);

/* L2 residency of the digest array (no counterpart in the paper; the
 * GB300's 126 MB L2 holds the whole digest array of a table up to 2^26
 * slots). Every probe reads a bucket's 128-byte digest line before anything
 * else; with a residency set, the probe and fill kernels of this table
 * launch with an access-policy window that marks its first digest_bytes of
 * digest lines persisting in L2 (0: no window). The window is capped at the device's
 * window limit, and the context's persisting L2 set-aside is raised to the
 * device maximum (a per-context limit, released with the context). Tables
 * start without a window. hkv_l2_residency
 * returns the bytes the window covers (0 if none, or if the device has no
 * persisting L2). */
hkv_status hkv_set_l2_residency(hkv_table_t t, uint64_t digest_bytes);
uint64_t hkv_l2_residency(hkv_table_t t);

/* Batched multi-table rounds (the paper has no batched multi-table API;
 * this is the library's serving-side addition). A batch object binds
 * n_slots distinct tables, each with the largest number of keys a round
 * may give it (max_keys[i] < 2^31), and owns their per-round scratch.
 * hkv_batch_run executes one round: ops[i] (HKV_OP_NONE, HKV_OP_FIND or
 * HKV_OP_UPSERT) on slot i's table, all slots side by side. With use_graph
 * the round is one launch of a CUDA graph captured once per combination of
 * operations and launch shapes; without, the same kernels are launched
 * directly on one stream per slot. Either way the round's sizes and buffer
 * pointers travel in a small descriptor copied to the device at the start
 * of the round, the caller's stream waits for every slot, and each table
 * takes its triple-group role (find: reader, upsert: inserter) for the
 * round. Results are those of hkv_find / hkv_insert_or_assign with
 * found[] / status_out[] in ops[i].flags (nullable for upserts); upsert
 * evictions are not reported. Value rows must be 16-byte aligned.
 * Asynchronous on `stream`; the op array is read before the call returns. */
typedef struct hkv_batch_s *hkv_batch_t;
enum { HKV_OP_NONE = 0, HKV_OP_FIND = 1, HKV_OP_UPSERT = 2 };
typedef struct {
  int32_t op;               /* HKV_OP_* */
  uint64_t n;               /* keys this round, <= the slot's max_keys */
  const uint64_t *keys;     /* device [n] */
  const float *values_in;   /* upsert: device [n][dim] */
  float *values_out;        /* find: device [n][dim] */
  uint8_t *flags;           /* find: found[n]; upsert: status[n] or NULL */
  const uint64_t *scores;   /* upsert under HKV_CUSTOM: device [n]; else NULL */
} hkv_batch_op;
hkv_status hkv_batch_create(int n_slots, const hkv_table_t *tables, const uint64_t *max_keys,
                            hkv_batch_t *out);
hkv_status hkv_batch_run(hkv_batch_t b, const hkv_batch_op *ops, int use_graph,
                         hkv_stream_t stream);
hkv_status hkv_batch_destroy(hkv_batch_t b);

/* Serving loop with continuous batching (the paper has no serving layer;
 * this is the library's addition). A server binds n_tables device-resident
 * tables (not HKV_CUSTOM) and gives each a staging ring of ring_keys keys in
 * HBM. hkv_serve_create refuses with HKV_ERR_OOM when the tables plus the
 * staging exceed hbm_budget_bytes (0: no budget).
 * hkv_serve_run replays a trace of requests in real time: a request is
 * admitted when its keys fit in its table's ring (its inputs are then copied
 * in on a copy stream); while fewer than max_inflight rounds are on the GPU,
 * a round takes, for every table with admitted work, the head of that
 * table's FIFO merged with the following finds that sit next to it in the
 * ring (an upsert always runs alone), runs them as one batched multi-table
 * launch (hkv_batch_run, with use_graph), copies each request's results
 * back to its host buffers and records a completion event. Every request
 * therefore sees its table exactly as it would alone, in arrival order.
 * A round with one busy table calls that table's hkv_find /
 * hkv_insert_or_assign directly instead (grids sized to the request). The
 * results of batched rounds travel back on a copy-out stream of the server,
 * so the next round's kernels overlap them, and every request has its own
 * completion event.
 * With batched = 0 the same trace runs one request at a time through
 * hkv_find / hkv_insert_or_assign, oldest first, results copied back on
 * `stream` (the plain path).
 * Synchronous: returns when every request has completed; results[i] gets
 * the admission and completion times (seconds since the run started,
 * host clock, completion stamped by polling the request's event) and the
 * round that carried it. Find rows of misses are left unspecified.
 * hkv_serve_stats_get copies out where the last run spent its time; the
 * device-time fields are filled only while hkv_serve_profile(s, 1) is on,
 * which brackets every round with timing events (host time of their own,
 * so latency runs leave it off). */
typedef struct hkv_server_s *hkv_server_t;
typedef struct {
  double arrival_s;        /* seconds from the start of the run; non-decreasing */
  int32_t table;           /* index into the server's tables */
  int32_t op;              /* HKV_OP_FIND or HKV_OP_UPSERT */
  uint64_t n;              /* 1..ring_keys */
  const uint64_t *keys;    /* pinned host [n] */
  const float *values_in;  /* upsert: pinned host [n][dim] */
  float *values_out;       /* find: pinned host [n][dim] */
  uint8_t *flags;          /* pinned host [n] (found / status) or NULL */
} hkv_serve_request;
typedef struct {
  double admit_s;
  double done_s;
  uint64_t round;
} hkv_serve_result;
hkv_status hkv_serve_create(const hkv_table_t *tables, int n_tables, uint64_t ring_keys,
                            uint64_t hbm_budget_bytes, int max_inflight, hkv_server_t *out);
uint64_t hkv_serve_hbm_bytes(hkv_server_t s);
hkv_status hkv_serve_run(hkv_server_t s, const hkv_serve_request *reqs, uint64_t n_req,
                         int batched, int use_graph, hkv_serve_result *results,
                         hkv_stream_t stream);
typedef struct {
  double wall_s;          /* start of the run to its last completion */
  double host_admit_s;    /* host loop: admitting arrivals, issuing their input copies */
  double host_launch_s;   /* host loop: forming rounds, launching them, issuing copies back */
  double host_retire_s;   /* host loop: polling completion events, retiring requests */
  double idle_s;          /* host loop: yielding with nothing to do */
  double gpu_compute_s;   /* device time of the rounds' kernels on `stream` (profiling on) */
  double gpu_copy_out_s;  /* device time of the copies back to the host (profiling on) */
  uint64_t requests;
  uint64_t direct_rounds;   /* rounds run through one table's own call */
  uint64_t batched_rounds;  /* rounds run through hkv_batch_run */
  uint64_t loop_iterations;
  uint64_t h2d_bytes;       /* request keys and upsert rows copied in */
  uint64_t d2h_bytes;       /* find rows and flags copied back */
} hkv_serve_stats;
hkv_status hkv_serve_stats_get(hkv_server_t s, hkv_serve_stats *out);
hkv_status hkv_serve_profile(hkv_server_t s, int on);
hkv_status hkv_serve_destroy(hkv_server_t s);

/* Host-buffer pipeline (the paper has no host API; this is the library's
 * end-to-end path). A pipeline owns `depth` (2..8) staging slots in HBM,
 * each big enough for max_keys keys with rows of up to max_dim floats, and
 * three streams: copy-in, compute, copy-out. hkv_pipeline_find and
 * hkv_pipeline_insert_or_assign take HOST buffers, queue the host-to-device
 * copy of the inputs into the next slot, the table operation on the compute
 * stream (hkv_find / hkv_insert_or_assign, with their results, statuses and
 * table roles) and the device-to-host copy of the results, and return at
 * once. So operation k's input copy overlaps operation k-1's kernels and
 * operation k-2's result copy; a slot is reused only after its previous
 * results reached the host. Operations run in call order, also across
 * tables. Host buffers must stay valid and untouched until
 * hkv_pipeline_sync returns; page-locked memory (cudaHostAlloc or
 * cudaHostRegister) is needed for the copies to overlap, pageable memory
 * works but serialises them. Arguments: keys [n], values [n][dim] (find:
 * output, the rows of misses are zeros; upsert: input), found[n] /
 * status[n] (nullable), scores[n] (HKV_CUSTOM upserts, else NULL). An
 * upsert whose `values` the device can address (page-locked host memory
 * mapped into its address space, checked per call with
 * cudaPointerGetAttributes on the first and last byte) sends only the rows
 * the table can store: after dedup one kernel gathers the row of each
 * distinct key's last occurrence into the slot, so rows of duplicates never
 * cross the link; other host memory is copied whole. HKV_ERR_INVALID_ARG for n > max_keys, dim > max_dim or a null required
 * buffer; evictions are not reported. */
typedef struct hkv_pipeline_s *hkv_pipeline_t;
hkv_status hkv_pipeline_create(uint64_t max_keys, uint32_t max_dim, int depth,
                               hkv_pipeline_t *out);
hkv_status hkv_pipeline_find(hkv_pipeline_t p, hkv_table_t t, uint64_t n, const uint64_t *keys,
                             float *values, uint8_t *found);
hkv_status hkv_pipeline_insert_or_assign(hkv_pipeline_t p, hkv_table_t t, uint64_t n,
                                         const uint64_t *keys, const float *values,
                                         const uint64_t *scores, uint8_t *status);
/* Wait until every queued operation's results are in host memory. */
hkv_status hkv_pipeline_sync(hkv_pipeline_t p);
hkv_status hkv_pipeline_destroy(hkv_pipeline_t p);

/* Measurement hook. While enabled, every kernel the library launches for
 * this table is bracketed by two CUDA events recorded on the launching
 * stream. hkv_profile_read waits for those events and returns, per kernel
 * kind (HKV_K_*), the summed device time in ms (ms_out[HKV_KERNEL_KINDS])
 * and the number of launches (launches_out[HKV_KERNEL_KINDS]), both HOST
 * arrays, then forgets the records. */
enum {
  HKV_K_FIND = 0,
  HKV_K_DEDUP = 1,
  HKV_K_UPDATE = 2,
  HKV_K_INSERT = 3,     /* insert_or_assign's phase I; on tables without host
                           slices or ordered waves one cooperative launch that
                           also runs the reconcile and status passes, which
                           then record no launches of their own */
  HKV_K_RECONCILE = 4,
  HKV_K_STATUS = 5,     /* after the host-row pass of a tiered table: one
                           launch that also runs the reconcile pass */
  HKV_K_ERASE = 6,
  HKV_K_EXPORT = 7,
  HKV_K_SIZE = 8,
  HKV_K_HOSTROWS = 9,  /* tiered tables: host-memory rows grouped by region
                          and moved (find's host hits, upsert's deferred rows) */
  HKV_KERNEL_KINDS = 10
};
hkv_status hkv_profile_enable(hkv_table_t t, int on);
hkv_status hkv_profile_read(hkv_table_t t, double *ms_out, uint64_t *launches_out);

/* Random-access rate of device memory (a measurement hook; the paper has
 * none). Hash-table kernels touch scattered lines and sectors, whose rate
 * HBM bounds well below its sequential copy bandwidth; this is the ceiling
 * their roofline is read against. Touches `accesses` uniformly random,
 * naturally aligned units of unit_bytes (8, 32 or 128) in a scratch buffer
 * of buffer_bytes (a multiple of 128, at least 1 MiB; allocated and freed
 * here, and far above L2 for a meaningful number; the units used span the
 * largest power of two of them that fits), reading (write = 0) or
 * writing (write = 1) each, with 8 independent accesses in flight per
 * thread, and stores the best of `repeats` timed launches in
 * *accesses_per_s (host). Synchronous, on the current device.
 * HKV_ERR_INVALID_ARG for other arguments, HKV_ERR_OOM if the buffer cannot
 * be allocated. */
hkv_status hkv_measure_random_access(uint32_t unit_bytes, int write, uint64_t buffer_bytes,
                                     uint64_t accesses, int repeats, double *accesses_per_s);

/* Message of the calling thread's last error ("" if none). */
const char *hkv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HKV_H */
