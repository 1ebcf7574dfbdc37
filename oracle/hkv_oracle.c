/*
 * Plain CPU oracle of the HierarchicalKV hot path (arxiv 2603.17168).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code with the CUDA library.
 *
 * It executes the paper's algorithms literally, one key at a time, single
 * threaded, on a table that is a list of <= S entries per bucket:
 *   - Algorithm 1 (digest-accelerated find), Sec. 3.2;
 *   - Algorithm 2 (upsert with bucket-local admission and eviction), Sec. 3.3;
 *   - Algorithm 3 (score-based dual-bucket upsert), Sec. 3.4;
 *   - the reader / updater / inserter API roles of Sec. 3.5 (assign, erase,
 *     contains, size, export);
 *   - find_or_insert, the cold-start primitive of Sec. 4.1.
 * Slot positions are not modelled: no observable result depends on them.
 *
 * Readings of points the paper leaves open (hash, digest bits, tie order,
 * batch semantics) are stated at each function. The batch semantics are:
 *   1. duplicates in a batch collapse to one entry per key: the value of the
 *      last occurrence, and the multiplicity m;
 *   2. the table step advances by one per score-writing call;
 *   3. phase U: keys resident at batch start are updated in place;
 *   4. phase I: the other keys run Algorithm 2 (or 3) in ascending order of
 *      their last occurrence in the batch;
 *   5. a key's status follows from where it ends up: UPDATED if it was
 *      resident at batch start, INSERTED if resident at batch end, REJECTED
 *      otherwise; the evicted output lists the keys resident at batch start
 *      that are gone at batch end.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OT_S 128u                       /* slots per bucket, Sec. 3.2 */
#define OT_EMPTY_KEY UINT64_MAX         /* reserved: empty slot sentinel */
#define OT_LOCKED_KEY (UINT64_MAX - 1)  /* reserved: slot lock sentinel */
#define OT_FIRST_RESERVED (1ull << 63)  /* keys >= 2^63 are refused */
#define OT_H2_SALT 0x9E3779B97F4A7C15ull

enum { OT_OK = 0, OT_ERR_INVALID_ARG = 1, OT_ERR_RESERVED_KEY = 2,
       OT_ERR_DUPLICATE_KEY = 3, OT_ERR_OOM = 4 };
enum { OT_LRU = 0, OT_LFU = 1, OT_EPOCH_LRU = 2, OT_EPOCH_LFU = 3,
       OT_CUSTOM = 4, OT_CUSTOM_TS_FREQ = 5 };
enum { OT_ST_UPDATED = 1, OT_ST_INSERTED = 2, OT_ST_REJECTED = 3 };

typedef struct {
  uint64_t B;        /* bucket count, a power of two */
  uint32_t dim;      /* fp32 elements per value */
  int policy;
  int dual;
  uint64_t step;     /* advanced once per insert_or_assign / assign call */
  uint64_t epoch;    /* caller-set epoch / timestamp */
  uint32_t *count;   /* [B] entries in use */
  uint64_t *keys;    /* [B][S] */
  uint64_t *scores;  /* [B][S] */
  uint8_t *digest;   /* [B][S] */
  uint8_t *fresh;    /* [B][S] 1 while the entry was inserted by the current batch */
  float *values;     /* [B][S][dim] */
  uint64_t key_compares; /* full-key comparisons made by find (Prop. 1) */
} ot_table;

/* ---------------------------------------------------------------- hashing */

/* MurmurHash3's 64-bit finaliser (fmix64), written from its published
 * description: xor-shift by 33, multiply, xor-shift, multiply, xor-shift.
 * The paper names "a GPU-optimized hash derived from Murmur3" (Sec. 3.2)
 * without giving it; this finaliser is our reading. */
uint64_t ot_fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

/* Bucket of a key: Hash(k) mod B (Algorithm 1). */
static uint64_t bucket1(const ot_table *t, uint64_t key) {
  return ot_fmix64(key) % t->B;
}

/* Second candidate bucket for dual mode, from an independent hash
 * (Sec. 3.4, Algorithm 3): the finaliser of the key xor a fixed odd salt. */
static uint64_t bucket2(const ot_table *t, uint64_t key) {
  return ot_fmix64(key ^ OT_H2_SALT) % t->B;
}

/* 8-bit digest: bits 32..39 of the hash (Sec. 3.2). The value 0 marks an
 * empty slot in the digest line, so a real digest of 0 is stored as 1. */
static uint8_t digest_of(uint64_t key) {
  uint8_t d = (uint8_t)(ot_fmix64(key) >> 32);
  return d == 0 ? 1 : d;
}

void ot_map_keys(uint64_t B, int dual, uint64_t n, const uint64_t *keys,
                 uint64_t *b1, uint64_t *b2, uint8_t *dg) {
  ot_table t;
  memset(&t, 0, sizeof t);
  t.B = B;
  for (uint64_t i = 0; i < n; ++i) {
    if (b1) b1[i] = bucket1(&t, keys[i]);
    if (b2) b2[i] = dual ? bucket2(&t, keys[i]) : bucket1(&t, keys[i]);
    if (dg) dg[i] = digest_of(keys[i]);
  }
}

/* ------------------------------------------------------------ table state */

static uint64_t at(uint64_t b, uint32_t j) { return b * OT_S + j; }

ot_table *ot_create(uint64_t B, uint32_t dim, int policy, int dual) {
  if (B == 0 || (B & (B - 1)) != 0 || dim == 0 || policy < OT_LRU ||
      policy > OT_CUSTOM_TS_FREQ)
    return NULL;
  ot_table *t = (ot_table *)calloc(1, sizeof *t);
  if (!t) return NULL;
  t->B = B;
  t->dim = dim;
  t->policy = policy;
  t->dual = dual ? 1 : 0;
  t->count = (uint32_t *)calloc(B, sizeof *t->count);
  t->keys = (uint64_t *)malloc(B * OT_S * sizeof *t->keys);
  t->scores = (uint64_t *)calloc(B * OT_S, sizeof *t->scores);
  t->digest = (uint8_t *)calloc(B * OT_S, 1);
  t->fresh = (uint8_t *)calloc(B * OT_S, 1);
  t->values = (float *)calloc(B * OT_S * (uint64_t)dim, sizeof(float));
  if (!t->count || !t->keys || !t->scores || !t->digest || !t->fresh || !t->values) {
    free(t->count); free(t->keys); free(t->scores); free(t->digest);
    free(t->fresh); free(t->values); free(t);
    return NULL;
  }
  for (uint64_t i = 0; i < B * OT_S; ++i) t->keys[i] = OT_EMPTY_KEY;
  return t;
}

void ot_destroy(ot_table *t) {
  if (!t) return;
  free(t->count); free(t->keys); free(t->scores); free(t->digest);
  free(t->fresh); free(t->values); free(t);
}

void ot_set_step(ot_table *t, uint64_t s) { t->step = s; }
uint64_t ot_get_step(const ot_table *t) { return t->step; }
void ot_set_epoch(ot_table *t, uint64_t e) { t->epoch = e; }
uint64_t ot_key_compares(const ot_table *t) { return t->key_compares; }
void ot_reset_key_compares(ot_table *t) { t->key_compares = 0; }

uint64_t ot_size(const ot_table *t) {
  uint64_t s = 0;
  for (uint64_t b = 0; b < t->B; ++b) s += t->count[b];
  return s;
}

uint32_t ot_bucket_count(const ot_table *t, uint64_t b) { return t->count[b]; }

/* Algorithm 1 on one bucket: compare the digest of every slot in use, and
 * the full key only where the digest matches. Returns the slot or -1. */
static int32_t probe_bucket(ot_table *t, uint64_t b, uint64_t key, uint8_t d) {
  for (uint32_t j = 0; j < t->count[b]; ++j) {
    if (t->digest[at(b, j)] != d) continue;
    t->key_compares++;
    if (t->keys[at(b, j)] == key) return (int32_t)j;
  }
  return -1;
}

/* Locate a key in its candidate bucket(s): b1 first, then b2 in dual mode. */
static int locate(ot_table *t, uint64_t key, uint64_t *b_out, uint32_t *j_out) {
  uint8_t d = digest_of(key);
  uint64_t b1 = bucket1(t, key);
  int32_t j = probe_bucket(t, b1, key, d);
  if (j >= 0) { *b_out = b1; *j_out = (uint32_t)j; return 1; }
  if (t->dual) {
    uint64_t b2 = bucket2(t, key);
    if (b2 != b1) {
      j = probe_bucket(t, b2, key, d);
      if (j >= 0) { *b_out = b2; *j_out = (uint32_t)j; return 1; }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ reads */

/* find (Algorithm 1): a hit copies the value (and score); a miss leaves
 * values_out[i] untouched and sets found[i] = 0. Readers never write scores
 * (Sec. 3.5, readers group). */
void ot_find(ot_table *t, uint64_t n, const uint64_t *keys, float *values_out,
             uint8_t *found, uint64_t *scores_out) {
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t b; uint32_t j;
    int hit = keys[i] < OT_FIRST_RESERVED && locate(t, keys[i], &b, &j);
    if (found) found[i] = (uint8_t)hit;
    if (!hit) continue;
    if (values_out)
      memcpy(values_out + i * t->dim, t->values + at(b, j) * t->dim,
             t->dim * sizeof(float));
    if (scores_out) scores_out[i] = t->scores[at(b, j)];
  }
}

void ot_contains(ot_table *t, uint64_t n, const uint64_t *keys, uint8_t *found) {
  ot_find(t, n, keys, NULL, found, NULL);
}

/* --------------------------------------------------------- batch handling */

typedef struct { uint64_t key; uint64_t idx; } kv_idx;

static int cmp_key_idx(const void *a, const void *b) {
  const kv_idx *x = (const kv_idx *)a, *y = (const kv_idx *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

typedef struct {
  uint64_t key;
  uint64_t last;     /* index of the last occurrence in the batch */
  uint64_t mult;     /* multiplicity m in the batch */
  int resident0;     /* resident at batch start */
  uint8_t status;
} uniq_t;

static int cmp_uniq_last(const void *a, const void *b) {
  const uniq_t *x = (const uniq_t *)a, *y = (const uniq_t *)b;
  return x->last < y->last ? -1 : (x->last > y->last);
}

static int cmp_uniq_key(const void *a, const void *b) {
  const uniq_t *x = (const uniq_t *)a, *y = (const uniq_t *)b;
  return x->key < y->key ? -1 : (x->key > y->key);
}

/* Collapse a batch to one record per key (last occurrence, multiplicity),
 * returned in ascending order of the last occurrence. */
static uniq_t *dedup(uint64_t n, const uint64_t *keys, uint64_t *nu_out) {
  kv_idx *p = (kv_idx *)malloc((n ? n : 1) * sizeof *p);
  uniq_t *u = (uniq_t *)calloc(n ? n : 1, sizeof *u);
  if (!p || !u) { free(p); free(u); return NULL; }
  for (uint64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].idx = i; }
  qsort(p, n, sizeof *p, cmp_key_idx);
  uint64_t nu = 0;
  for (uint64_t i = 0; i < n;) {
    uint64_t r = i;
    while (r + 1 < n && p[r + 1].key == p[i].key) ++r;
    u[nu].key = p[i].key;
    u[nu].last = p[r].idx;
    u[nu].mult = r - i + 1;
    ++nu;
    i = r + 1;
  }
  free(p);
  qsort(u, nu, sizeof *u, cmp_uniq_last);
  *nu_out = nu;
  return u;
}

static uint64_t sat_add(uint64_t a, uint64_t b, uint64_t cap) {
  return (a > cap - (b < cap ? b : cap)) ? cap : a + b;
}

/* Score of a key under the table's policy (Sec. 3.3 "Scoring policies").
 * The paper names the policies but gives no formulas; our readings:
 *   LRU        the table step of this call, for new and updated keys;
 *   LFU        new: m; hit: old + m (saturating);
 *   EPOCH_LRU  (epoch << 32) | low 32 bits of the step;
 *   EPOCH_LFU  (epoch << 32) | saturating 32-bit count;
 *   CUSTOM     the caller's score for the last occurrence, verbatim;
 *   TS_FREQ    (epoch << 16) | saturating 16-bit count, epoch = timestamp. */
static uint64_t policy_score(const ot_table *t, int hit, uint64_t old, uint64_t m,
                             int have_caller, uint64_t caller) {
  switch (t->policy) {
    case OT_LRU:
      return t->step;
    case OT_LFU:
      return hit ? sat_add(old, m, UINT64_MAX) : m;
    case OT_EPOCH_LRU:
      return (t->epoch << 32) | (t->step & 0xFFFFFFFFull);
    case OT_EPOCH_LFU: {
      uint64_t f = hit ? sat_add(old & 0xFFFFFFFFull, m, 0xFFFFFFFFull)
                       : (m < 0xFFFFFFFFull ? m : 0xFFFFFFFFull);
      return (t->epoch << 32) | f;
    }
    case OT_CUSTOM:
      return have_caller ? caller : old;
    case OT_CUSTOM_TS_FREQ: {
      uint64_t f = hit ? sat_add(old & 0xFFFFull, m, 0xFFFFull)
                       : (m < 0xFFFFull ? m : 0xFFFFull);
      return (t->epoch << 16) | f;
    }
  }
  return 0;
}

/* (score, key) lexicographic order: the admission and victim order. The
 * paper compares scores only, with contradictory tie rules (Algorithm 2
 * admits on s = min, Algorithm 3 rejects); with the key as tie-break no two
 * entries are equal, so every decision is strict. */
static int sk_less(uint64_t s1, uint64_t k1, uint64_t s2, uint64_t k2) {
  return s1 < s2 || (s1 == s2 && k1 < k2);
}

/* Slot of the minimum (score, key) in a full bucket (Algorithm 2: argmin). */
static uint32_t min_slot(const ot_table *t, uint64_t b) {
  uint32_t m = 0;
  for (uint32_t j = 1; j < t->count[b]; ++j)
    if (sk_less(t->scores[at(b, j)], t->keys[at(b, j)], t->scores[at(b, m)],
                t->keys[at(b, m)]))
      m = j;
  return m;
}

typedef struct {
  uint64_t *keys, *scores;
  float *values;
  uint64_t n;
} evict_out;

static void write_slot(ot_table *t, uint64_t b, uint32_t j, uint64_t key, uint64_t s,
                       const float *v) {
  t->keys[at(b, j)] = key;
  t->scores[at(b, j)] = s;
  t->digest[at(b, j)] = digest_of(key);
  t->fresh[at(b, j)] = 1;
  memcpy(t->values + at(b, j) * t->dim, v, t->dim * sizeof(float));
}

/* Record the entry in slot (b, j) as evicted if it was resident at batch
 * start; an entry inserted by this same batch and displaced again is not an
 * eviction (its key ends up REJECTED). */
static void note_victim(const ot_table *t, uint64_t b, uint32_t j, evict_out *ev) {
  if (t->fresh[at(b, j)]) return;
  if (ev->keys) ev->keys[ev->n] = t->keys[at(b, j)];
  if (ev->scores) ev->scores[ev->n] = t->scores[at(b, j)];
  if (ev->values)
    memcpy(ev->values + ev->n * t->dim, t->values + at(b, j) * t->dim,
           t->dim * sizeof(float));
  ev->n++;
}

/* Algorithm 2 from the free-slot test on (the probe already missed): insert
 * into a free slot, else admit iff (s, k) beats the bucket minimum and
 * replace that minimum. */
static void upsert_single(ot_table *t, uint64_t b, uint64_t key, uint64_t s,
                          const float *v, evict_out *ev) {
  if (t->count[b] < OT_S) {
    write_slot(t, b, t->count[b], key, s, v);
    t->count[b]++;
    return;
  }
  uint32_t m = min_slot(t, b);
  if (!sk_less(t->scores[at(b, m)], t->keys[at(b, m)], s, key)) return; /* rejected */
  note_victim(t, b, m, ev);
  write_slot(t, b, m, key, s, v);
}

/* Algorithm 3: phase D1 while either candidate has a free slot (the less
 * occupied one, b1 on equal occupancy); phase D2 when both are full (evict
 * in the bucket holding the lower minimum, admit iff (s, k) beats it). */
static void upsert_dual(ot_table *t, uint64_t key, uint64_t s, const float *v,
                        evict_out *ev) {
  uint64_t b1 = bucket1(t, key), b2 = bucket2(t, key);
  if (b1 == b2) { upsert_single(t, b1, key, s, v, ev); return; }
  uint32_t o1 = t->count[b1], o2 = t->count[b2];
  if (o1 < OT_S || o2 < OT_S) {
    uint64_t b = (o1 <= o2) ? b1 : b2;
    write_slot(t, b, t->count[b], key, s, v);
    t->count[b]++;
    return;
  }
  uint32_t m1 = min_slot(t, b1), m2 = min_slot(t, b2);
  uint64_t bs = b1;
  uint32_t ms = m1;
  if (sk_less(t->scores[at(b2, m2)], t->keys[at(b2, m2)], t->scores[at(b1, m1)],
              t->keys[at(b1, m1)])) {
    bs = b2;
    ms = m2;
  }
  if (!sk_less(t->scores[at(bs, ms)], t->keys[at(bs, ms)], s, key)) return; /* rejected */
  note_victim(t, bs, ms, ev);
  write_slot(t, bs, ms, key, s, v);
}

static int validate_keys(uint64_t n, const uint64_t *keys) {
  for (uint64_t i = 0; i < n; ++i)
    if (keys[i] >= OT_FIRST_RESERVED) return OT_ERR_RESERVED_KEY;
  return OT_OK;
}

/* Phase U shared by both upsert formulations and by assign: update every
 * key resident at batch start in place. */
static void phase_u(ot_table *t, uniq_t *u, uint64_t nu, const float *values,
                    const uint64_t *scores) {
  for (uint64_t q = 0; q < nu; ++q) {
    uint64_t b; uint32_t j;
    u[q].resident0 = locate(t, u[q].key, &b, &j);
    if (!u[q].resident0) continue;
    uint64_t x = at(b, j);
    t->scores[x] = policy_score(t, 1, t->scores[x], u[q].mult, scores != NULL,
                                scores ? scores[u[q].last] : 0);
    if (values)
      memcpy(t->values + x * t->dim, values + u[q].last * t->dim, t->dim * sizeof(float));
    u[q].status = OT_ST_UPDATED;
  }
}

/* Statuses from final residency, broadcast to every occurrence, then clear
 * the per-batch "fresh" marks. */
static void finish_batch(ot_table *t, uniq_t *u, uint64_t nu, uint64_t n,
                         const uint64_t *keys, uint8_t *status_out) {
  for (uint64_t q = 0; q < nu; ++q) {
    uint64_t b; uint32_t j;
    if (u[q].resident0) continue;
    u[q].status = locate(t, u[q].key, &b, &j) ? OT_ST_INSERTED : OT_ST_REJECTED;
  }
  if (status_out) {
    qsort(u, nu, sizeof *u, cmp_uniq_key);
    for (uint64_t i = 0; i < n; ++i) {
      uniq_t probe = {keys[i], 0, 0, 0, 0};
      uniq_t *hit = (uniq_t *)bsearch(&probe, u, nu, sizeof *u, cmp_uniq_key);
      status_out[i] = hit->status;
    }
  }
  memset(t->fresh, 0, t->B * OT_S);
}

/* Deterministic mode takes duplicate-free batches only. */
static int check_dups(uint64_t nu, uint64_t n, int deterministic) {
  return (deterministic && nu != n) ? OT_ERR_DUPLICATE_KEY : OT_OK;
}

/* insert_or_assign of a batch, literal form: phase U, then Algorithm 2 (or
 * Algorithm 3 in dual mode) for each new key in ascending order of its last
 * occurrence. scores may be NULL unless the policy is CUSTOM.
 * Returns the number of evicted entries through *n_evicted. */
int ot_insert_or_assign(ot_table *t, uint64_t n, const uint64_t *keys,
                        const float *values, const uint64_t *scores, int deterministic,
                        uint8_t *status_out, uint64_t *ev_keys, uint64_t *ev_scores,
                        float *ev_values, uint64_t *n_evicted) {
  if (n_evicted) *n_evicted = 0;
  if (t->policy == OT_CUSTOM && !scores && n) return OT_ERR_INVALID_ARG;
  int rc = validate_keys(n, keys);
  if (rc) return rc;
  if (n == 0) return OT_OK;
  uint64_t nu;
  uniq_t *u = dedup(n, keys, &nu);
  if (!u) return OT_ERR_OOM;
  rc = check_dups(nu, n, deterministic);
  if (rc) { free(u); return rc; }
  t->step++;
  phase_u(t, u, nu, values, scores);
  evict_out ev = {ev_keys, ev_scores, ev_values, 0};
  for (uint64_t q = 0; q < nu; ++q) {
    if (u[q].resident0) continue;
    uint64_t s = policy_score(t, 0, 0, u[q].mult, scores != NULL,
                              scores ? scores[u[q].last] : 0);
    const float *v = values + u[q].last * t->dim;
    if (t->dual)
      upsert_dual(t, u[q].key, s, v, &ev);
    else
      upsert_single(t, bucket1(t, u[q].key), u[q].key, s, v, &ev);
  }
  finish_batch(t, u, nu, n, keys, status_out);
  if (n_evicted) *n_evicted = ev.n;
  free(u);
  return OT_OK;
}

/* find_or_insert of a batch (the cold-start primitive of Sec. 4.1): a key
 * resident at batch start keeps its value and has its score updated as an
 * access (phase U without the value write); every other key is inserted
 * with the value of its last occurrence under the same rules as
 * insert_or_assign. Then each row of values_io becomes the key's value in
 * the table, or stays the caller's row for a key the table refused;
 * found_out[i] = 1 iff the key was resident at batch start. */
int ot_find_or_insert(ot_table *t, uint64_t n, const uint64_t *keys, float *values_io,
                      const uint64_t *scores, uint8_t *found_out) {
  if (t->policy == OT_CUSTOM && !scores && n) return OT_ERR_INVALID_ARG;
  int rc = validate_keys(n, keys);
  if (rc) return rc;
  if (n == 0) return OT_OK;
  uint64_t nu;
  uniq_t *u = dedup(n, keys, &nu);
  if (!u) return OT_ERR_OOM;
  t->step++;
  phase_u(t, u, nu, NULL, scores);
  evict_out ev = {NULL, NULL, NULL, 0};
  for (uint64_t q = 0; q < nu; ++q) {
    if (u[q].resident0) continue;
    uint64_t s = policy_score(t, 0, 0, u[q].mult, scores != NULL,
                              scores ? scores[u[q].last] : 0);
    const float *v = values_io + u[q].last * t->dim;
    if (t->dual)
      upsert_dual(t, u[q].key, s, v, &ev);
    else
      upsert_single(t, bucket1(t, u[q].key), u[q].key, s, v, &ev);
  }
  if (found_out) {
    qsort(u, nu, sizeof *u, cmp_uniq_key);
    for (uint64_t i = 0; i < n; ++i) {
      uniq_t probe = {keys[i], 0, 0, 0, 0};
      uniq_t *hit = (uniq_t *)bsearch(&probe, u, nu, sizeof *u, cmp_uniq_key);
      found_out[i] = hit->resident0 ? 1 : 0;
    }
  }
  memset(t->fresh, 0, t->B * OT_S);
  free(u);
  /* rows from the table: every key resident now, in every occurrence */
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t b; uint32_t j;
    if (locate(t, keys[i], &b, &j))
      memcpy(values_io + i * t->dim, t->values + at(b, j) * t->dim, t->dim * sizeof(float));
  }
  return OT_OK;
}

/* ------------------------------------------- closed-form single-bucket form */

typedef struct {
  uint64_t key, score;
  const float *v;    /* value source */
  int resident0;
} cand_t;

static int cmp_cand_desc(const void *a, const void *b) {
  const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
  if (sk_less(x->score, x->key, y->score, y->key)) return 1;
  if (sk_less(y->score, y->key, x->score, x->key)) return -1;
  return 0;
}

/* Second, independent formulation of single-bucket phase I: each bucket
 * keeps the S largest (score, key) pairs among its entries after phase U
 * and the batch's new keys that map to it. Streaming Algorithm 2 over any
 * order of the new keys reaches exactly this set, because "insert if free,
 * else replace the minimum iff larger" keeps a bucket equal to the top S of
 * everything seen so far. Single-bucket tables only. */
int ot_insert_or_assign_topk(ot_table *t, uint64_t n, const uint64_t *keys,
                             const float *values, const uint64_t *scores,
                             int deterministic, uint8_t *status_out, uint64_t *ev_keys,
                             uint64_t *ev_scores, float *ev_values, uint64_t *n_evicted) {
  if (n_evicted) *n_evicted = 0;
  if (t->dual) return OT_ERR_INVALID_ARG;
  if (t->policy == OT_CUSTOM && !scores && n) return OT_ERR_INVALID_ARG;
  int rc = validate_keys(n, keys);
  if (rc) return rc;
  if (n == 0) return OT_OK;
  uint64_t nu;
  uniq_t *u = dedup(n, keys, &nu);
  if (!u) return OT_ERR_OOM;
  rc = check_dups(nu, n, deterministic);
  if (rc) { free(u); return rc; }
  t->step++;
  phase_u(t, u, nu, values, scores);

  /* group the new keys by bucket: counting sort on the bucket index */
  uint64_t *start = (uint64_t *)calloc(t->B + 1, sizeof *start);
  uint64_t *order = (uint64_t *)malloc((nu ? nu : 1) * sizeof *order);
  cand_t *c = (cand_t *)malloc((OT_S + nu) * sizeof *c);
  float *vbuf = (float *)malloc((uint64_t)OT_S * t->dim * sizeof(float));
  if (!start || !order || !c || !vbuf) {
    free(start); free(order); free(c); free(vbuf); free(u);
    return OT_ERR_OOM;
  }
  for (uint64_t q = 0; q < nu; ++q)
    if (!u[q].resident0) start[bucket1(t, u[q].key) + 1]++;
  for (uint64_t b = 0; b < t->B; ++b) start[b + 1] += start[b];
  uint64_t *fill = (uint64_t *)malloc((t->B ? t->B : 1) * sizeof *fill);
  if (!fill) { free(start); free(order); free(c); free(vbuf); free(u); return OT_ERR_OOM; }
  memcpy(fill, start, t->B * sizeof *fill);
  for (uint64_t q = 0; q < nu; ++q)
    if (!u[q].resident0) order[fill[bucket1(t, u[q].key)]++] = q;
  free(fill);

  evict_out ev = {ev_keys, ev_scores, ev_values, 0};
  for (uint64_t b = 0; b < t->B; ++b) {
    if (start[b] == start[b + 1]) continue;
    uint64_t nc = 0;
    /* snapshot resident values: the rebuild below overwrites the slots */
    memcpy(vbuf, t->values + at(b, 0) * t->dim, (uint64_t)t->count[b] * t->dim * sizeof(float));
    for (uint32_t j = 0; j < t->count[b]; ++j) {
      c[nc].key = t->keys[at(b, j)];
      c[nc].score = t->scores[at(b, j)];
      c[nc].v = vbuf + (uint64_t)j * t->dim;
      c[nc].resident0 = 1;
      nc++;
    }
    for (uint64_t p = start[b]; p < start[b + 1]; ++p) {
      uniq_t *q = &u[order[p]];
      c[nc].key = q->key;
      c[nc].score = policy_score(t, 0, 0, q->mult, scores != NULL, scores ? scores[q->last] : 0);
      c[nc].v = values + q->last * t->dim;
      c[nc].resident0 = 0;
      nc++;
    }
    qsort(c, nc, sizeof *c, cmp_cand_desc);
    uint32_t keep = nc < OT_S ? (uint32_t)nc : OT_S;
    for (uint64_t r = keep; r < nc; ++r) {
      if (!c[r].resident0) continue;
      if (ev.keys) ev.keys[ev.n] = c[r].key;
      if (ev.scores) ev.scores[ev.n] = c[r].score;
      if (ev.values) memcpy(ev.values + ev.n * t->dim, c[r].v, t->dim * sizeof(float));
      ev.n++;
    }
    /* values of kept residents must be copied from the snapshot before any
     * slot is overwritten: stage them in candidate order */
    float *stage = (float *)malloc((uint64_t)keep * t->dim * sizeof(float));
    if (!stage) { free(start); free(order); free(c); free(vbuf); free(u); return OT_ERR_OOM; }
    for (uint32_t r = 0; r < keep; ++r)
      memcpy(stage + (uint64_t)r * t->dim, c[r].v, t->dim * sizeof(float));
    for (uint32_t r = 0; r < keep; ++r) {
      t->keys[at(b, r)] = c[r].key;
      t->scores[at(b, r)] = c[r].score;
      t->digest[at(b, r)] = digest_of(c[r].key);
      memcpy(t->values + at(b, r) * t->dim, stage + (uint64_t)r * t->dim,
             t->dim * sizeof(float));
    }
    free(stage);
    for (uint32_t r = keep; r < OT_S; ++r) {
      t->keys[at(b, r)] = OT_EMPTY_KEY;
      t->digest[at(b, r)] = 0;
      t->scores[at(b, r)] = 0;
    }
    t->count[b] = keep;
  }
  finish_batch(t, u, nu, n, keys, status_out);
  if (n_evicted) *n_evicted = ev.n;
  free(start); free(order); free(c); free(vbuf); free(u);
  return OT_OK;
}

/* ---------------------------------------------------- updaters, inserters */

/* assign (updater, Sec. 3.5): phase U only; keys not resident are ignored.
 * scores may be NULL (CUSTOM then keeps the old score). */
int ot_assign(ot_table *t, uint64_t n, const uint64_t *keys, const float *values,
              const uint64_t *scores) {
  int rc = validate_keys(n, keys);
  if (rc) return rc;
  if (n == 0) return OT_OK;
  uint64_t nu;
  uniq_t *u = dedup(n, keys, &nu);
  if (!u) return OT_ERR_OOM;
  t->step++;
  phase_u(t, u, nu, values, scores);
  free(u);
  return OT_OK;
}

/* erase (inserter, Sec. 3.5): remove each key that is resident. With no
 * probe chains, an emptied slot needs no tombstone. */
int ot_erase(ot_table *t, uint64_t n, const uint64_t *keys) {
  int rc = validate_keys(n, keys);
  if (rc) return rc;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t b; uint32_t j;
    if (!locate(t, keys[i], &b, &j)) continue;
    uint32_t last = t->count[b] - 1;
    if (j != last) {
      t->keys[at(b, j)] = t->keys[at(b, last)];
      t->scores[at(b, j)] = t->scores[at(b, last)];
      t->digest[at(b, j)] = t->digest[at(b, last)];
      memcpy(t->values + at(b, j) * t->dim, t->values + at(b, last) * t->dim,
             t->dim * sizeof(float));
    }
    t->keys[at(b, last)] = OT_EMPTY_KEY;
    t->digest[at(b, last)] = 0;
    t->scores[at(b, last)] = 0;
    t->count[b] = last;
  }
  return OT_OK;
}

/* ---------------------------------------------------------- export / load */

/* Every entry with its bucket; returns the number written (cap = room). */
uint64_t ot_export(const ot_table *t, uint64_t cap, uint64_t *keys, uint64_t *scores,
                   float *values, uint64_t *buckets) {
  uint64_t w = 0;
  for (uint64_t b = 0; b < t->B; ++b)
    for (uint32_t j = 0; j < t->count[b] && w < cap; ++j, ++w) {
      if (keys) keys[w] = t->keys[at(b, j)];
      if (scores) scores[w] = t->scores[at(b, j)];
      if (values) memcpy(values + w * t->dim, t->values + at(b, j) * t->dim,
                         t->dim * sizeof(float));
      if (buckets) buckets[w] = b;
    }
  return w;
}

/* Place entries into given buckets (a state read back from elsewhere). Each
 * bucket must be one of the key's candidates, hold at most S entries, and no
 * key may appear twice. */
int ot_load(ot_table *t, uint64_t n, const uint64_t *keys, const uint64_t *scores,
            const float *values, const uint64_t *buckets) {
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t b = buckets[i], k = keys[i];
    if (k >= OT_FIRST_RESERVED || b >= t->B) return OT_ERR_INVALID_ARG;
    if (b != bucket1(t, k) && !(t->dual && b == bucket2(t, k))) return OT_ERR_INVALID_ARG;
    if (t->count[b] >= OT_S) return OT_ERR_INVALID_ARG;
    uint64_t bb; uint32_t jj;
    if (locate(t, k, &bb, &jj)) return OT_ERR_DUPLICATE_KEY;
    uint32_t j = t->count[b]++;
    t->keys[at(b, j)] = k;
    t->scores[at(b, j)] = scores ? scores[i] : 0;
    t->digest[at(b, j)] = digest_of(k);
    if (values) memcpy(t->values + at(b, j) * t->dim, values + i * t->dim,
                       t->dim * sizeof(float));
  }
  return OT_OK;
}

/* Minimum (score, key) of a bucket; returns 0 for an empty bucket. */
int ot_bucket_min(const ot_table *t, uint64_t b, uint64_t *score, uint64_t *key) {
  if (t->count[b] == 0) return 0;
  uint32_t m = min_slot(t, b);
  *score = t->scores[at(b, m)];
  *key = t->keys[at(b, m)];
  return 1;
}
