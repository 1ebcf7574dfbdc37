// insert_or_assign / assign / erase (Algorithms 2 and 3, Sec. 3.3-3.4;
// updater and inserter groups of Sec. 3.5).
//
// A batch runs as a short pipeline on one stream:
//   dedup     collapse duplicate keys (last occurrence's value, multiplicity
//             m): per-block shared-memory hash aggregation, then a global
//             open-addressing table, so a Zipf-hot key costs one global
//             atomic per block instead of one per occurrence. The distinct
//             keys get dense indices u (one list reservation per block);
//   update    phase U: probe every distinct key (G lanes per key, digest
//             line + key confirm) and update residents in place. A miss
//             claims a free slot of the less occupied candidate bucket
//             (per-bucket occupancy counters, a CAS on the slot's digest
//             byte 0 -> digest); a miss whose buckets are all full is left
//             at its index u for phase I;
//   insert    phase I: a warp takes 32 consecutive u and runs a
//             warp-cooperative victim search for each full-bucket miss: the
//             minimum (score, key) over the 128 (256) slots, admission
//             control, a CAS lock on the victim, replacement (the
//             full-bucket branch of Algorithm 2, and Algorithm 3). The next
//             search's score and key lines are bulk-prefetched into L2;
//   reconcile a victim that was itself inserted by this batch is not an
//             eviction: its key becomes REJECTED and it is dropped from the
//             evicted output, which is compacted here;
//   status    broadcast each distinct key's status to all its occurrences.
// On the plain path insert, reconcile and status are one cooperative launch
// (insert_finish_kernel; finish_kernel, reconcile and status only, after the
// host-row pass of tiered tables).
// Phase U finishing before phase I starts is what guarantees, for real
// batches, that no in-place update of a resident runs while its slot is
// being evicted (the update/insert group separation of Sec. 3.5).
//
// Single-bucket claims are linearisable: while a bucket is full a slot's
// (score, key) only grows; a victim search that meets a locked slot among
// the minimum-score candidates re-reads instead of choosing around it; and
// the victim is locked with one 128-bit CAS on its (key, score) pair, which
// fails for a key and score read from two different occupants. Any serial
// order of "insert if free, else replace the minimum iff larger" ends with
// each bucket holding the largest 128 (score, key) pairs, so the
// single-bucket result does not depend on the schedule.
#include "hkv_internal.h"

namespace hkv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct DedupEntry {
  unsigned long long key;   // kEmptyKey when unused
  unsigned int nlast;       // ~(largest batch index of the key): atomicMin
  unsigned int cnt_m1;      // multiplicity - 1 (starts at 0xFFFFFFFF)
};
static_assert(sizeof(DedupEntry) == 16, "dedup entry layout");

enum : int {
  kCntUnique = 0,
  kCntEvOut = 1,
  kAbort = 2,
  kCntPending = 3,
  kCntInsCursor = 4,  // next 32-key chunk of phase I to hand out
  kCntDeferred = 5,   // keys phase U left to phase I (mflag != 0)
  kBarCount = 6,      // ordered phase I in one launch: grid barrier arrivals
  kBarGen = 7,        // and generation
  kCntPending2 = 8,   // pending keys of odd / even waves (kCntPending, this)
  kCntWords = 10
};

struct Scratch {
  DedupEntry* tab;
  uint64_t tab_mask;
  int tab_bits;
  uint8_t* tstatus;          // [T] status per dedup entry
  uint32_t* slot_of;         // [n] dedup entry of each batch position
  uint32_t* ulist;           // [n] dedup entry of distinct key u
  uint8_t* mflag;            // [n] 1 if distinct key u missed in phase U
  uint64_t* mkey;            // [n] key u (written by dedup for every distinct key)
  uint32_t* mi;              // [n] batch index of its last occurrence (misses)
  uint32_t* mm;              // [n] its multiplicity (misses)
  unsigned long long* cnt;   // [kCntWords]
  uint64_t* evk;             // [n] victim of distinct key u, kEmptyKey if none
  uint64_t* evs;             // [n] its score
  float* evv;                // [n][dim] its value, or null
  const OpDesc* d;           // batched rounds: size, buffers and score context
  unsigned long long* owner; // [B] ordered phase I: (wave, ~batch index) of
                             // each bucket's first pending key, or null
  int keep_hits;             // find_or_insert: residents keep their values
  int row_prefetch;          // input rows are in device memory: the insert
                             // phase may pull them into L2 by bulk prefetch
  uint64_t* gdefer;          // [n] phase I: host-memory slot taken by distinct
                             // key u whose row is written after the phase
                             // (kNoHostSlot if none), or null: rows now
  uint64_t host_slot0;       // first global slot whose row lives in host memory
};


__device__ __forceinline__ uint64_t dedup_pos(uint64_t key, int bits) {
  // top bits of a hash independent of the table's bucket bits
  return fmix64(key ^ 0xD6E8FEB86659FD93ull) >> (64 - bits);
}

__device__ __forceinline__ bool aborted(const Scratch& s) {
  return *reinterpret_cast<volatile unsigned long long*>(s.cnt + kAbort) != 0;
}

__device__ __forceinline__ void abort_batch(const Scratch& s, uint32_t* err, uint32_t code) {
  latch_error(err, code);
  atomicExch(s.cnt + kAbort, 1ull);
}

// ------------------------------------------------------------------- dedup

// A tile of 1024 keys per block, deduplicated in a shared table of 1536
// entries (load at most 2/3; 24 KiB). Blocks spend most of their life
// waiting on global atomics, so a batch whose tiles do not all fit at once
// pays a whole block lifetime for its second wave: batches of more than six
// tiles per SM (2^20 keys: 1024 blocks on 152 SMs) take an instantiation
// bounded to seven blocks per SM (32 registers), the others one bounded to
// six (40 registers, no spills, faster per block).
constexpr int kDedupThreads = 256;
constexpr int kDedupKPT = 4;
constexpr int kDedupTile = kDedupThreads * kDedupKPT;           // 1024 keys
constexpr int kDedupEntries = 1536;
constexpr int kDedupPerThread = kDedupEntries / kDedupThreads;  // 6
constexpr int kDedupSmem = kDedupEntries * (int)sizeof(DedupEntry);
constexpr int kDedupMergeGroup = 2;  // global-table attempts a thread has in flight
static_assert(kDedupTile / kDedupThreads <= 32, "dedup first-key mask");
static_assert(kDedupEntries % kDedupThreads == 0, "dedup table split");
// seven blocks' tables, static scratch (the entry list and scan words,
// under 3 KiB) and per-block reserve fit an SM's 228 KiB
static_assert(7 * (kDedupSmem + 3072 + 1024) <= 228 * 1024, "seven dedup blocks per SM");
static_assert(2 * kDedupEntries >= 3 * kDedupTile, "dedup table load");

// Exclusive prefix sum of count over the block's threads (kDedupThreads);
// *total receives the block's sum. Synchronises the block.
__device__ __forceinline__ unsigned block_scan_excl(unsigned count, unsigned* total) {
  constexpr int kWarps = kDedupThreads / 32;
  __shared__ unsigned wsum[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned incl = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  unsigned before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const unsigned c = wsum[w];
    before += w < wid ? c : 0u;
    tot += c;
  }
  *total = tot;
  return before + incl - count;
}

// Home slot of a key in the shared table: the top 32 bits of the key's hash
// scaled to [0, kDedupEntries).
__device__ __forceinline__ uint32_t dedup_smem_pos(uint64_t key) {
  return (uint32_t)((dedup_pos(key, 32) * (uint64_t)kDedupEntries) >> 32);
}

template <int MIN_BLOCKS>
__global__ void __launch_bounds__(kDedupThreads, MIN_BLOCKS)
    dedup_kernel(uint64_t n, const uint64_t* __restrict__ keys, Scratch s, TableDev t,
                 int deterministic) {
  extern __shared__ DedupEntry sm[];
  int tab_bits = s.tab_bits;
  uint64_t tab_mask = s.tab_mask;
  if (s.d) {  // grid sized for the batch object's largest round
    n = s.d->n;
    keys = s.d->keys;
    tab_bits = tab_bits_for(n);
    tab_mask = (1ull << tab_bits) - 1;
    if ((uint64_t)blockIdx.x * kDedupTile >= n) return;
  }
  for (int p = threadIdx.x; p < kDedupEntries; p += kDedupThreads) {
    sm[p].key = kEmptyKey;
    sm[p].nlast = 0xFFFFFFFFu;
    sm[p].cnt_m1 = 0xFFFFFFFFu;
  }
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * kDedupTile;
  int pos[kDedupKPT];
  uint64_t kin[kDedupKPT];  // all of the tile's loads in flight at once
#pragma unroll
  for (int j = 0; j < kDedupKPT; ++j) {
    const uint64_t idx = tile0 + (uint64_t)j * kDedupThreads + threadIdx.x;
    kin[j] = idx < n ? __ldg(keys + idx) : 0;
  }
#pragma unroll
  for (int j = 0; j < kDedupKPT; ++j) {
    pos[j] = -1;
    const uint64_t idx = tile0 + (uint64_t)j * kDedupThreads + threadIdx.x;
    if (idx >= n) continue;
    const uint64_t k = kin[j];
    if (k >= kFirstReserved) {
      abort_batch(s, t.err, HKV_ERR_RESERVED_KEY);
      continue;
    }
    uint32_t p = dedup_smem_pos(k);
    for (;;) {  // at most 1024 distinct keys in 1536 entries: terminates
      const unsigned long long old = atomicCAS(&sm[p].key, kEmptyKey, (unsigned long long)k);
      if (old == kEmptyKey || old == k) break;
      p = p + 1 == (uint32_t)kDedupEntries ? 0u : p + 1;
    }
    atomicMin(&sm[p].nlast, ~(uint32_t)idx);
    atomicAdd(&sm[p].cnt_m1, 1u);
    pos[j] = (int)p;
  }
  __syncthreads();
  // The occupied entries (one per distinct key of the tile, so at most
  // kDedupTile) as a dense list, so that each thread merges at most
  // kDedupMergeGroup of them per round of global round trips.
  __shared__ uint16_t occ[kDedupTile];
  unsigned mine = 0;
#pragma unroll
  for (int q = 0; q < kDedupPerThread; ++q)
    mine += sm[threadIdx.x + q * kDedupThreads].key != kEmptyKey ? 1u : 0u;
  unsigned nocc;
  unsigned o = block_scan_excl(mine, &nocc);
#pragma unroll
  for (int q = 0; q < kDedupPerThread; ++q) {
    const int p = threadIdx.x + q * kDedupThreads;
    if (sm[p].key != kEmptyKey) occ[o++] = (uint16_t)p;
  }
  __syncthreads();
  // Merge the listed keys into the global table. A thread's keys of a round
  // go together: their CAS attempts are issued at once (independent
  // addresses), and keys that met another key walk on in lockstep, one
  // round trip per step for all of them.
  unsigned nfirst = 0, firsts = 0;  // bit m: list item threadIdx.x + m * kDedupThreads
  for (unsigned r0 = 0; r0 < nocc; r0 += kDedupMergeGroup * kDedupThreads) {
    unsigned long long kq[kDedupMergeGroup], old[kDedupMergeGroup];
    uint64_t gq[kDedupMergeGroup];
    int pp[kDedupMergeGroup];
#pragma unroll
    for (int j = 0; j < kDedupMergeGroup; ++j) {
      const unsigned r = r0 + j * kDedupThreads + threadIdx.x;
      pp[j] = r < nocc ? (int)occ[r] : -1;
      kq[j] = pp[j] >= 0 ? sm[pp[j]].key : kEmptyKey;
      gq[j] = dedup_pos(kq[j], tab_bits);
      old[j] = kq[j] != kEmptyKey ? atomicCAS(&s.tab[gq[j]].key, kEmptyKey, kq[j]) : kEmptyKey;
    }
    // the table holds >= 2n entries: every walk ends
    for (;;) {
      bool walking = false;
#pragma unroll
      for (int j = 0; j < kDedupMergeGroup; ++j)
        if (old[j] != kEmptyKey && old[j] != kq[j]) {
          gq[j] = (gq[j] + 1) & tab_mask;
          old[j] = atomicCAS(&s.tab[gq[j]].key, kEmptyKey, kq[j]);
          walking = true;
        }
      if (!walking) break;
    }
#pragma unroll
    for (int j = 0; j < kDedupMergeGroup; ++j) {
      if (pp[j] < 0) continue;
      const int p = pp[j];
      const bool first = old[j] == kEmptyKey;
      const uint32_t c = sm[p].cnt_m1 + 1u;
      atomicMin(&s.tab[gq[j]].nlast, sm[p].nlast);
      atomicAdd(&s.tab[gq[j]].cnt_m1, c);
      if (deterministic && (!first || c > 1)) abort_batch(s, t.err, HKV_ERR_DUPLICATE_KEY);
      sm[p].cnt_m1 = (uint32_t)gq[j];  // reuse: global entry of this key
      if (first) {
        firsts |= 1u << (r0 / kDedupThreads + j);
        nfirst++;
      }
    }
  }
  // One list reservation per block for the keys this block saw first
  // (block_reserve also synchronises the block: the smem entries are final).
  unsigned long long u = block_reserve(s.cnt + kCntUnique, nfirst);
  for (int m = 0; m < kDedupTile / kDedupThreads; ++m)
    if (firsts & (1u << m)) {
      const int p = occ[threadIdx.x + m * kDedupThreads];
      s.ulist[u] = sm[p].cnt_m1;
      s.mkey[u] = sm[p].key;
      ++u;
    }
#pragma unroll
  for (int j = 0; j < kDedupKPT; ++j) {
    if (pos[j] < 0) continue;
    const uint64_t idx = tile0 + (uint64_t)j * kDedupThreads + threadIdx.x;
    s.slot_of[idx] = sm[pos[j]].cnt_m1;
  }
  const int which[1] = {HKV_CNT_UNIQUE};
  const unsigned vals[1] = {nfirst};
  flush_counts(t, which, vals);
}

// Publish a slot's key with a release store at GPU scope: every write the
// publishing thread has made, or has observed through a warp barrier (the
// other lanes' value stores), becomes visible before the key does.
__device__ __forceinline__ void publish_key(uint64_t* addr, uint64_t key) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(addr), "l"(key) : "memory");
}

// Compare-and-swap of a slot's whole (key, score) pair with one 128-bit
// atomic (sm_90 and later): succeeds iff the pair still equals
// (key_old, score_old), which then becomes (key_new, score_new).
__device__ __forceinline__ bool cas_pair(uint64_t* pair, uint64_t key_old, uint64_t score_old,
                                         uint64_t key_new, uint64_t score_new) {
  unsigned long long k, sc;
  asm volatile(
      "{\n\t.reg .b128 cmp, swp, old;\n\t"
      "mov.b128 cmp, {%2, %3};\n\t"
      "mov.b128 swp, {%4, %5};\n\t"
      "atom.relaxed.gpu.global.cas.b128 old, [%6], cmp, swp;\n\t"
      "mov.b128 {%0, %1}, old;\n\t}"
      : "=l"(k), "=l"(sc)
      : "l"(key_old), "l"(score_old), "l"(key_new), "l"(score_new), "l"(pair)
      : "memory");
  return k == key_old && sc == score_old;
}

// L2 prefetch of a contiguous range with one TMA bulk instruction
// (cp.async.bulk.prefetch.L2; size a multiple of 16 bytes).
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Slot of the first free digest (0) in a 16-slot piece of a digest line,
// or -1.
__device__ __forceinline__ int free_in_piece(const uint4& v) {
  const uint32_t z[4] = {__vcmpeq4(v.x, 0u), __vcmpeq4(v.y, 0u), __vcmpeq4(v.z, 0u),
                         __vcmpeq4(v.w, 0u)};
  int slot = -1;
#pragma unroll
  for (int j = 3; j >= 0; --j)
    if (z[j]) slot = j * 4 + ((__ffs(z[j]) - 1) >> 3);
  return slot;
}

// A free slot of a bucket, scanning its digest line through L2 two pieces
// (32 slots, one sector) per round trip from a key-dependent start, so that
// keys claiming in one bucket rarely race for the same slot. -1 if the line
// shows no free slot. `sectors` counts the 32-byte reads.
__device__ __forceinline__ int find_free(const uint8_t* line, unsigned start, unsigned& sectors) {
  const uint4* p = reinterpret_cast<const uint4*>(line);
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    const unsigned q0 = (start + 2 * r) & 6;  // sector-aligned pair of pieces
    const uint4 a = __ldcg(p + q0), b = __ldcg(p + q0 + 1);
    sectors++;
    int s = free_in_piece(a);
    if (s >= 0) return (int)q0 * 16 + s;
    s = free_in_piece(b);
    if (s >= 0) return (int)(q0 + 1) * 16 + s;
  }
  return -1;
}

// One thread writes (digest, score, value) into a slot it holds LOCKED and
// publishes the key (digest first: see fill_slot). RELEASE orders the
// digest, score and value stores before the key for readers in the same
// kernel that act on a published key's score or value (victim searches).
// Phase U has no such reader (no eviction runs beside it, probes of other
// keys never match this key) and the kernel boundary orders everything for
// the next phase, so its claims publish with a plain store.
template <bool VEC16, bool RELEASE>
__device__ __forceinline__ void fill_slot_thread(const TableDev& t, uint64_t g, uint64_t key,
                                                 uint64_t sc, uint32_t dg, const float* src) {
  t.digests[g] = (uint8_t)dg;
  __stcg(reinterpret_cast<unsigned long long*>(score_ptr(t, g)), (unsigned long long)sc);
  float* dst = value_ptr(t, g);
  if (VEC16) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (uint32_t j = 0; j < (t.dim >> 2); ++j) __stcg(d4 + j, __ldg(s4 + j));
  } else if (t.vec8 && (t.dim & 1) == 0 &&
             ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 7) == 0) {
    const float2* s2 = reinterpret_cast<const float2*>(src);
    float2* d2 = reinterpret_cast<float2*>(dst);
    for (uint32_t j = 0; j < (t.dim >> 1); ++j) __stcg(d2 + j, __ldg(s2 + j));
  } else {
    for (uint32_t j = 0; j < t.dim; ++j) __stcg(dst + j, __ldg(src + j));
  }
  if (RELEASE)
    publish_key(key_ptr(t, g), key);
  else
    __stcg(reinterpret_cast<unsigned long long*>(key_ptr(t, g)), (unsigned long long)key);
}

// Back-off before retry `attempt` (> 0): exponential up to ~16 us, with
// per-key jitter so colliding warps fall apart. With kMaxClaimAttempts
// retries a claim waits at most ~65 ms before it gives up.
__device__ __forceinline__ void claim_backoff(int attempt, uint64_t h) {
  const unsigned base = 32u << (attempt < 9 ? attempt : 9);
  __nanosleep(base + ((unsigned)(h >> 17) & 255u));
}

// Free-slot claim for one missing key, run by one thread (the free-slot
// branch of Algorithm 2; Algorithm 3 phase D1: a free slot of the less occupied
// candidate bucket, b1 on equal occupancy). Occupancy comes from the
// per-bucket counters, which count a slot from the moment its claim CAS
// succeeds, so a counter never exceeds the slots really taken: a counter at
// 128 means full, and a bucket whose counter lags behind its digests is
// simply scanned again. The thread takes the slot by setting its digest
// byte (claim_digest), then writes score and key; the caller's lane group
// then copies the value row into slot `g_out`
// (phase U has no reader of a claimed slot's value, and the kernel boundary
// orders the row before phase I). One thread storing a whole row issues
// half-sector stores to 32 rows per instruction, which cost the update
// kernel 40% of its time; a group's lanes write whole sectors. Returns 0
// when the key was placed (g_out = its global slot; or the bounded wait ran
// out, the error was latched and g_out = kNoSlot), 2 when every candidate
// bucket is full and the key needs a victim search.
constexpr uint64_t kNoSlot = ~0ull;

// Claim free slot g by setting its digest byte (0 -> dg) with a CAS on the
// 32-bit digest word. The probe has just read that line, so the atomic is
// an L2 hit, where a CAS on the slot's (key, score) sector waited on a DRAM
// read (update_kernel 5% faster). A slot with digest 0 holds the empty key
// between kernels (erase clears the key first, a fill sets the digest
// first), and no other group's kernels run beside an inserter's, so the
// byte alone decides the claim; keys are distinct after dedup, so a probe
// that meets a claimed slot whose key is not written yet compares unequal.
// At most three other claims can change the word, so the loop is bounded.
__device__ __forceinline__ bool claim_digest(const TableDev& t, uint64_t g, uint32_t dg) {
  unsigned int* word = reinterpret_cast<unsigned int*>(t.digests + (g & ~3ull));
  const int sh = (int)(g & 3ull) * 8;
  unsigned int old = __ldcg(word);
  for (int k = 0; k < 8; ++k) {
    if ((old >> sh) & 0xFFu) return false;
    const unsigned int prev = atomicCAS(word, old, old | (dg << sh));
    if (prev == old) return true;
    old = prev;
  }
  return false;
}

// The writes of a claim that won slot g of bucket b (its digest set): the
// bucket's count, the score, then the key.
__device__ __forceinline__ void write_claimed(const TableDev& t, uint64_t b, uint64_t g,
                                              uint64_t key, uint64_t sc) {
  atomicAdd(t.sizes + b, 1u);
  __stcg(reinterpret_cast<unsigned long long*>(score_ptr(t, g)), (unsigned long long)sc);
  __stcg(reinterpret_cast<unsigned long long*>(key_ptr(t, g)), (unsigned long long)key);
}

// First claim attempt of a missing key, from the digest lines its probe
// read (Algorithm 3 phase D1 on the free counts the probe saw: the bucket
// with more free slots, b1 on a tie): a CAS on the free slot the probe
// offered, with no further reads. Returns 0 when the key was placed (g_out
// set), 2 when both candidates were full at the probe (no slot is freed
// during a batch, so they still are), 1 when the CAS lost and the caller
// must claim through the occupancy counters (claim_free_slot).
__device__ __forceinline__ uint8_t claim_probed_slot(const TableDev& t, const Scratch& s,
                                                     uint32_t e, uint64_t key, uint64_t h,
                                                     uint64_t sc, uint64_t b1, unsigned f1,
                                                     unsigned f2, uint64_t& g_out,
                                                     unsigned& inserted, unsigned& retries) {
  const uint64_t b2 = t.dual ? second_bucket(t, key) : b1;
  const int c1 = free_count(f1), c2 = b2 != b1 ? free_count(f2) : 0;
  if (c1 == 0 && c2 == 0) return 2;
  const bool first = c1 >= c2;
  const uint64_t b = first ? b1 : b2;
  const int slot = free_slot_of(first ? f1 : f2);
  if (slot < 0) return 1;
  const uint64_t g = b * kSlots + (uint64_t)slot;
  if (!claim_digest(t, g, digest_from_hash(h))) {
    retries++;
    return 1;
  }
  write_claimed(t, b, g, key, sc);
  g_out = g;
  s.tstatus[e] = HKV_ST_INSERTED;
  inserted++;
  return 0;
}

__device__ __forceinline__ uint8_t claim_free_slot(const TableDev& t, const Scratch& s, uint32_t e,
                                                   uint64_t key, uint64_t h, uint64_t sc,
                                                   uint64_t& g_out, unsigned& sectors,
                                                   unsigned& inserted, unsigned& retries) {
  const uint64_t b1 = h & t.bucket_mask;
  const uint64_t b2 = t.dual ? second_bucket(t, key) : b1;
  const bool two = b2 != b1;
  for (int attempt = 0; attempt < kMaxClaimAttempts; ++attempt) {
    if (attempt) claim_backoff(attempt, h);
    const uint32_t n1 = __ldcg(t.sizes + b1);
    const uint32_t n2 = two ? __ldcg(t.sizes + b2) : kSlots;
    if (n1 >= kSlots && n2 >= kSlots) return 2;
    const uint64_t b = n1 <= n2 ? b1 : b2;
    const int slot = find_free(t.digests + b * kSlots, (unsigned)(h >> 40) + 2u * attempt, sectors);
    if (slot < 0) {
      retries++;
      continue;
    }
    const uint64_t g = b * kSlots + (uint64_t)slot;
    if (!claim_digest(t, g, digest_from_hash(h))) {
      retries++;
      continue;
    }
    write_claimed(t, b, g, key, sc);
    g_out = g;
    s.tstatus[e] = HKV_ST_INSERTED;
    inserted++;
    return 0;
  }
  latch_error(t.err, HKV_ERR_TIMEOUT);
  atomicAdd(t.counters + HKV_CNT_TIMEOUT_FREE, 1ull);
  atomicExch(t.counters + HKV_CNT_TIMEOUT_WHY, 5ull);
  atomicExch(t.counters + HKV_CNT_TIMEOUT_KEY, (unsigned long long)key);
  s.tstatus[e] = HKV_ST_REJECTED;
  return 0;
}

// ----------------------------------------------------------- phase U probe

// New score of a resident key (the hit branch of the table policy) written
// with the fewest memory round trips: LRU-type and caller scores are plain
// stores, LFU is an add whose result nobody waits for (an LFU score is a sum
// of batch multiplicities, so it never reaches the saturation point 2^64 - 1
// and the saturating add is a plain add), CUSTOM without caller scores keeps
// the score; the saturating sub-field counters read the old score first.
__device__ __forceinline__ void update_resident_score(const TableDev& t, uint64_t g, uint64_t m,
                                                      bool have_caller, uint64_t caller,
                                                      const ScoreCtx& c) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(score_ptr(t, g));
  switch (t.policy) {
    case HKV_LFU:
      atomicAdd(p, (unsigned long long)m);
      return;
    case HKV_LRU:
    case HKV_EPOCH_LRU:
      *p = policy_score(t.policy, true, 0, m, have_caller, caller, c);
      return;
    case HKV_CUSTOM:
      if (have_caller) *p = caller;
      return;
    default:
      *p = policy_score(t.policy, true, *p, m, have_caller, caller, c);
  }
}


constexpr int kUpdThreads = 256;
constexpr int kUpdBlocksPerSm = 4;  // resident blocks per SM (register bound)

template <int G, bool VEC16, bool UPSERT>
__global__ void __launch_bounds__(kUpdThreads, kUpdBlocksPerSm)
    update_kernel(TableDev t, Scratch s, const float* __restrict__ values,
                  const uint64_t* __restrict__ scores_in, ScoreCtx ctx) {
  if (aborted(s)) return;
  if (s.d) {
    values = s.d->values_in;
    scores_in = s.d->scores;
    ctx.step = s.d->step;
    ctx.epoch = s.d->epoch;
  }
  constexpr int KPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int lane_g = lane & (G - 1);
  const int group_base = lane & ~(G - 1);
  const unsigned group_bits = G == 32 ? kFull : (((1u << G) - 1u) << group_base);
  const uint64_t warp = (blockIdx.x * (uint64_t)kUpdThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kUpdThreads) >> 5;
  const uint64_t nu = s.cnt[kCntUnique];
  unsigned updated = 0, lines = 0, kreads = 0, inserted = 0, ins_lines = 0, retries = 0;
  unsigned deferred = 0;

  for (uint64_t base = warp * KPW; base < nu; base += nwarps * KPW) {
    const uint64_t u = base + (lane / G);
    const bool active = u < nu;
    // The distinct key comes from the dense list dedup wrote (no load
    // dependent on its dedup entry); the entry's (last index, count) word
    // is fetched beside it.
    uint32_t e = 0;
    uint64_t key = kEmptyKey;
    uint2 nc = make_uint2(0u, 0u);
    if (active) {
      e = __ldg(s.ulist + u);
      key = __ldg(s.mkey + u);
      nc = __ldg(reinterpret_cast<const uint2*>(s.tab + e) + 1);
    }
    const uint64_t i = (uint32_t)~nc.x;
    const uint64_t m = (uint64_t)nc.y + 1;
    const uint64_t h = fmix64(key);
    uint64_t b = h & t.bucket_mask;
    const uint32_t pat4 = digest_from_hash(h) * 0x01010101u;
    // upsert: the probes also report each candidate's free slots
    const unsigned pick = (unsigned)(h >> 40);
    unsigned f1 = 0, f2 = 0;
    int slot = probe_bucket<G, false, true, UPSERT>(t, b, key, pat4, active, lane_g, group_bits,
                                                    group_base, kreads, pick, &f1);
    lines += active && lane_g == 0;
    if (t.dual) {
      const uint64_t b2 = second_bucket(t, key);
      const bool need = active && slot < 0 && b2 != b;
      lines += need && lane_g == 0;
      if (__any_sync(kFull, need)) {
        const int s2 = probe_bucket<G, false, true, UPSERT>(t, b2, key, pat4, need, lane_g,
                                                            group_bits, group_base, kreads,
                                                            pick, &f2);
        if (need && s2 >= 0) {
          slot = s2;
          b = b2;
        }
      }
    }
    const bool hit = active && slot >= 0;
    // the slot whose value row this key's group writes below: a hit's own
    // slot (find_or_insert keeps a resident's row), or the slot a miss claims
    uint64_t gclaim = kNoSlot;
    if (active) {
      if (hit) {
        const uint64_t g = b * kSlots + (uint64_t)slot;
        if (values && !s.keep_hits && lane_g == 0) gclaim = g;
        if (lane_g == 0) {
          update_resident_score(t, g, m, scores_in != nullptr, scores_in ? __ldg(scores_in + i) : 0,
                                ctx);
          s.tstatus[e] = HKV_ST_UPDATED;
          updated++;
        }
      }
      if (UPSERT && lane_g == 0) {
        // mflag: 0 placed (updated, or claimed here), 1 miss left to the
        // ordered phase I, 2 miss whose candidate buckets are all full. A
        // miss claims its free slot right
        // here: a claim into an empty slot cannot race the in-place updates
        // of this phase (they touch other slots); only evictions must wait
        // for phase U to end.
        uint8_t flag = 0;
        if (!hit && s.owner) {
          flag = 1;  // ordered phase I places it (deterministic dual-bucket mode)
        } else if (!hit) {
          const uint64_t sc = policy_score(t.policy, false, 0, m, scores_in != nullptr,
                                           scores_in ? __ldg(scores_in + i) : 0, ctx);
          // a miss: b is still its first bucket
          flag = claim_probed_slot(t, s, e, key, h, sc, b, f1, f2, gclaim, inserted, retries);
          if (flag == 1)
            flag = claim_free_slot(t, s, e, key, h, sc, gclaim, ins_lines, inserted, retries);
        }
        s.mflag[u] = flag;
        if (flag) {
          s.mi[u] = (uint32_t)i;
          s.mm[u] = (uint32_t)m;
          deferred++;
        }
      }
    }
    {
      // one row copy per warp iteration for hits and claims together, by the
      // key's G lanes, after the claims (a host-memory row later, in region
      // order)
      const uint64_t gc = __shfl_sync(kFull, gclaim, group_base);
      if (gc != kNoSlot) {
        if (UPSERT && s.gdefer && !s.evv && gc >= s.host_slot0) {
          if (lane_g == 0) {
            s.gdefer[u] = gc;
            s.mi[u] = (uint32_t)i;
          }
        } else {
          copy_row<G, VEC16, false>(value_ptr(t, gc), values + i * t.dim, t.dim, lane_g,
                                    t.vec8);
        }
      }
    }
  }
  const int which[7] = {HKV_CNT_UPDATED, HKV_CNT_UPD_LINES, HKV_CNT_UPD_KEYS, HKV_CNT_INSERTED,
                        HKV_CNT_UPD_CLAIMS, HKV_CNT_UPD_CLAIM_LINES, HKV_CNT_RETRIES};
  const unsigned vals[7] = {updated, lines, kreads, inserted, inserted, ins_lines, retries};
  flush_counts(t, which, vals);
  if (UPSERT) block_reserve(s.cnt + kCntDeferred, deferred);
}

// --------------------------------------------------------- phase I insert

constexpr int kInsThreads = 256;
constexpr int kInsBlocksPerSm = 4;  // resident blocks per SM (register bound)

// Warp minimum of a 64-bit value as two 32-bit min-reductions (redux.sync).
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  const uint32_t hi = __reduce_min_sync(kFull, (uint32_t)(v >> 32));
  const uint32_t lo = __reduce_min_sync(kFull, (uint32_t)(v >> 32) == hi ? (uint32_t)v : ~0u);
  return ((unsigned long long)hi << 32) | lo;
}

// Warp-wide lexicographic minimum of the lanes' (s, k) pairs as four 32-bit
// min-reductions, most significant word first, each over the lanes still
// tied; `mine` is set on the lanes holding the minimum pair.
__device__ __forceinline__ void warp_min_sk(unsigned long long s, unsigned long long k,
                                            unsigned long long& smin, unsigned long long& kmin,
                                            bool& mine) {
  const uint32_t w[4] = {(uint32_t)(s >> 32), (uint32_t)s, (uint32_t)(k >> 32), (uint32_t)k};
  uint32_t m[4];
  bool tied = true;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    m[j] = __reduce_min_sync(kFull, tied ? w[j] : ~0u);
    tied = tied && w[j] == m[j];
  }
  smin = ((unsigned long long)m[0] << 32) | m[1];
  kmin = ((unsigned long long)m[2] << 32) | m[3];
  mine = tied;
}

// Slot of a bucket held by `lane` in a victim search's pair reads: slot
// 32q + lane for q = 0..3, so each of the warp's four reads covers 512
// contiguous bytes (16 whole sectors).
__device__ __forceinline__ int held_slot(int lane, int q) { return 32 * q + lane; }

// Write (value, score, digest) into a slot this warp holds LOCKED; its key
// is published afterwards (PendingKey). The digest and score go first, so
// other claimers see the slot taken at once even while a value row is still
// travelling to host memory; the lanes' value stores are ordered before the
// key by this function's warp barrier and the GPU-scope fence lane 0 runs
// before the key store, so no later writer of the slot can be overtaken by
// them.
//
// With `row` false the value row is left to the deferred-row pass (a slot
// in host memory, see flush_deferred_rows_kernel).
template <bool VEC16>
__device__ __forceinline__ void fill_slot(const TableDev& t, uint64_t g, uint64_t sc, uint32_t dg,
                                          const float* src, int lane, bool row = true) {
  if (lane == 0) {
    t.digests[g] = (uint8_t)dg;
    __stcg(reinterpret_cast<unsigned long long*>(score_ptr(t, g)), (unsigned long long)sc);
  }
  float* dst = value_ptr(t, g);
  if (!row) {
  } else if (VEC16) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (uint32_t j = lane; j < (t.dim >> 2); j += 32) __stcg(d4 + j, __ldg(s4 + j));
  } else if (t.vec8 && (t.dim & 1) == 0 &&
             ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 7) == 0) {
    const float2* s2 = reinterpret_cast<const float2*>(src);
    float2* d2 = reinterpret_cast<float2*>(dst);
    for (uint32_t j = lane; j < (t.dim >> 1); j += 32) __stcg(d2 + j, __ldg(s2 + j));
  } else {
    for (uint32_t j = lane; j < t.dim; j += 32) __stcg(dst + j, __ldg(src + j));
  }
  __syncwarp();
}

// A warp's replacements publish their keys in pairs: the first waits, LOCKED,
// until the second is filled, then one GPU-scope fence orders both slots'
// stores before both keys (the fence has a cost of its own, whatever is in
// flight: two replacements per fence measured 2.5% faster at lambda 1). A
// key still waiting is published alone before the warp retries a search
// (the retry may be waiting on that very slot) and at the end of a chunk.
// Warp-uniform; lane 0 stores.
struct PendingKey {
  bool on = false;
  uint64_t g = 0, key = 0;

  __device__ __forceinline__ void flush(const TableDev& t, int lane) {
    if (!on) return;
    if (lane == 0) publish_key(key_ptr(t, g), key);
    __syncwarp();
    on = false;
  }
  // slot g2 was just filled (fill_slot's warp barrier is behind us)
  __device__ __forceinline__ void add(const TableDev& t, uint64_t g2, uint64_t key2, int lane) {
    if (!on) {
      on = true;
      g = g2;
      key = key2;
      return;
    }
    if (lane == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(key_ptr(t, g)), "l"(key) : "memory");
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(key_ptr(t, g2)), "l"(key2)
                   : "memory");
    }
    __syncwarp();
    on = false;
  }
};

constexpr int kPrefetchAhead = 1;  // victim searches whose lines are prefetched ahead

// Phase I by every block of the launch, on a live batch whose phase U left
// keys for it (insert_kernel; insert_finish_kernel).
template <bool VEC16>
__device__ __forceinline__ void insert_body(const TableDev& t, const Scratch& s,
                                            const float* __restrict__ values,
                                            const uint64_t* __restrict__ scores_in, ScoreCtx ctx) {
  int row_prefetch = s.row_prefetch;
  if (s.d) {
    values = s.d->values_in;
    scores_in = s.d->scores;
    ctx.step = s.d->step;
    ctx.epoch = s.d->epoch;
    row_prefetch = s.d->row_prefetch;
  }
  const int lane = threadIdx.x & 31;
  const uint64_t nu = s.cnt[kCntUnique];
  const uint64_t nchunks = (nu + 31) / 32;
  unsigned inserted = 0, evicted = 0, rejected = 0, retries = 0;
  unsigned score_lines = 0;

  // Chunks of 32 distinct keys. With victim searches to do (at least one
  // full-bucket key per chunk on average) a chunk goes to whichever warp
  // is free next: how many searches a chunk holds varies widely, and a
  // fixed stride left warps idle while others still searched. Otherwise a
  // fixed stride, which spares the shared counter a burst of atomics.
  const uint64_t warp = (blockIdx.x * (uint64_t)kInsThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kInsThreads) >> 5;
  const bool dynamic = s.cnt[kCntDeferred] >= nchunks;
  PendingKey pend;
  for (uint64_t k = 0;; ++k) {
    unsigned long long c = warp + k * nwarps;
    if (dynamic) {
      if (lane == 0) c = atomicAdd(s.cnt + kCntInsCursor, 1ull);
      c = __shfl_sync(kFull, c, 0);
    }
    if (c >= nchunks) break;
    // The chunk's 32 distinct keys: flags and miss records, coalesced.
    const uint64_t my_u = c * 32 + lane;
    const uint8_t my_flag = my_u < nu ? s.mflag[my_u] : 0;
    const bool miss = my_flag != 0;
    uint64_t my_key = 0;
    uint32_t my_i = 0, my_m = 0, my_e = 0;
    if (miss) {
      my_key = s.mkey[my_u];
      my_i = s.mi[my_u];
      my_m = s.mm[my_u];
      my_e = s.ulist[my_u];
    }
    const uint64_t my_h = fmix64(my_key);
    const uint64_t my_b1 = my_h & t.bucket_mask;
    const uint64_t my_b2 = t.dual ? second_bucket(t, my_key) : my_b1;
    const bool my_two = my_b2 != my_b1;
    const uint64_t my_sc = policy_score(t.policy, false, 0, my_m, scores_in != nullptr,
                                        (miss && scores_in) ? __ldg(scores_in + my_i) : 0, ctx);

    // Misses with a free slot were placed by the update phase; what is
    // left (mflag 2) found every candidate bucket full.
    const bool full = my_flag == 2;

    // Warp-cooperative victim search for the keys whose buckets were
    // full, one key after another. The (key, score) pair runs of the next
    // search are pulled into L2 by bulk prefetches while the current one
    // runs (deeper prefetching measured slower: it competes for L2 and
    // DRAM).
    unsigned todo = __ballot_sync(kFull, full);
    {
      unsigned ahead = todo;
      for (int k = 0; k < kPrefetchAhead && ahead; ++k) {
        const int l = __ffs(ahead) - 1;
        ahead &= ahead - 1;
        if (lane == l) {
          bulk_prefetch_l2(key_ptr(t, my_b1 * kSlots), kSlots * 16);
          if (my_two) bulk_prefetch_l2(key_ptr(t, my_b2 * kSlots), kSlots * 16);
          if (VEC16 && row_prefetch)
            bulk_prefetch_l2(values + (uint64_t)my_i * t.dim, t.dim * 4);
        }
      }
    }
    while (todo) {
      const int src_lane = __ffs(todo) - 1;
      todo &= todo - 1;
      {
        // prefetch the search kPrefetchAhead positions ahead
        unsigned ahead = todo;
        for (int k = 1; k < kPrefetchAhead && ahead; ++k) ahead &= ahead - 1;
        if (ahead) {
          const int l = __ffs(ahead) - 1;
          if (lane == l) {
            bulk_prefetch_l2(key_ptr(t, my_b1 * kSlots), kSlots * 16);
            if (my_two) bulk_prefetch_l2(key_ptr(t, my_b2 * kSlots), kSlots * 16);
            if (VEC16 && row_prefetch)
              bulk_prefetch_l2(values + (uint64_t)my_i * t.dim, t.dim * 4);
          }
        }
      }
      const uint64_t u = c * 32 + src_lane;
      const uint64_t key = __shfl_sync(kFull, my_key, src_lane);
      const uint64_t i = __shfl_sync(kFull, my_i, src_lane);
      const uint32_t e = __shfl_sync(kFull, my_e, src_lane);
      const uint64_t sc = __shfl_sync(kFull, my_sc, src_lane);
      const uint64_t h = __shfl_sync(kFull, my_h, src_lane);
      const uint64_t b1 = __shfl_sync(kFull, my_b1, src_lane);
      const uint64_t b2 = __shfl_sync(kFull, my_b2, src_lane);
      const bool two = b2 != b1;
      const float* src = values + i * t.dim;
      const uint32_t dg = digest_from_hash(h);
      uint8_t outcome = HKV_ST_REJECTED;
      uint64_t victim_key = kEmptyKey;
      unsigned why = 0;
      int attempt = 0;
      for (; attempt < kMaxClaimAttempts; ++attempt) {
        if (attempt) {
          pend.flush(t, lane);
          claim_backoff(attempt, h);
        }
        // Buckets stay full during a batch (no erase runs beside an
        // inserter), so the victim search needs no free-slot re-check.
        // Each lane reads its slots' (key, score) pairs, coalesced (slots
        // l, 32+l, 64+l and 96+l of each candidate bucket) and keeps
        // its smallest (score, key); one warp argmin gives the victim. A slot
        // locked by another warp is mid-replacement: if its visible score
        // does not exceed the minimum, its next (score, key) could be the
        // minimum, so re-read later rather than choose around it.
        score_lines += two ? 2 : 1;
        unsigned long long bs = ~0ull, bk = ~0ull, lockmin = ~0ull;
        int bq = -1;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          if (half == 1 && !two) break;
          const uint64_t bb = half ? b2 : b1;
          // (key, score) pairs of the held slots 32q + l
          const ulonglong2* pp = reinterpret_cast<const ulonglong2*>(key_ptr(t, bb * kSlots));
          const ulonglong2 p0 = __ldcg(pp + held_slot(lane, 0)), p1 = __ldcg(pp + held_slot(lane, 1));
          const ulonglong2 p2 = __ldcg(pp + held_slot(lane, 2)), p3 = __ldcg(pp + held_slot(lane, 3));
          const unsigned long long sq[4] = {p0.y, p1.y, p2.y, p3.y};
          const unsigned long long kq[4] = {p0.x, p1.x, p2.x, p3.x};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (kq[j] >= kLockedKey) {
              lockmin = sq[j] < lockmin ? sq[j] : lockmin;
            } else if (sk_less(sq[j], kq[j], bs, bk)) {
              bs = sq[j];
              bk = kq[j];
              bq = half * 4 + j;
            }
          }
        }
        unsigned long long smin, kmin;
        bool mine;
        warp_min_sk(bs, bk, smin, kmin, mine);
        lockmin = warp_min_u64(lockmin);
        if (lockmin <= smin || kmin == ~0ull) {
          why = kmin == ~0ull ? 2u : 1u;
          retries += lane == 0;
          continue;
        }
        const int qbest = bq;
        // Admission control: admit iff (s, k) > (s_min, k_min).
        if (!sk_less(smin, kmin, sc, key)) {
          outcome = HKV_ST_REJECTED;
          rejected++;
          break;
        }
        const unsigned own = __ballot_sync(kFull, qbest >= 0 && mine);
        const int owner = __ffs(own) - 1;
        int ok = 0;
        uint64_t g = 0;
        if (lane == owner) {
          const uint64_t bqk = qbest < 4 ? b1 : b2;
          g = bqk * kSlots + (uint64_t)held_slot(lane, qbest & 3);
          // Lock the victim only if its pair is still the (key, score) the
          // minimum was read from: a key and score read from two different
          // occupants of the slot cannot pass.
          ok = cas_pair(key_ptr(t, g), kmin, smin, kLockedKey, smin);
        }
        ok = __shfl_sync(kFull, ok, owner);
        g = __shfl_sync(kFull, g, owner);
        if (!ok) {
          why = 3u;
          retries += lane == 0;
          continue;
        }
        if (lane == 0) s.evs[u] = smin;
        if (s.evv) {
          const float* vsrc = value_ptr(t, g);
          for (uint32_t d = lane; d < t.dim; d += 32) s.evv[u * t.dim + d] = __ldcg(vsrc + d);
        }
        // a row bound for host memory waits for the deferred-row pass
        const bool defer = s.gdefer != nullptr && g >= s.host_slot0;
        if (defer && lane == 0) s.gdefer[u] = g;
        fill_slot<VEC16>(t, g, sc, dg, src, lane, !defer);
        pend.add(t, g, key, lane);
        victim_key = kmin;
        outcome = HKV_ST_INSERTED;
        evicted++;
        break;
      }
      if (lane == 0) {
        if (attempt == kMaxClaimAttempts) {
          latch_error(t.err, HKV_ERR_TIMEOUT);
          atomicAdd(t.counters + HKV_CNT_TIMEOUT_EVICT, 1ull);
          atomicExch(t.counters + HKV_CNT_TIMEOUT_WHY, (unsigned long long)why);
          atomicExch(t.counters + HKV_CNT_TIMEOUT_KEY, (unsigned long long)key);
        }
        s.evk[u] = victim_key;
        s.tstatus[e] = outcome;
      }
    }
    pend.flush(t, lane);
  }
  const int which[7] = {HKV_CNT_INSERTED, HKV_CNT_EVICTED, HKV_CNT_REJECTED, HKV_CNT_RETRIES,
                        HKV_CNT_INS_LINES, HKV_CNT_INS_SCORES, HKV_CNT_INS_KEYS};
  const unsigned vals[7] = {inserted, lane == 0 ? evicted : 0u, lane == 0 ? rejected : 0u,
                            retries, 0u, lane == 0 ? score_lines : 0u, 0u};
  flush_counts(t, which, vals);
}

template <bool VEC16>
__global__ void __launch_bounds__(kInsThreads, kInsBlocksPerSm)
    insert_kernel(TableDev t, Scratch s, const float* __restrict__ values,
                  const uint64_t* __restrict__ scores_in, ScoreCtx ctx) {
  if (aborted(s)) return;
  // Phase U placed every key: no victim search (the same for the whole grid)
  if (s.cnt[kCntDeferred] == 0) return;
  insert_body<VEC16>(t, s, values, scores_in, ctx);
}

// ------------------------------------------------- ordered phase I (waves)
//
// Deterministic dual-bucket mode: phase I must equal Algorithm 3 run key by
// key in batch order, because a key's D1 choice and D2 victim depend on what
// earlier keys did to its two buckets. Keys run in waves: in wave w every
// pending key bids for both candidate buckets with tag (w, ~i) (a 64-bit
// atomicMax, so a bucket's word needs no reset between waves and holds the
// smallest pending batch index i of the wave); a key that wins both of its
// buckets runs Algorithm 3 alone on them. Keys of one wave touch disjoint
// buckets, and every key runs after all earlier keys sharing a bucket with
// it, so the result is the sequential one. The key with the smallest
// pending i always wins, so the waves end after at most one per key.

constexpr int kOrdThreads = 256;

__device__ __forceinline__ unsigned long long wave_tag(uint64_t wave, uint32_t i) {
  return (wave << 32) | (unsigned long long)(0xFFFFFFFFu - i);
}

// Wave `wave`'s bids of every pending key (Algorithm 3 order: the smallest
// batch index wins each bucket).
__device__ __forceinline__ void ordered_bid(const TableDev& t, const Scratch& s, uint64_t wave) {
  const uint64_t nu = s.cnt[kCntUnique];
  for (uint64_t u = blockIdx.x * (uint64_t)kOrdThreads + threadIdx.x; u < nu;
       u += (uint64_t)gridDim.x * kOrdThreads) {
    if (__ldcg(s.mflag + u) != 1) continue;
    const uint64_t key = s.mkey[u];
    const uint64_t b1 = fmix64(key) & t.bucket_mask;
    const uint64_t b2 = t.dual ? second_bucket(t, key) : b1;
    const unsigned long long tag = wave_tag(wave, s.mi[u]);
    atomicMax(s.owner + b1, tag);
    if (b2 != b1) atomicMax(s.owner + b2, tag);
  }
}

__global__ void __launch_bounds__(kOrdThreads)
    ordered_bid_kernel(TableDev t, Scratch s, uint64_t wave) {
  if (aborted(s)) return;
  ordered_bid(t, s, wave);
}

// A warp of the ordered phase I takes 32 consecutive u. Every lane checks
// whether its key won both buckets this wave; winners with a free slot take
// it alone (D1), winners whose candidates are full run the D2 victim search
// as a warp, one key after another: coalesced (score, key) pairs of both
// buckets, one warp argmin, admission, replacement. A winner owns its
// buckets for the wave, so nothing here locks or re-checks.
template <bool VEC16>
__device__ __forceinline__ void ordered_insert(const TableDev& t, const Scratch& s,
                                               const float* __restrict__ values,
                                               const uint64_t* __restrict__ scores_in,
                                               const ScoreCtx& ctx, uint64_t wave,
                                               unsigned& pending, unsigned& inserted,
                                               unsigned& evicted, unsigned& rejected) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)kOrdThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kOrdThreads) >> 5;
  const uint64_t nu = s.cnt[kCntUnique];
  for (uint64_t c = warp; c * 32 < nu; c += nwarps) {
    const uint64_t u = c * 32 + lane;
    bool won = u < nu && __ldcg(s.mflag + u) == 1;
    uint64_t key = 0, b1 = 0, b2 = 0, sc = 0;
    uint32_t i = 0, e = 0, dg = 0;
    bool full = false;
    if (won) {
      key = s.mkey[u];
      i = s.mi[u];
      e = s.ulist[u];
      const uint64_t h = fmix64(key);
      dg = digest_from_hash(h);
      b1 = h & t.bucket_mask;
      b2 = t.dual ? second_bucket(t, key) : b1;
      const unsigned long long tag = wave_tag(wave, i);
      if (__ldcg(s.owner + b1) != tag || (b2 != b1 && __ldcg(s.owner + b2) != tag)) {
        pending++;
        won = false;
      }
    }
    if (won) {
      sc = policy_score(t.policy, false, 0, s.mm[u], scores_in != nullptr,
                        scores_in ? __ldg(scores_in + i) : 0, ctx);
      const uint32_t n1 = __ldcg(t.sizes + b1);
      const uint32_t n2 = b2 != b1 ? __ldcg(t.sizes + b2) : kSlots;
      if (n1 < kSlots || n2 < kSlots) {
        // D1: the less occupied candidate, b1 on equal occupancy
        const uint64_t b = n1 <= n2 ? b1 : b2;
        unsigned sectors = 0;
        const int slot = find_free(t.digests + b * kSlots, 0u, sectors);
        if (slot < 0) {  // a counter out of step with its digests: refuse the batch
          abort_batch(s, t.err, HKV_ERR_CUDA);
        } else {
          t.sizes[b] = (n1 <= n2 ? n1 : n2) + 1u;
          fill_slot_thread<VEC16, false>(t, b * kSlots + (uint64_t)slot, key, sc, dg,
                                         values + (uint64_t)i * t.dim);
          s.evk[u] = kEmptyKey;
          s.tstatus[e] = HKV_ST_INSERTED;
          inserted++;
        }
        s.mflag[u] = 2;
      } else {
        full = true;
      }
    }
    // D2, warp-cooperative, for the winners whose candidates are both full
    unsigned todo = __ballot_sync(kFull, full);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint64_t uu = c * 32 + src;
      const uint64_t k = __shfl_sync(kFull, key, src);
      const uint64_t ks = __shfl_sync(kFull, sc, src);
      const uint64_t c1 = __shfl_sync(kFull, b1, src), c2 = __shfl_sync(kFull, b2, src);
      const uint32_t ki = __shfl_sync(kFull, i, src), ke = __shfl_sync(kFull, e, src);
      const uint32_t kdg = __shfl_sync(kFull, dg, src);
      const bool two = c2 != c1;
      unsigned long long bs = ~0ull, bk = ~0ull;
      int bq = -1;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (half == 1 && !two) break;
        const uint64_t bb = half ? c2 : c1;
        const ulonglong2* pp = reinterpret_cast<const ulonglong2*>(key_ptr(t, bb * kSlots));
        const ulonglong2 p0 = __ldcg(pp + held_slot(lane, 0)), p1 = __ldcg(pp + held_slot(lane, 1));
        const ulonglong2 p2 = __ldcg(pp + held_slot(lane, 2)), p3 = __ldcg(pp + held_slot(lane, 3));
        const unsigned long long sq[4] = {p0.y, p1.y, p2.y, p3.y};
        const unsigned long long kq[4] = {p0.x, p1.x, p2.x, p3.x};
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (sk_less(sq[j], kq[j], bs, bk)) {
            bs = sq[j];
            bk = kq[j];
            bq = half * 4 + j;
          }
      }
      unsigned long long smin, kmin;
      bool at_min;
      warp_min_sk(bs, bk, smin, kmin, at_min);
      const int holder = __ffs(__ballot_sync(kFull, bq >= 0 && at_min)) - 1;
      const uint64_t gl = (uint64_t)(bq < 4 ? c1 : c2) * kSlots + (uint64_t)held_slot(lane, bq & 3);
      const uint64_t g = __shfl_sync(kFull, gl, holder);
      if (sk_less(smin, kmin, ks, k)) {  // admitted: replace the minimum
        if (s.evv) {
          const float* vsrc = value_ptr(t, g);
          for (uint32_t d = lane; d < t.dim; d += 32) s.evv[uu * t.dim + d] = __ldcg(vsrc + d);
        }
        __syncwarp();
        float* dst = value_ptr(t, g);
        const float* vin = values + (uint64_t)ki * t.dim;
        for (uint32_t d = lane; d < t.dim; d += 32) __stcg(dst + d, __ldg(vin + d));
        if (lane == 0) {
          t.digests[g] = (uint8_t)kdg;
          __stcg(reinterpret_cast<unsigned long long*>(score_ptr(t, g)), (unsigned long long)ks);
          __stcg(reinterpret_cast<unsigned long long*>(key_ptr(t, g)), (unsigned long long)k);
          s.evk[uu] = kmin;
          s.evs[uu] = smin;
          s.tstatus[ke] = HKV_ST_INSERTED;
          evicted++;
        }
      } else if (lane == 0) {
        s.evk[uu] = kEmptyKey;
        s.tstatus[ke] = HKV_ST_REJECTED;
        rejected++;
      }
      if (lane == 0) s.mflag[uu] = 2;
    }
  }
}

template <bool VEC16>
__global__ void __launch_bounds__(kOrdThreads)
    ordered_insert_kernel(TableDev t, Scratch s, const float* __restrict__ values,
                          const uint64_t* __restrict__ scores_in, ScoreCtx ctx, uint64_t wave) {
  if (aborted(s)) return;
  unsigned pending = 0, inserted = 0, evicted = 0, rejected = 0;
  ordered_insert<VEC16>(t, s, values, scores_in, ctx, wave, pending, inserted, evicted, rejected);
  const int which[3] = {HKV_CNT_INSERTED, HKV_CNT_EVICTED, HKV_CNT_REJECTED};
  const unsigned vals[3] = {inserted, evicted, rejected};
  flush_counts(t, which, vals);
  const unsigned long long p = block_reserve(s.cnt + kCntPending, pending);
  (void)p;
}

// All waves in one cooperative launch (every block resident): bid pass,
// grid barrier, insert pass, grid barrier, and stop when the wave left no
// key pending. Removes two launches per wave and the host's check every few
// waves. The pending count alternates between two words by wave parity:
// block 0 clears the next wave's word after this wave's first barrier, when
// every block has read it. Flags other blocks write are read from L2.
constexpr unsigned kBarrierSpins = 1u << 22;  // 64-ns naps: ~0.3 s, then give up

// Grid-wide barrier; false (after latching HKV_ERR_TIMEOUT and aborting the
// batch) if the other blocks did not all arrive within the bound.
__device__ bool grid_barrier(const Scratch& s, uint32_t* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned long long* gen = s.cnt + kBarGen;
    const unsigned long long g = *gen;
    __threadfence();
    if (atomicAdd(s.cnt + kBarCount, 1ull) == gridDim.x - 1) {
      atomicExch(s.cnt + kBarCount, 0ull);
      __threadfence();
      atomicAdd(s.cnt + kBarGen, 1ull);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (++it > kBarrierSpins) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (!ok) abort_batch(s, err, HKV_ERR_TIMEOUT);
  }
  __syncthreads();
  const int r = ok;
  __syncthreads();
  return r != 0;
}

template <bool VEC16>
__global__ void __launch_bounds__(kOrdThreads)
    ordered_waves_kernel(TableDev t, Scratch s, const float* __restrict__ values,
                         const uint64_t* __restrict__ scores_in, ScoreCtx ctx) {
  unsigned inserted = 0, evicted = 0, rejected = 0;
  const uint64_t nu = s.cnt[kCntUnique];
  // each wave places the smallest pending key, so nu waves always suffice
  __shared__ int stop;
  for (uint64_t wave = 1; wave <= nu; ++wave) {
    // one decision per block: another block may abort between two reads
    __syncthreads();
    if (threadIdx.x == 0) stop = aborted(s) ? 1 : 0;
    __syncthreads();
    if (stop) break;
    unsigned long long* pend = s.cnt + ((wave & 1) ? kCntPending : kCntPending2);
    unsigned long long* next = s.cnt + ((wave & 1) ? kCntPending2 : kCntPending);
    ordered_bid(t, s, wave);
    if (!grid_barrier(s, t.err)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) *next = 0;
    unsigned pw = 0;
    ordered_insert<VEC16>(t, s, values, scores_in, ctx, wave, pw, inserted, evicted, rejected);
    block_reserve(pend, pw);
    if (!grid_barrier(s, t.err)) break;
    if (__ldcg(pend) == 0) break;
  }
  const int which[3] = {HKV_CNT_INSERTED, HKV_CNT_EVICTED, HKV_CNT_REJECTED};
  const unsigned vals[3] = {inserted, evicted, rejected};
  flush_counts(t, which, vals);
}

// ------------------------------------------------- gather of input rows

constexpr int kGatherThreads = 256;

// For every distinct key of the batch, copy the row of its last occurrence
// from src (rows the update and insert phases would read slowly in place,
// e.g. page-locked host memory) to the same position of dst (device). One
// thread per 16 bytes (vec16: dim % 4 == 0 and both arrays 16-byte aligned)
// or per float; each pass of the grid has all of its loads in flight.
__global__ void __launch_bounds__(kGatherThreads)
    gather_last_rows_kernel(Scratch s, const float* __restrict__ src, float* __restrict__ dst,
                            uint32_t dim, int vec16) {
  if (aborted(s)) return;
  const uint64_t nu = s.cnt[kCntUnique];
  const uint32_t per_row = vec16 ? dim / 4 : dim;
  const uint64_t units = nu * per_row;
  for (uint64_t q = blockIdx.x * (uint64_t)kGatherThreads + threadIdx.x; q < units;
       q += (uint64_t)gridDim.x * kGatherThreads) {
    const uint64_t u = q / per_row;
    const uint32_t j = (uint32_t)(q - u * per_row);
    const uint64_t i = (uint32_t)~s.tab[s.ulist[u]].nlast;  // last occurrence of key u
    if (vec16)
      reinterpret_cast<float4*>(dst)[i * per_row + j] =
          __ldg(reinterpret_cast<const float4*>(src) + i * per_row + j);
    else
      dst[i * dim + j] = __ldg(src + i * dim + j);
  }
}

// --------------------------------------------------------------- reconcile

constexpr int kRecThreads = 256;
constexpr int kRecPerThread = 4;  // distinct keys a thread has in flight per round

// Every distinct key whose phase I displaced a resident entry reports that
// entry as evicted, unless the displaced key is itself a key of this batch
// inserted earlier in the same call (then it is refused instead). A round
// takes kRecPerThread keys per thread, strided by the grid: their loads and
// dedup-chain walks are in flight together, and one list reservation per
// block covers all of them.
// The reconcile pass over the batch's distinct keys, by every block of the
// launch (grid-stride); the caller has checked that the batch is live and
// that phase I ran.
__device__ __forceinline__ void reconcile_body(const TableDev& t, const Scratch& s,
                                               uint64_t* __restrict__ ev_keys,
                                               uint64_t* __restrict__ ev_scores,
                                               float* __restrict__ ev_values) {
  const int tab_bits = s.d ? tab_bits_for(s.d->n) : s.tab_bits;
  const uint64_t tab_mask = (1ull << tab_bits) - 1;
  const uint64_t nu = s.cnt[kCntUnique];
  const uint64_t stride = (uint64_t)gridDim.x * kRecThreads;
  for (uint64_t base = (uint64_t)blockIdx.x * kRecThreads; base < nu;
       base += kRecPerThread * stride) {
    uint64_t k[kRecPerThread], gp[kRecPerThread];
    bool out[kRecPerThread], walking[kRecPerThread];
    uint8_t f[kRecPerThread];
#pragma unroll
    for (int r = 0; r < kRecPerThread; ++r) {
      const uint64_t u = base + r * stride + threadIdx.x;
      f[r] = u < nu ? s.mflag[u] : 0;
    }
#pragma unroll
    for (int r = 0; r < kRecPerThread; ++r) {
      const uint64_t u = base + r * stride + threadIdx.x;
      k[r] = f[r] ? s.evk[u] : kEmptyKey;
    }
#pragma unroll
    for (int r = 0; r < kRecPerThread; ++r) {
      out[r] = walking[r] = k[r] != kEmptyKey;
      gp[r] = dedup_pos(k[r], tab_bits);
    }
    for (;;) {  // the table holds >= 2n entries: every walk ends
      uint64_t tk[kRecPerThread];
#pragma unroll
      for (int r = 0; r < kRecPerThread; ++r) tk[r] = walking[r] ? s.tab[gp[r]].key : 0ull;
      bool any = false;
#pragma unroll
      for (int r = 0; r < kRecPerThread; ++r) {
        if (!walking[r]) continue;
        if (tk[r] == k[r]) {
          // displaced by a later key of this batch: not an eviction
          if (s.tstatus[gp[r]] == HKV_ST_INSERTED) {
            s.tstatus[gp[r]] = HKV_ST_REJECTED;
            out[r] = false;
          }
          walking[r] = false;
        } else if (tk[r] == kEmptyKey) {
          walking[r] = false;
        } else {
          gp[r] = (gp[r] + 1) & tab_mask;
          any = true;
        }
      }
      if (!any) break;
    }
    unsigned cnt = 0;
#pragma unroll
    for (int r = 0; r < kRecPerThread; ++r) cnt += out[r] ? 1u : 0u;
    unsigned long long o = block_reserve(s.cnt + kCntEvOut, cnt);
#pragma unroll
    for (int r = 0; r < kRecPerThread; ++r) {
      if (!out[r]) continue;
      const uint64_t u = base + r * stride + threadIdx.x;
      if (ev_keys) ev_keys[o] = k[r];
      if (ev_scores) ev_scores[o] = s.evs[u];
      if (ev_values && s.evv)
        for (uint32_t d = 0; d < t.dim; ++d) ev_values[o * t.dim + d] = s.evv[u * t.dim + d];
      ++o;
    }
  }
}

__global__ void __launch_bounds__(kRecThreads)
    reconcile_kernel(TableDev t, Scratch s, uint64_t* __restrict__ ev_keys,
                     uint64_t* __restrict__ ev_scores, float* __restrict__ ev_values) {
  if (aborted(s)) return;
  // Phase U placed every key, so no key displaced anything (grid-uniform)
  if (s.cnt[kCntDeferred] == 0) return;
  reconcile_body(t, s, ev_keys, ev_scores, ev_values);
}

constexpr int kStatusPerThread = 4;  // positions a thread has in flight per round

// Deferred rows (tables with host-memory slices). A slot in host memory
// that phase U updated or claimed, or that phase I replaced, got its key,
// score and digest in its phase but not its value row: phase U would have
// scattered rows over the whole host range, and phase I would have waited
// for each row to cross the host link before publishing the key. The
// distinct keys that own such slots are grouped by host region
// (region_sort) and each writes its row here, in that order, if its slot
// still holds it (a slot replaced again later in the batch belongs to the
// later key, whose own entry writes it). Phase U keeps its rows direct when
// evicted values are asked for, so that a victim's reported row is its
// value after phase U. Groups of 8 lanes per row keep many rows in flight.
constexpr int kFlushThreads = 256;
constexpr int kFlushLanes = 8;

template <bool VEC16>
__global__ void __launch_bounds__(kFlushThreads)
    flush_deferred_rows_kernel(TableDev t, Scratch s, RegionOrder ro,
                               const float* __restrict__ values) {
  const uint64_t m = *ro.count;
  const int lane_g = threadIdx.x & (kFlushLanes - 1);
  const uint64_t grp = (blockIdx.x * (uint64_t)kFlushThreads + threadIdx.x) / kFlushLanes;
  const uint64_t ngrp = (uint64_t)gridDim.x * kFlushThreads / kFlushLanes;
  for (uint64_t p = grp; p < m; p += ngrp) {
    const uint64_t u = ro.order[p];
    const uint64_t g = s.gdefer[u];
    if (__ldcg(reinterpret_cast<const unsigned long long*>(key_ptr(t, g))) != s.mkey[u]) continue;
    copy_row<kFlushLanes, VEC16, false>(value_ptr(t, g), values + (uint64_t)s.mi[u] * t.dim,
                                        t.dim, lane_g, t.vec8);
  }
}

// The status broadcast, by every block of the launch (grid-stride), on a
// live batch.
__device__ __forceinline__ void status_body(uint64_t n, const Scratch& s,
                                            uint8_t* __restrict__ status_out,
                                            uint64_t* __restrict__ n_evicted) {
  if (s.d) {
    n = s.d->n;
    status_out = s.d->flags;
  }
  if (status_out) {
    // each position's status is its dedup entry's: both loads of a round's
    // positions go out together
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < n;
         i0 += kStatusPerThread * stride) {
      uint32_t e[kStatusPerThread];
      uint8_t v[kStatusPerThread];
#pragma unroll
      for (int r = 0; r < kStatusPerThread; ++r) {
        const uint64_t i = i0 + r * stride;
        e[r] = i < n ? s.slot_of[i] : 0u;
      }
#pragma unroll
      for (int r = 0; r < kStatusPerThread; ++r) v[r] = i0 + r * stride < n ? s.tstatus[e[r]] : 0;
#pragma unroll
      for (int r = 0; r < kStatusPerThread; ++r)
        if (i0 + r * stride < n) status_out[i0 + r * stride] = v[r];
    }
  }
  if (n_evicted && blockIdx.x == 0 && threadIdx.x == 0) *n_evicted = s.cnt[kCntEvOut];
}

__global__ void status_kernel(uint64_t n, Scratch s, uint8_t* __restrict__ status_out,
                              uint64_t* __restrict__ n_evicted) {
  if (aborted(s)) return;
  status_body(n, s, status_out, n_evicted);
}

// Reconcile and status in one cooperative launch (the plain upsert path):
// below lambda 1 phase U places every key and the reconcile pass has nothing
// to do, so the launch is the status broadcast alone; otherwise a grid
// barrier separates the two passes (status reads what reconcile settled).
// The batch's abort flag and deferred count were set by earlier kernels, so
// every block takes the same branch and meets the barrier.
__global__ void __launch_bounds__(kRecThreads)
    finish_kernel(TableDev t, Scratch s, uint64_t* __restrict__ ev_keys,
                  uint64_t* __restrict__ ev_scores, float* __restrict__ ev_values, uint64_t n,
                  uint8_t* __restrict__ status_out, uint64_t* __restrict__ n_evicted) {
  if (aborted(s)) return;
  if (s.cnt[kCntDeferred] != 0) {
    reconcile_body(t, s, ev_keys, ev_scores, ev_values);
    if (!grid_barrier(s, t.err)) return;
  }
  status_body(n, s, status_out, n_evicted);
}

// Phase I, reconcile and status in one cooperative launch (plain upserts of
// tables without host rows or ordered waves): below lambda 1 phase U placed
// every key and the launch is the status broadcast alone, one launch where
// there were two; otherwise grid barriers separate the three passes. Phase I
// latches its timeouts without setting the abort flag, so every block takes
// the same branch and meets both barriers.
template <bool VEC16>
__global__ void __launch_bounds__(kInsThreads, kInsBlocksPerSm)
    insert_finish_kernel(TableDev t, Scratch s, const float* __restrict__ values,
                         const uint64_t* __restrict__ scores_in, ScoreCtx ctx,
                         uint64_t* __restrict__ ev_keys, uint64_t* __restrict__ ev_scores,
                         float* __restrict__ ev_values, uint64_t n,
                         uint8_t* __restrict__ status_out, uint64_t* __restrict__ n_evicted) {
  if (aborted(s)) return;
  if (s.cnt[kCntDeferred] != 0) {
    insert_body<VEC16>(t, s, values, scores_in, ctx);
    if (!grid_barrier(s, t.err)) return;
    reconcile_body(t, s, ev_keys, ev_scores, ev_values);
    if (!grid_barrier(s, t.err)) return;
  }
  status_body(n, s, status_out, n_evicted);
}

// -------------------------------------------------------------------- erase

__global__ void validate_kernel(uint64_t n, const uint64_t* __restrict__ keys, Scratch s,
                                uint32_t* err) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (__ldg(keys + i) >= kFirstReserved) abort_batch(s, err, HKV_ERR_RESERVED_KEY);
}

template <int G>
__global__ void __launch_bounds__(kUpdThreads)
    erase_kernel(TableDev t, uint64_t n, const uint64_t* __restrict__ keys, Scratch s) {
  if (aborted(s)) return;
  constexpr int KPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int lane_g = lane & (G - 1);
  const int group_base = lane & ~(G - 1);
  const unsigned group_bits = G == 32 ? kFull : (((1u << G) - 1u) << group_base);
  const uint64_t warp = (blockIdx.x * (uint64_t)kUpdThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kUpdThreads) >> 5;
  for (uint64_t base = warp * KPW; base < n; base += nwarps * KPW) {
    const uint64_t i = base + (lane / G);
    const bool active = i < n;
    const uint64_t key = active ? __ldg(keys + i) : kEmptyKey;
    const uint64_t h = fmix64(key);
    uint64_t b = h & t.bucket_mask;
    const uint32_t pat4 = digest_from_hash(h) * 0x01010101u;
    // Duplicates in the batch may clear the slot concurrently: read through L2.
    unsigned kreads = 0;
    int slot = probe_bucket<G, true, false>(t, b, key, pat4, active, lane_g, group_bits,
                                            group_base, kreads);
    if (t.dual) {
      const uint64_t b2 = second_bucket(t, key);
      const bool need = active && slot < 0 && b2 != b;
      if (__any_sync(kFull, need)) {
        const int s2 = probe_bucket<G, true, false>(t, b2, key, pat4, need, lane_g,
                                                    group_bits, group_base, kreads);
        if (need && s2 >= 0) { slot = s2; b = b2; }
      }
    }
    if (active && slot >= 0 && lane_g == 0) {
      const uint64_t g = b * kSlots + (uint64_t)slot;
      // Duplicates of a key in one erase batch all find its slot: the CAS
      // lets exactly one of them clear it and count it out of its bucket.
      if (atomicCAS(reinterpret_cast<unsigned long long*>(key_ptr(t, g)), key, kEmptyKey) == key) {
        t.digests[g] = 0;
        *score_ptr(t, g) = 0;
        atomicSub(t.sizes + b, 1u);
      }
    }
  }
}

// ---------------------------------------------------------------- scratch

struct ScratchAlloc {
  Scratch s{};
  void* base = nullptr;
  void* region = nullptr;  // region_sort scratch of the deferred rows, or null
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

hkv_status alloc_scratch(hkv_table_s* t, uint64_t n, bool upsert, bool want_ev_values,
                         cudaStream_t st, ScratchAlloc* a) {
  int bits = 10;
  while ((1ull << bits) < 2 * n) ++bits;
  const uint64_t T = 1ull << bits;
  const uint64_t sz_tab = align256(T * sizeof(DedupEntry));
  const uint64_t sz_ts = align256(T);
  const uint64_t sz_u8 = align256(n);
  const uint64_t sz_u32 = align256(n * 4);
  const uint64_t sz_u64 = align256(n * 8);
  const uint64_t sz_cnt = align256(kCntWords * 8);
  const uint64_t sz_evv = want_ev_values ? align256(n * (uint64_t)t->dev.dim * 4) : 0;
  // deterministic dual-bucket upserts run phase I in ordered waves
  const bool ordered = upsert && t->opts.deterministic && t->dev.dual;
  const uint64_t sz_owner = ordered ? align256(t->num_buckets * 8) : 0;
  // phase I defers the rows of host-memory slots (tiered tables)
  const bool defer = upsert && !ordered && !t->host_slices.empty();
  const uint64_t sz_defer = defer ? sz_u64 + align256(region_sort_bytes(t, n)) : 0;
  uint64_t total = sz_tab + sz_ts + 2 * sz_u32 + sz_cnt + sz_u64;
  if (upsert) total += sz_u8 + 2 * sz_u64 + 2 * sz_u32 + sz_evv + sz_owner + sz_defer;
  cudaError_t e = cudaMallocFromPoolAsync(&a->base, total, t->pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error("scratch allocation failed");
    return HKV_ERR_OOM;
  }
  char* p = static_cast<char*>(a->base);
  Scratch& s = a->s;
  s.tab = reinterpret_cast<DedupEntry*>(p); p += sz_tab;
  s.tab_bits = bits;
  s.tab_mask = T - 1;
  s.tstatus = reinterpret_cast<uint8_t*>(p); p += sz_ts;
  s.slot_of = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.ulist = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.cnt = reinterpret_cast<unsigned long long*>(p); p += sz_cnt;
  s.mkey = reinterpret_cast<uint64_t*>(p); p += sz_u64;
  if (upsert) {
    s.mflag = reinterpret_cast<uint8_t*>(p); p += sz_u8;
    s.evk = reinterpret_cast<uint64_t*>(p); p += sz_u64;
    s.evs = reinterpret_cast<uint64_t*>(p); p += sz_u64;
    s.mi = reinterpret_cast<uint32_t*>(p); p += sz_u32;
    s.mm = reinterpret_cast<uint32_t*>(p); p += sz_u32;
    s.evv = want_ev_values ? reinterpret_cast<float*>(p) : nullptr;
    p += sz_evv;
    s.owner = ordered ? reinterpret_cast<unsigned long long*>(p) : nullptr;
    p += sz_owner;
    if (ordered) cudaMemsetAsync(s.owner, 0, t->num_buckets * 8, st);
    s.gdefer = defer ? reinterpret_cast<uint64_t*>(p) : nullptr;
    a->region = defer ? p + sz_u64 : nullptr;
    s.host_slot0 = t->hbm_value_slots;
    if (defer) cudaMemsetAsync(s.gdefer, 0xFF, n * 8, st);
  }
  cudaMemsetAsync(s.tab, 0xFF, T * sizeof(DedupEntry), st);
  cudaMemsetAsync(s.cnt, 0, kCntWords * 8, st);
  return HKV_OK;
}

unsigned grid_for(const hkv_table_s* t, uint64_t threads_needed, int block, int per_sm) {
  uint64_t blocks = (threads_needed + block - 1) / block;
  const uint64_t cap = (uint64_t)t->num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  return blocks ? (unsigned)blocks : 1u;
}

// Blocks of reconcile_kernel for a batch of n keys: kRecPerThread distinct
// keys per thread, at most four blocks per SM (48 registers: all resident).
unsigned reconcile_grid(const hkv_table_s* t, uint64_t n) {
  return grid_for(t, (n + kRecPerThread - 1) / kRecPerThread, kRecThreads, 4);
}

template <int G, bool UPSERT>
void launch_update_g(hkv_table_s* t, uint64_t n, const Scratch& s, const float* values,
                     const uint64_t* scores, ScoreCtx ctx, bool vec16, cudaStream_t st) {
  // Two waves of resident blocks: a block whose warps finish early hands
  // its slot to a waiting block instead of idling at the closing barrier
  // (measured faster than one wave of longer-running blocks).
  const unsigned grid = grid_for(t, n * G, kUpdThreads, 2 * kUpdBlocksPerSm);
  KernelTimer timer(t->prof, HKV_K_UPDATE, st);
  if (vec16)
    launch_table_kernel(t, update_kernel<G, true, UPSERT>, grid, kUpdThreads, 0, st, t->dev, s,
                        values, scores, ctx);
  else
    launch_table_kernel(t, update_kernel<G, false, UPSERT>, grid, kUpdThreads, 0, st, t->dev, s,
                        values, scores, ctx);
}

template <bool UPSERT>
void launch_update(hkv_table_s* t, uint64_t n, const Scratch& s, const float* values,
                   const uint64_t* scores, ScoreCtx ctx, bool vec16, cudaStream_t st) {
  switch (t->launch.update_tpk) {
    case 1: launch_update_g<1, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
    case 2: launch_update_g<2, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
    case 4: launch_update_g<4, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
    case 16: launch_update_g<16, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
    case 32: launch_update_g<32, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
    default: launch_update_g<8, UPSERT>(t, n, s, values, scores, ctx, vec16, st); break;
  }
}

void launch_dedup(hkv_table_s* t, uint64_t n, const uint64_t* keys, const Scratch& s,
                  cudaStream_t st) {
  const unsigned grid = (unsigned)((n + kDedupTile - 1) / kDedupTile);
  KernelTimer timer(t->prof, HKV_K_DEDUP, st);
  if (grid > (unsigned)t->num_sms * 6)
    dedup_kernel<7><<<grid, kDedupThreads, kDedupSmem, st>>>(n, keys, s, t->dev,
                                                             t->opts.deterministic);
  else
    dedup_kernel<6><<<grid, kDedupThreads, kDedupSmem, st>>>(n, keys, s, t->dev,
                                                             t->opts.deterministic);
}

// The waves of the ordered phase I, driven from the host: waves go out in
// groups of kWavesPerCheck, and the last wave's pending count comes back
// before the next group is launched (a wave with nothing pending costs two
// short kernels; a host round trip per wave cost more). The call returns
// only after phase I has finished; the rest of the pipeline stays queued.
constexpr int kWavesPerCheck = 4;

hkv_status run_ordered_phase_i(hkv_table_s* t, uint64_t n, const Scratch& s, const float* values,
                               const uint64_t* scores, ScoreCtx ctx, bool vec16,
                               cudaStream_t st) {
  KernelTimer timer(t->prof, HKV_K_INSERT, st);
  {
    // all waves in one cooperative launch, one grid of resident blocks
    void (*k)(TableDev, Scratch, const float*, const uint64_t*, ScoreCtx) =
        vec16 ? ordered_waves_kernel<true> : ordered_waves_kernel<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kOrdThreads, 0) ==
            cudaSuccess &&
        per_sm > 0) {
      TableDev dv = t->dev;
      Scratch sv = s;
      const float* vv = values;
      const uint64_t* sc = scores;
      ScoreCtx cv = ctx;
      void* args[] = {&dv, &sv, &vv, &sc, &cv};
      const unsigned grid = (unsigned)std::max<uint64_t>(
          1, std::min<uint64_t>((uint64_t)t->num_sms * (unsigned)per_sm,
                                (n + kOrdThreads - 1) / kOrdThreads));
      if (cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), grid, kOrdThreads, args, 0, st) ==
          cudaSuccess)
        return HKV_OK;
    }
    cudaGetLastError();  // refused: fall back to one launch pair per wave
  }
  const unsigned og = grid_for(t, n, kOrdThreads, 8);
  for (uint64_t wave = 1;; ) {
    for (int k = 0; k < kWavesPerCheck; ++k, ++wave) {
      cudaMemsetAsync(s.cnt + kCntPending, 0, 8, st);
      ordered_bid_kernel<<<og, kOrdThreads, 0, st>>>(t->dev, s, wave);
      if (vec16)
        ordered_insert_kernel<true><<<og, kOrdThreads, 0, st>>>(t->dev, s, values, scores, ctx,
                                                                 wave);
      else
        ordered_insert_kernel<false><<<og, kOrdThreads, 0, st>>>(t->dev, s, values, scores, ctx,
                                                                  wave);
    }
    cudaMemcpyAsync(t->host_word, s.cnt + kCntPending, 8, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "ordered phase I");
    if (*t->host_word == 0) return HKV_OK;
    if (wave > n + kWavesPerCheck) {  // cannot happen: each wave places the smallest pending key
      set_last_error("ordered phase I made no progress");
      return HKV_ERR_TIMEOUT;
    }
  }
}

}  // namespace

// Phase I, reconcile and status of a plain upsert as one cooperative launch
// (insert_finish_kernel); false if the launch was refused, and the caller
// launches insert_kernel and the finish instead.
template <bool VEC16>
bool launch_insert_finish_t(hkv_table_s* t, uint64_t n, const Scratch& s, const float* values,
                            const uint64_t* scores, ScoreCtx ctx, uint64_t* ev_keys,
                            uint64_t* ev_scores, float* ev_values, uint8_t* status_out,
                            uint64_t* n_evicted, cudaStream_t st) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, insert_finish_kernel<VEC16>, kInsThreads,
                                                      0) != cudaSuccess) {
      cudaGetLastError();
      b = 0;
    }
    return b;
  }();
  if (per_sm <= 0) return false;
  const unsigned grid = grid_for(t, (n + 31) / 32 * 32, kInsThreads,
                                 std::min(per_sm, kInsBlocksPerSm));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kInsThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[2]{};
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  unsigned na = 1;
  if (t->l2win.num_bytes) {
    attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[1].val.accessPolicyWindow = t->l2win;
    na = 2;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  KernelTimer timer(t->prof, HKV_K_INSERT, st);
  if (cudaLaunchKernelEx(&cfg, insert_finish_kernel<VEC16>, t->dev, s, values, scores, ctx,
                         ev_keys, ev_scores, ev_values, n, status_out, n_evicted) == cudaSuccess)
    return true;
  cudaGetLastError();
  return false;
}

bool launch_insert_finish(hkv_table_s* t, uint64_t n, const Scratch& s, const float* values,
                          const uint64_t* scores, ScoreCtx ctx, bool vec16, uint64_t* ev_keys,
                          uint64_t* ev_scores, float* ev_values, uint8_t* status_out,
                          uint64_t* n_evicted, cudaStream_t st) {
  return vec16 ? launch_insert_finish_t<true>(t, n, s, values, scores, ctx, ev_keys, ev_scores,
                                              ev_values, status_out, n_evicted, st)
               : launch_insert_finish_t<false>(t, n, s, values, scores, ctx, ev_keys, ev_scores,
                                               ev_values, status_out, n_evicted, st);
}

// Reconcile and status of a plain upsert as one cooperative launch
// (finish_kernel); false if the launch was refused, and the caller launches
// the two kernels instead.
bool launch_finish(hkv_table_s* t, uint64_t n, const Scratch& s, uint64_t* ev_keys,
                   uint64_t* ev_scores, float* ev_values, uint8_t* status_out,
                   uint64_t* n_evicted, cudaStream_t st) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, finish_kernel, kRecThreads, 0) !=
        cudaSuccess) {
      cudaGetLastError();
      b = 0;
    }
    return b;
  }();
  if (per_sm <= 0) return false;
  const unsigned grid = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((uint64_t)t->num_sms * (unsigned)per_sm,
                            (n + kRecThreads * kRecPerThread - 1) / (kRecThreads * kRecPerThread)));
  TableDev dv = t->dev;
  Scratch sv = s;
  uint64_t nn = n;
  void* args[] = {&dv, &sv, &ev_keys, &ev_scores, &ev_values, &nn, &status_out, &n_evicted};
  KernelTimer timer(t->prof, HKV_K_STATUS, st);
  if (cudaLaunchCooperativeKernel(reinterpret_cast<void*>(finish_kernel), grid, kRecThreads, args,
                                  0, st) == cudaSuccess)
    return true;
  cudaGetLastError();
  return false;
}

hkv_status launch_upsert(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                         const uint64_t* scores, uint8_t* status_out, uint64_t* ev_keys,
                         uint64_t* ev_scores, float* ev_values, uint64_t* n_evicted,
                         ScoreCtx ctx, cudaStream_t st, bool keep_hits, const float* gather_src) {
  if (n == 0) {
    if (n_evicted) cudaMemsetAsync(n_evicted, 0, 8, st);
    return cuda_status(cudaGetLastError(), "upsert");
  }
  ScratchAlloc a;
  hkv_status rc = alloc_scratch(t, n, true, ev_values != nullptr, st, &a);
  if (rc) return rc;
  a.s.keep_hits = keep_hits ? 1 : 0;
  a.s.row_prefetch = in_device_memory(values) ? 1 : 0;
  const Scratch& s = a.s;
  const bool vec16 = row_vector_bytes(t, values, gather_src) == 16;
  launch_dedup(t, n, keys, s, st);
  if (gather_src) {
    // values is the staging array: fill the rows the later phases read
    const uint64_t rows_max = n * (vec16 ? t->dev.dim / 4 : t->dev.dim);
    gather_last_rows_kernel<<<grid_for(t, rows_max, kGatherThreads, 8), kGatherThreads, 0, st>>>(
        s, gather_src, const_cast<float*>(values), t->dev.dim, vec16 ? 1 : 0);
  }
  launch_update<true>(t, n, s, values, scores, ctx, vec16, st);
  // without host rows or ordered waves, phase I, reconcile and status run
  // as one cooperative launch
  bool finished = false;
  if (s.owner) {
    rc = run_ordered_phase_i(t, n, s, values, scores, ctx, vec16, st);
    if (rc) {
      cudaFreeAsync(a.base, st);
      return rc;
    }
  } else if (!s.gdefer && launch_insert_finish(t, n, s, values, scores, ctx, vec16, ev_keys,
                                                ev_scores, ev_values, status_out, n_evicted,
                                                st)) {
    finished = true;
  } else {
    const unsigned ig = grid_for(t, (n + 31) / 32 * 32, kInsThreads, kInsBlocksPerSm);
    KernelTimer timer(t->prof, HKV_K_INSERT, st);
    if (vec16)
      launch_table_kernel(t, insert_kernel<true>, ig, kInsThreads, 0, st, t->dev, s, values,
                          scores, ctx);
    else
      launch_table_kernel(t, insert_kernel<false>, ig, kInsThreads, 0, st, t->dev, s, values,
                          scores, ctx);
  }
  if (s.gdefer) {
    {
      KernelTimer timer(t->prof, HKV_K_HOSTROWS, st);
      RegionOrder ro;
      rc = region_sort(t, s.gdefer, n, s.cnt + kCntUnique, a.region, &ro, st);
      if (rc) {
        cudaFreeAsync(a.base, st);
        return rc;
      }
      const unsigned fg = grid_for(t, n * kFlushLanes, kFlushThreads, 8);
      if (vec16)
        flush_deferred_rows_kernel<true><<<fg, kFlushThreads, 0, st>>>(t->dev, s, ro, values);
      else
        flush_deferred_rows_kernel<false><<<fg, kFlushThreads, 0, st>>>(t->dev, s, ro, values);
    }
  }
  if (!finished &&
      !launch_finish(t, n, s, ev_keys, ev_scores, ev_values, status_out, n_evicted, st)) {
    {
      KernelTimer timer(t->prof, HKV_K_RECONCILE, st);
      reconcile_kernel<<<reconcile_grid(t, n), kRecThreads, 0, st>>>(
          t->dev, s, ev_keys, ev_scores, ev_values);
    }
    if (status_out || n_evicted) {
      KernelTimer timer(t->prof, HKV_K_STATUS, st);
      status_kernel<<<grid_for(t, n, 256, 8), 256, 0, st>>>(n, s, status_out, n_evicted);
    }
  }
  cudaFreeAsync(a.base, st);
  return cuda_status(cudaGetLastError(), "insert_or_assign launch");
}

hkv_status launch_assign(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                         const uint64_t* scores, ScoreCtx ctx, cudaStream_t st) {
  if (n == 0) return HKV_OK;
  ScratchAlloc a;
  hkv_status rc = alloc_scratch(t, n, false, false, st, &a);
  if (rc) return rc;
  const bool vec16 = row_vector_bytes(t, values) == 16;
  launch_dedup(t, n, keys, a.s, st);
  launch_update<false>(t, n, a.s, values, scores, ctx, vec16, st);
  cudaFreeAsync(a.base, st);
  return cuda_status(cudaGetLastError(), "assign launch");
}

hkv_status launch_erase(hkv_table_s* t, uint64_t n, const uint64_t* keys, cudaStream_t st) {
  if (n == 0) return HKV_OK;
  // Only the abort word of the scratch block is used here.
  void* base = nullptr;
  if (cudaMallocFromPoolAsync(&base, 256, t->pool, st) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("scratch allocation failed");
    return HKV_ERR_OOM;
  }
  Scratch s{};
  s.cnt = static_cast<unsigned long long*>(base);
  cudaMemsetAsync(s.cnt, 0, kCntWords * 8, st);
  KernelTimer timer(t->prof, HKV_K_ERASE, st);
  validate_kernel<<<grid_for(t, n, 256, 8), 256, 0, st>>>(n, keys, s, t->dev.err);
  erase_kernel<8><<<grid_for(t, n * 8, kUpdThreads, 2048 / kUpdThreads), kUpdThreads, 0, st>>>(
      t->dev, n, keys, s);
  cudaFreeAsync(base, st);
  return cuda_status(cudaGetLastError(), "erase launch");
}

}  // namespace hkv

// ------------------------------------------- upsert into caller-given scratch

namespace hkv {
namespace {

// Lay the per-call scratch out in a caller-provided block (no allocation);
// returns false if the block is too small. Evicted values are not kept.
bool carve_scratch(void* base, uint64_t bytes, uint64_t n, Scratch* out) {
  int bits = 10;
  while ((1ull << bits) < 2 * n) ++bits;
  const uint64_t T = 1ull << bits;
  const uint64_t sz_tab = align256(T * sizeof(DedupEntry));
  const uint64_t sz_ts = align256(T);
  const uint64_t sz_u8 = align256(n);
  const uint64_t sz_u32 = align256(n * 4);
  const uint64_t sz_u64 = align256(n * 8);
  const uint64_t sz_cnt = align256(kCntWords * 8);
  const uint64_t total = sz_tab + sz_ts + 4 * sz_u32 + sz_cnt + sz_u8 + 3 * sz_u64;
  if (total > bytes) return false;
  char* p = static_cast<char*>(base);
  Scratch s{};
  s.tab = reinterpret_cast<DedupEntry*>(p); p += sz_tab;
  s.tab_bits = bits;
  s.tab_mask = T - 1;
  s.tstatus = reinterpret_cast<uint8_t*>(p); p += sz_ts;
  s.slot_of = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.ulist = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.cnt = reinterpret_cast<unsigned long long*>(p); p += sz_cnt;
  s.mflag = reinterpret_cast<uint8_t*>(p); p += sz_u8;
  s.mkey = reinterpret_cast<uint64_t*>(p); p += sz_u64;
  s.evk = reinterpret_cast<uint64_t*>(p); p += sz_u64;
  s.evs = reinterpret_cast<uint64_t*>(p); p += sz_u64;
  s.mi = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.mm = reinterpret_cast<uint32_t*>(p); p += sz_u32;
  s.evv = nullptr;
  *out = s;
  return true;
}

}  // namespace

hkv_status launch_upsert_in(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                            const uint64_t* scores, uint8_t* status_out, uint64_t* ev_keys,
                            uint64_t* ev_scores, uint64_t* n_evicted, ScoreCtx ctx,
                            void* scratch, uint64_t scratch_bytes, cudaStream_t st) {
  if (n == 0) {
    if (n_evicted) cudaMemsetAsync(n_evicted, 0, 8, st);
    return cuda_status(cudaGetLastError(), "upsert");
  }
  if (t->opts.deterministic && t->dev.dual) {
    set_last_error("deterministic dual-bucket tables take hkv_insert_or_assign only");
    return HKV_ERR_INVALID_ARG;
  }
  Scratch s;
  if (!carve_scratch(scratch, scratch_bytes, n, &s)) {
    set_last_error("batch too large for the scratch block");
    return HKV_ERR_INVALID_ARG;
  }
  // The block keeps the previous call's contents: reset what must start
  // empty or zero.
  cudaMemsetAsync(s.tab, 0xFF, (s.tab_mask + 1) * sizeof(DedupEntry), st);
  cudaMemsetAsync(s.cnt, 0, kCntWords * 8, st);
  s.row_prefetch = in_device_memory(values) ? 1 : 0;
  const bool vec16 = row_vector_bytes(t, values) == 16;
  launch_dedup(t, n, keys, s, st);
  launch_update<true>(t, n, s, values, scores, ctx, vec16, st);
  {
    const unsigned ig = grid_for(t, (n + 31) / 32 * 32, kInsThreads, kInsBlocksPerSm);
    KernelTimer timer(t->prof, HKV_K_INSERT, st);
    if (vec16)
      launch_table_kernel(t, insert_kernel<true>, ig, kInsThreads, 0, st, t->dev, s, values,
                          scores, ctx);
    else
      launch_table_kernel(t, insert_kernel<false>, ig, kInsThreads, 0, st, t->dev, s, values,
                          scores, ctx);
  }
  {
    KernelTimer timer(t->prof, HKV_K_RECONCILE, st);
    reconcile_kernel<<<reconcile_grid(t, n), kRecThreads, 0, st>>>(
        t->dev, s, ev_keys, ev_scores, nullptr);
  }
  if (status_out || n_evicted) {
    KernelTimer timer(t->prof, HKV_K_STATUS, st);
    status_kernel<<<grid_for(t, n, 256, 8), 256, 0, st>>>(n, s, status_out, n_evicted);
  }
  return cuda_status(cudaGetLastError(), "insert_or_assign launch");
}

}  // namespace hkv

// ------------------------------------------------ batched rounds (OpDesc)

namespace hkv {
namespace {

// Reset the dedup table entries a round of d->n keys uses, and the counters.
__global__ void clear_kernel(Scratch s) {
  const uint64_t T = 1ull << tab_bits_for(s.d->n);
  uint4* p = reinterpret_cast<uint4*>(s.tab);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
       i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
  if (blockIdx.x == 0 && threadIdx.x < kCntWords) s.cnt[threadIdx.x] = 0;
}

}  // namespace

uint64_t upsert_scratch_bytes(uint64_t n) {
  const uint64_t T = 1ull << tab_bits_for(n);
  return align256(T * sizeof(DedupEntry)) + align256(T) + 4 * align256(n * 4) +
         align256(kCntWords * 8) + align256(n) + 3 * align256(n * 8);
}

hkv_status launch_upsert_desc(hkv_table_s* t, uint64_t n_max, const OpDesc* d, void* scratch,
                              uint64_t scratch_bytes, cudaStream_t st) {
  Scratch s;
  const uint64_t n = n_max ? n_max : 1;
  if (!carve_scratch(scratch, scratch_bytes, n, &s)) {
    set_last_error("batch slot scratch too small");
    return HKV_ERR_INVALID_ARG;
  }
  s.d = d;
  const bool vec16 = row_vector_bytes(t, nullptr) == 16;  // rows checked 16-byte aligned
  clear_kernel<<<grid_for(t, s.tab_mask + 1, 256, 8), 256, 0, st>>>(s);
  launch_dedup(t, n, nullptr, s, st);
  launch_update<true>(t, n, s, nullptr, nullptr, ScoreCtx{0, 0}, vec16, st);
  const unsigned ig = grid_for(t, (n + 31) / 32 * 32, kInsThreads, kInsBlocksPerSm);
  if (vec16)
    launch_table_kernel(t, insert_kernel<true>, ig, kInsThreads, 0, st, t->dev, s,
                        (const float*)nullptr, (const uint64_t*)nullptr, ScoreCtx{0, 0});
  else
    launch_table_kernel(t, insert_kernel<false>, ig, kInsThreads, 0, st, t->dev, s,
                        (const float*)nullptr, (const uint64_t*)nullptr, ScoreCtx{0, 0});
  reconcile_kernel<<<reconcile_grid(t, n), kRecThreads, 0, st>>>(t->dev, s, nullptr, nullptr,
                                                                 nullptr);
  status_kernel<<<grid_for(t, n, 256, 8), 256, 0, st>>>(n, s, nullptr, nullptr);
  return cuda_status(cudaGetLastError(), "batched upsert launch");
}

}  // namespace hkv

// ---------------------------------------------------------- find_or_insert

namespace hkv {
namespace {

// found[i] = 1 iff the key was resident at batch start (status UPDATED).
__global__ void status_to_found_kernel(uint64_t n, uint8_t* flags) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = flags[i] == HKV_ST_UPDATED ? 1 : 0;
}

}  // namespace

hkv_status launch_find_or_insert(hkv_table_s* t, uint64_t n, const uint64_t* keys,
                                 float* values_io, const uint64_t* scores, uint8_t* found_out,
                                 ScoreCtx ctx, cudaStream_t st) {
  // phase U without the value write, phase I as insert_or_assign (the
  // caller's rows are the values of new keys), then every row of a key
  // resident now is overwritten with its stored value
  hkv_status rc = launch_upsert(t, n, keys, values_io, scores, found_out, nullptr, nullptr,
                                nullptr, nullptr, ctx, st, true);
  if (rc) return rc;
  rc = launch_find(t, n, keys, values_io, nullptr, nullptr, st);
  if (rc) return rc;
  if (found_out && n)
    status_to_found_kernel<<<grid_for(t, n, 256, 8), 256, 0, st>>>(n, found_out);
  return cuda_status(cudaGetLastError(), "find_or_insert launch");
}

}  // namespace hkv
