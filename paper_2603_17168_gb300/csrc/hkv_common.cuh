// Device-side building blocks shared by the hot-path kernels (sm_103a).
//
// Table layout in HBM (Sec. 3.2, Fig. 4; Sec. 3.6; Sec. 4.2):
//   digests [B][128] uint8   one 128-byte line per bucket; 0 = empty slot
//   kv      [B][128][2] uint64  each slot's (key, score) as one 16-byte pair:
//                            key 2^64-1 = empty, 2^64-2 = locked (slot CAS
//                            lock); the score is the eviction metadata
//                            itself (Sec. 3.3). A key confirmation brings the
//                            score's sector along, a claim writes key and
//                            score in one sector, and a victim search reads
//                            one 2 KiB run per bucket.
//   sizes   [B] uint32       occupied (or claimed) slots per bucket: the
//                            dual-bucket choice reads two counters instead
//                            of counting 256 digests
//   values  slices of (1 << slice_shift) slots x dim fp32, addressed by the
//           global slot g = bucket * 128 + position; slice 0.. in HBM, the
//           rest in pinned, mapped host memory (position-based addressing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hkv.h"

#ifndef HKV_COPY_ROW_R
#define HKV_COPY_ROW_R 1
#endif

namespace hkv {

constexpr uint32_t kSlots = 128;
constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint64_t kLockedKey = ~0ull - 1;
constexpr uint64_t kFirstReserved = 1ull << 63;
constexpr uint64_t kH2Salt = 0x9E3779B97F4A7C15ull;  // second-hash salt (dual mode)
constexpr int kMaxClaimAttempts = 4096;             // bound on slot-claim retries
constexpr uint64_t kNoHostSlot = ~0ull;             // "no host row" in host-row lists

// A list of item indices grouped by the 2 MiB host region of their slots
// (region_sort): order[0 .. *count).
struct RegionOrder {
  uint32_t* order;
  unsigned long long* count;
};

struct TableDev {
  uint8_t* digests;
  uint64_t* kv;              // [B][128] (key, score) pairs
  uint32_t* sizes;           // [B] slots claimed per bucket
  float* values0;            // slice 0 base
  float* const* slices;      // [n_slices] slice bases (device array)
  uint64_t bucket_mask;      // B - 1
  uint32_t dim;
  uint32_t slice_shift;      // log2(slots per slice)
  int32_t policy;
  int32_t dual;
  int32_t vec8;              // copies without 16-byte vectors use 8-byte ones
  uint32_t* err;             // latched device error (first error wins)
  unsigned long long* counters;  // [HKV_COUNTER_COUNT]
};

struct ScoreCtx {
  uint64_t step;
  uint64_t epoch;
};

// One table's work in a batched round, kept in device memory so that a
// captured launch sequence can be replayed with new sizes and buffers: the
// kernels read their size, pointers and score context from here when given
// one.
struct OpDesc {
  uint64_t n;
  const uint64_t* keys;
  const float* values_in;   // upsert input rows
  float* values_out;        // find output rows
  uint8_t* flags;           // find: found; upsert: status (may be null)
  const uint64_t* scores;   // caller scores (HKV_CUSTOM), else null
  uint64_t step;
  uint64_t epoch;
  int row_prefetch;         // values_in is device memory (bulk L2 prefetch allowed)
};

// log2 of the dedup table size for a batch of n keys (>= 2n, >= 1024).
__host__ __device__ __forceinline__ int tab_bits_for(uint64_t n) {
  int b = 10;
  while ((1ull << b) < 2 * n) ++b;
  return b;
}

// ------------------------------------------------------------------ hashing

// MurmurHash3 64-bit finaliser (public-domain construction): the table's
// key hash. b1 = h & (B-1); digest = bits 32..39 of h, 0 folded onto 1.
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint32_t digest_from_hash(uint64_t h) {
  uint32_t d = (uint32_t)(h >> 32) & 0xFFu;
  return d == 0 ? 1u : d;
}

__device__ __forceinline__ uint64_t second_bucket(const TableDev& t, uint64_t key) {
  return fmix64(key ^ kH2Salt) & t.bucket_mask;
}

// Key and score words of global slot g.
__host__ __device__ __forceinline__ uint64_t* key_ptr(const TableDev& t, uint64_t g) {
  return t.kv + 2 * g;
}
__host__ __device__ __forceinline__ uint64_t* score_ptr(const TableDev& t, uint64_t g) {
  return t.kv + 2 * g + 1;
}

// ------------------------------------------------------------ value arena

__device__ __forceinline__ float* value_ptr(const TableDev& t, uint64_t g) {
  uint64_t s = g >> t.slice_shift;
  if (s == 0) return t.values0 + g * t.dim;
  return t.slices[s] + (g & ((1ull << t.slice_shift) - 1)) * t.dim;
}

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ void latch_error(uint32_t* err, uint32_t code) {
  atomicCAS(err, 0u, code);
}

__device__ __forceinline__ void count_add(const TableDev& t, int which, unsigned long long v) {
  if (v) atomicAdd(t.counters + which, v);
}

__device__ __forceinline__ bool sk_less(uint64_t s1, uint64_t k1, uint64_t s2, uint64_t k2) {
  return s1 < s2 || (s1 == s2 && k1 < k2);
}

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b, uint64_t cap) {
  uint64_t bb = b < cap ? b : cap;
  return a > cap - bb ? cap : a + bb;
}

// Score of a key under the table policy (see hkv_policy in hkv.h).
__device__ __forceinline__ uint64_t policy_score(int policy, bool hit, uint64_t old, uint64_t m,
                                                 bool have_caller, uint64_t caller,
                                                 const ScoreCtx& c) {
  switch (policy) {
    case HKV_LRU:
      return c.step;
    case HKV_LFU:
      return hit ? sat_add(old, m, ~0ull) : m;
    case HKV_EPOCH_LRU:
      return (c.epoch << 32) | (c.step & 0xFFFFFFFFull);
    case HKV_EPOCH_LFU: {
      uint64_t f = hit ? sat_add(old & 0xFFFFFFFFull, m, 0xFFFFFFFFull)
                       : (m < 0xFFFFFFFFull ? m : 0xFFFFFFFFull);
      return (c.epoch << 32) | f;
    }
    case HKV_CUSTOM:
      return have_caller ? caller : old;
    default: {  // HKV_CUSTOM_TS_FREQ
      uint64_t f = hit ? sat_add(old & 0xFFFFull, m, 0xFFFFull) : (m < 0xFFFFull ? m : 0xFFFFull);
      return (c.epoch << 16) | f;
    }
  }
}

// ------------------------------------------------------ block-level atomics
//
// Atomics with a return value on one address serialise in L2; issued per
// warp they dominated whole kernels. These helpers aggregate a block first
// and touch the global word once per block. Every thread of the block must
// call them (they synchronise the block).

// Add per-thread values to NC table counters, one global atomic per counter
// per block.
template <int NC>
__device__ __forceinline__ void flush_counts(const TableDev& t, const int (&which)[NC],
                                             const unsigned (&vals)[NC]) {
  __shared__ unsigned long long acc[NC];
  if (threadIdx.x < NC) acc[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const unsigned w = __reduce_add_sync(0xFFFFFFFFu, vals[c]);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&acc[c], (unsigned long long)w);
  }
  __syncthreads();
  if (threadIdx.x < NC && acc[threadIdx.x]) atomicAdd(t.counters + which[threadIdx.x], acc[threadIdx.x]);
}

// Reserve `count` consecutive list positions per thread from a global
// counter; returns this thread's first position.
__device__ __forceinline__ unsigned long long block_reserve(unsigned long long* counter,
                                                            unsigned count) {
  __shared__ unsigned wsum[32];
  __shared__ unsigned long long base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned incl = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < nw; ++w) {
      const unsigned c = wsum[w];
      wsum[w] = tot;
      tot += c;
    }
    base = tot ? atomicAdd(counter, (unsigned long long)tot) : 0ull;
  }
  __syncthreads();
  const unsigned long long pos = base + wsum[wid] + (incl - count);
  __syncthreads();
  return pos;
}

// Byte mask of slots whose digest byte equals the pattern: SIMD compare of
// four digests per 32-bit word (Algorithm 1's __vcmpeq4 step).
__device__ __forceinline__ uint32_t match4(uint32_t word, uint32_t pat4) {
  return __vcmpeq4(word, pat4);
}

// Load this lane's share (128/G bytes) of a bucket's digest line.
// Read-only path unless CG (cache-global, bypass L1) is asked for.
template <int G, bool CG>
__device__ __forceinline__ void load_line(const uint8_t* line, int lane_g, uint32_t (&w)[32 / G]) {
  constexpr int W = 32 / G;  // 32-bit words per lane
  if constexpr (W >= 4) {
    const uint4* p = reinterpret_cast<const uint4*>(line) + lane_g * (W / 4);
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      uint4 v = CG ? __ldcg(p + q) : __ldg(p + q);
      w[4 * q + 0] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
  } else if constexpr (W == 2) {
    const uint2* p = reinterpret_cast<const uint2*>(line) + lane_g;
    uint2 v = CG ? __ldcg(p) : __ldg(p);
    w[0] = v.x; w[1] = v.y;
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(line) + lane_g;
    w[0] = CG ? __ldcg(p) : __ldg(p);
  }
}

// The rest of a probe, for a lane whose share of the bucket held more
// digest matches than the first pass recorded: walk the share again and
// confirm every match other than c0..c2. Rare, so kept out of line (it
// would otherwise hold registers across the common path).
template <int G, bool CG>
__device__ __noinline__ int probe_rest(const uint8_t* line, const uint64_t* kb, uint64_t key,
                                       uint32_t pat4, int lane_g, int c0, int c1, int c2,
                                       unsigned* key_reads) {
  constexpr int W = 32 / G;
  const int first = lane_g * (128 / G);
  uint32_t w[W];
  load_line<G, CG>(line, lane_g, w);
  int my = -1;
  unsigned reads = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    uint32_t m = match4(w[q], pat4);
    while (m) {
      const int bit = __ffs(m) - 1;
      const int slot = first + q * 4 + (bit >> 3);
      m &= ~(0xFFu << (bit & ~7));
      if (slot == c0 || slot == c1 || slot == c2) continue;
      const uint64_t k = CG ? __ldcg(kb + 2 * slot) : __ldg(kb + 2 * slot);
      reads++;
      if (k == key) my = slot;
    }
  }
  *key_reads += reads;
  return my;
}

// Probe one bucket for `key` with a group of G lanes (G divides 32). Each
// lane compares its 128/G digests and confirms matches against the full
// key. Every lane of the warp must call this (it ends with a warp ballot).
// Returns the slot (0..127) of the key in the bucket, or -1; identical on
// all lanes of a group. Adds the full-key loads this lane made to key_reads.
//
// TWO_PASS: a lane waits on key memory once per bucket rather than once per
// matching digest word: the first pass only records up to three digest
// matches of the lane's share, whose key words are then loaded together. A
// full bucket holds about 0.5 false matches per probe (128 digests of 255
// values), so a lane whose three candidates were all false and whose share
// held more (well under 1% of probes) re-walks the line for the rest. This
// pays off in kernels with few warps per SM to hide latency (the update
// phase); at full occupancy the one-pass form, which confirms each match as
// it meets it, issues fewer instructions (find).
//
// FREE (two-pass form only): the digest words the probe already holds also
// give the bucket's free slots (digest byte 0) as they were when the line
// was read. *fi receives, on every lane of the group, their number and one
// of them packed as free_info(count, slot), slot -1 when there is none: the
// group lane `pick >> 8` (mod G) offers it, the free byte of its share
// nearest to word `pick & 255` (mod 32/G), so keys claiming in one bucket
// tend to pick different slots. (One packed word keeps the update kernel
// within its register budget.)
__device__ __forceinline__ unsigned free_info(int count, int slot) {
  return ((unsigned)count << 8) | (unsigned)(slot + 1);
}
__device__ __forceinline__ int free_count(unsigned fi) { return (int)(fi >> 8); }
__device__ __forceinline__ int free_slot_of(unsigned fi) { return (int)(fi & 255u) - 1; }

template <int G, bool CG, bool TWO_PASS, bool FREE = false>
__device__ __forceinline__ int probe_bucket(const TableDev& t, uint64_t b, uint64_t key,
                                            uint32_t pat4, bool active, int lane_g,
                                            unsigned group_bits, int group_base,
                                            unsigned& key_reads, unsigned pick = 0,
                                            unsigned* fi = nullptr) {
  constexpr int W = 32 / G;
  int my = -1;
  int nfree = 0, free_slot = -1;
  if (active && !TWO_PASS) {
    uint32_t w[W];
    load_line<G, CG>(t.digests + b * kSlots, lane_g, w);
    const uint64_t* kb = key_ptr(t, b * kSlots);  // key of slot j at kb[2 j]
#pragma unroll
    for (int q = 0; q < W; ++q) {
      uint32_t m = match4(w[q], pat4);
      while (m) {
        const int bit = __ffs(m) - 1;
        const int slot = lane_g * (128 / G) + q * 4 + (bit >> 3);
        const uint64_t k = CG ? __ldcg(kb + 2 * slot) : __ldg(kb + 2 * slot);
        key_reads++;
        if (k == key) my = slot;
        m &= ~(0xFFu << (bit & ~7));
      }
    }
  } else if (active) {
    const uint8_t* line = t.digests + b * kSlots;
    const uint64_t* kb = key_ptr(t, b * kSlots);  // key of slot j at kb[2 j]
    const int first = lane_g * (128 / G);
    int c0 = -1, c1 = -1, c2 = -1;
    bool more = false;
    auto push = [&](int slot) {
      if (c0 < 0) c0 = slot;
      else if (c1 < 0) c1 = slot;
      else if (c2 < 0) c2 = slot;
      else more = true;
    };
    {
      uint32_t w[W];
      load_line<G, CG>(line, lane_g, w);
      int best = W;  // distance of free_slot's word from the start word
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const uint32_t m = match4(w[q], pat4);
        if (m) {  // 0xFF per matching byte: record the lowest and highest
          const int sa = first + q * 4 + ((__ffs(m) - 1) >> 3);
          const int sb = first + q * 4 + ((31 - __clz(m)) >> 3);
          push(sa);
          if (sb != sa) push(sb);
          more |= __popc(m) > 16;
        }
        if constexpr (FREE) {
          const uint32_t z = __vcmpeq4(w[q], 0u);
          nfree += __popc(z) >> 3;
          const int d = (q - (int)(pick & 255u)) & (W - 1);
          if (z && d < best) {
            best = d;
            free_slot = first + q * 4 + ((__ffs(z) - 1) >> 3);
          }
        }
      }
    }
    uint64_t k0 = 0, k1 = 0, k2 = 0;
    if (c0 >= 0) k0 = CG ? __ldcg(kb + 2 * c0) : __ldg(kb + 2 * c0);
    if (c1 >= 0) k1 = CG ? __ldcg(kb + 2 * c1) : __ldg(kb + 2 * c1);
    if (c2 >= 0) k2 = CG ? __ldcg(kb + 2 * c2) : __ldg(kb + 2 * c2);
    key_reads += (c0 >= 0) + (c1 >= 0) + (c2 >= 0);
    if (c0 >= 0 && k0 == key) my = c0;
    else if (c1 >= 0 && k1 == key) my = c1;
    else if (c2 >= 0 && k2 == key) my = c2;
    else if (more) my = probe_rest<G, CG>(line, kb, key, pat4, lane_g, c0, c1, c2, &key_reads);
  }
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, my >= 0) & group_bits;
  const int src = bal ? __ffs(bal) - 1 : group_base;
  const int slot = __shfl_sync(0xFFFFFFFFu, my, src);
  if constexpr (FREE) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) nfree += __shfl_xor_sync(0xFFFFFFFFu, nfree, o);
    // the offering lane: the first lane with a free byte from lane pick >> 8
    const unsigned offer = __ballot_sync(0xFFFFFFFFu, free_slot >= 0) & group_bits;
    const unsigned rel = G == 32 ? offer : (offer >> group_base) & ((1u << G) - 1u);
    const int rot = (int)((pick >> 8) & (unsigned)(G - 1));
    const uint64_t twice = (uint64_t)rel | ((uint64_t)rel << G);  // rotation without wrap
    const uint64_t from = twice >> rot;
    const int off = from ? (__ffsll((long long)from) - 1 + rot) & (G - 1) : 0;
    const int fs = __shfl_sync(0xFFFFFFFFu, free_slot, group_base + off);
    *fi = free_info(nfree, offer ? fs : -1);
  }
  return bal ? slot : -1;
}

// Copy one value row of `dim` floats with G cooperating lanes, using 16-byte
// vectors when VEC16 (dim % 4 == 0 and 16-byte aligned rows), else 8-byte
// vectors when vec8 (set by the launcher for even dim and 8-byte aligned
// rows), else 4-byte words. Each lane issues R loads before it stores them,
// so a row costs one memory latency per R vectors per lane rather than one
// per vector (rows in mapped host memory are a link round trip away).
template <int G, bool VEC16, bool STREAM_DST, int R = HKV_COPY_ROW_R>
__device__ __forceinline__ void copy_row(float* dst, const float* src, uint32_t dim, int lane_g,
                                         bool vec8 = false) {
  if constexpr (VEC16) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    const uint32_t n4 = dim >> 2;
    for (uint32_t j0 = lane_g; j0 < n4; j0 += R * G) {
      float4 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (j0 + r * G < n4) v[r] = __ldg(s4 + j0 + r * G);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (j0 + r * G >= n4) break;
        if (STREAM_DST) __stcs(d4 + j0 + r * G, v[r]); else d4[j0 + r * G] = v[r];
      }
    }
  } else if (vec8 && (dim & 1) == 0 &&
             ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 7) == 0) {
    const float2* s2 = reinterpret_cast<const float2*>(src);
    float2* d2 = reinterpret_cast<float2*>(dst);
    for (uint32_t j = lane_g; j < (dim >> 1); j += G) {
      float2 v = __ldg(s2 + j);
      if (STREAM_DST) __stcs(d2 + j, v); else d2[j] = v;
    }
  } else {
    for (uint32_t j = lane_g; j < dim; j += G) {
      float v = __ldg(src + j);
      if (STREAM_DST) __stcs(dst + j, v); else dst[j] = v;
    }
  }
}

}  // namespace hkv
