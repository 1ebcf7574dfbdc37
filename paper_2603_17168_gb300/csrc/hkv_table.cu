// Table lifecycle, size / export kernels and the C-ABI entry points.
//
// Storage (Sec. 4.2, "Tiered Storage Engine"): the digest, key and score
// arrays always sit in HBM, in one allocation. Values are cut into slices of
// a power-of-two number of whole buckets; slices are taken from HBM while the
// value budget lasts, then from pinned host memory mapped into the device
// address space, so kernels reach both through the same position-based
// address and no CPU thread is on the data path. The host slices are one
// anonymous mapping advised for transparent huge pages and registered with
// CUDA (pinned, mapped): on GB300, scattered 512-byte row reads over 64 GiB
// of host memory ran 41 M rows/s from such a mapping against 19 M rows/s
// from cudaHostAlloc, and 365 M against 228 M rows/s when visited in
// address order (the device's address translation, not the link, limits
// scattered host access). cudaHostAlloc per slice is the fallback.
#include <sys/mman.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "hkv_internal.h"

namespace hkv {

namespace {
thread_local std::string g_last_error;

// Bytes of [p, p + len) backed by transparent huge pages, summed over the
// process's mappings that overlap it (/proc/self/smaps; 0 if unreadable).
uint64_t huge_page_bytes(const void* p, uint64_t len) {
  FILE* f = fopen("/proc/self/smaps", "r");
  if (!f) return 0;
  const uintptr_t lo = reinterpret_cast<uintptr_t>(p), hi = lo + len;
  char line[512];
  bool in = false;
  uint64_t total = 0;
  while (fgets(line, sizeof line, f)) {
    unsigned long a = 0, b = 0;
    char c = 0;
    if (sscanf(line, "%lx-%lx%c", &a, &b, &c) == 3 && c == ' ') {
      in = a < hi && lo < b;
    } else if (in && strncmp(line, "AnonHugePages:", 14) == 0) {
      unsigned long kb = 0;
      if (sscanf(line + 14, "%lu", &kb) == 1) total += (uint64_t)kb << 10;
    }
  }
  fclose(f);
  return total;
}

constexpr uint64_t kDefaultSlice = 1ull << 30;

__global__ void init_meta_kernel(uint8_t* digests, uint64_t* kv, uint64_t slots) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < slots;
       i += (uint64_t)gridDim.x * blockDim.x) {
    reinterpret_cast<ulonglong2*>(kv)[i] = make_ulonglong2(kEmptyKey, 0ull);
    if ((i & 15) == 0) reinterpret_cast<uint4*>(digests)[i >> 4] = make_uint4(0, 0, 0, 0);
  }
}

// Occupied slots = non-zero digest bytes, 16 per thread per step.
__global__ void size_kernel(const uint8_t* __restrict__ digests, uint64_t n16,
                            unsigned long long* out) {
  unsigned long long c = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(digests) + i);
    c += 16 - ((__popc(__vcmpeq4(v.x, 0)) + __popc(__vcmpeq4(v.y, 0)) + __popc(__vcmpeq4(v.z, 0)) +
                __popc(__vcmpeq4(v.w, 0))) >> 3);
  }
  c = __reduce_add_sync(0xFFFFFFFFu, (unsigned)c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// One warp per 32 consecutive slots: the ballot compacts the occupied ones,
// then the warp copies their value rows cooperatively.
__global__ void export_kernel(TableDev t, uint64_t offset, uint64_t n_slots,
                              unsigned long long* count, uint64_t* __restrict__ keys,
                              float* __restrict__ values, uint64_t* __restrict__ scores,
                              uint64_t* __restrict__ slots, uint64_t score_min,
                              uint64_t score_max) {
  const bool any_score = score_min == 0 && score_max == ~0ull;
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = warp * 32; base < n_slots; base += nwarps * 32) {
    const uint64_t g = offset + base + lane;
    const bool in = base + lane < n_slots;
    const uint64_t k = in ? *key_ptr(t, g) : kEmptyKey;
    bool occ = in && k < kLockedKey;
    uint64_t sc = 0;
    if (occ && (scores || !any_score)) sc = *score_ptr(t, g);
    if (!any_score) occ = occ && sc >= score_min && sc <= score_max;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, occ);
    if (!bal) continue;
    unsigned long long o0 = 0;
    if (lane == 0) o0 = atomicAdd(count, (unsigned long long)__popc(bal));
    o0 = __shfl_sync(0xFFFFFFFFu, o0, 0);
    if (occ) {
      const unsigned long long o = o0 + __popc(bal & ((1u << lane) - 1u));
      if (keys) keys[o] = k;
      if (scores) scores[o] = sc;
      if (slots) slots[o] = g;
    }
    if (values) {
      unsigned rest = bal;
      for (int r = 0; rest; ++r) {
        const int src_lane = __ffs(rest) - 1;
        rest &= rest - 1;
        const uint64_t gs = offset + base + src_lane;
        const float* v = value_ptr(t, gs);
        for (uint32_t d = lane; d < t.dim; d += 32) values[(o0 + r) * t.dim + d] = v[d];
      }
    }
  }
}

hkv_status fail(hkv_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

int row_vector_bytes(const hkv_table_s* t, const void* a, const void* b) {
  const uintptr_t m = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b);
  const uint32_t dim = t->dev.dim;
  if (t->launch.vec_bytes >= 16 && dim % 4 == 0 && (m & 15) == 0) return 16;
  if (t->launch.vec_bytes >= 8 && dim % 2 == 0 && (m & 7) == 0) return 8;
  return 4;
}

bool in_device_memory(const void* p) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

hkv_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HKV_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HKV_ERR_OOM : HKV_ERR_CUDA;
}

void set_l2_window(hkv_table_s* t, uint64_t want) {
  t->l2win = cudaAccessPolicyWindow{};
  const uint64_t digest_bytes = t->num_buckets * kSlots;
  if (want > digest_bytes) want = digest_bytes;
  if (want == 0) return;
  int max_win = 0, max_persist = 0;
  cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, t->device);
  cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, t->device);
  if (max_win <= 0 || max_persist <= 0) return;  // no persisting L2 on this device
  size_t cur = 0;
  cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
  if (cur < (size_t)max_persist &&
      cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)max_persist) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
  const uint64_t bytes = std::min<uint64_t>(want, (uint64_t)max_win);
  t->l2win.base_ptr = t->dev.digests;
  t->l2win.num_bytes = bytes;
  // more window than set-aside: mark only that share persisting, so the
  // persisting lines do not evict each other
  t->l2win.hitRatio = std::min(1.0f, (float)((double)cur / (double)bytes));
  t->l2win.hitProp = cudaAccessPropertyPersisting;
  t->l2win.missProp = cudaAccessPropertyStreaming;
}

hkv_status launch_size(hkv_table_s* t, unsigned long long* out_dev, cudaStream_t s) {
  cudaMemsetAsync(out_dev, 0, 8, s);
  const uint64_t n16 = t->num_buckets * kSlots / 16;
  uint64_t blocks = std::min<uint64_t>((n16 + 255) / 256, (uint64_t)t->num_sms * 8);
  KernelTimer timer(t->prof, HKV_K_SIZE, s);
  size_kernel<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(t->dev.digests, n16, out_dev);
  return cuda_status(cudaGetLastError(), "size launch");
}

hkv_status launch_export(hkv_table_s* t, uint64_t offset, uint64_t n_slots, uint64_t* count_out,
                         uint64_t* keys, float* values, uint64_t* scores, uint64_t* slots,
                         cudaStream_t s, uint64_t score_min, uint64_t score_max) {
  cudaMemsetAsync(count_out, 0, 8, s);
  if (n_slots == 0) return cuda_status(cudaGetLastError(), "export");
  uint64_t blocks = std::min<uint64_t>((n_slots + 255) / 256, (uint64_t)t->num_sms * 8);
  KernelTimer timer(t->prof, HKV_K_EXPORT, s);
  export_kernel<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(
      t->dev, offset, n_slots, reinterpret_cast<unsigned long long*>(count_out), keys, values,
      scores, slots, score_min, score_max);
  return cuda_status(cudaGetLastError(), "export launch");
}

}  // namespace hkv

using namespace hkv;

namespace {

void free_table(hkv_table_s* t) {
  for (void* p : t->hbm_slices) cudaFree(p);
  if (t->host_map) {
    cudaHostUnregister(t->host_base);
    munmap(t->host_map, t->host_map_bytes);
  } else {
    for (void* p : t->host_slices) cudaFreeHost(p);
  }
  if (t->slices_dev) cudaFree(t->slices_dev);
  if (t->meta) cudaFree(t->meta);
  if (t->pool) cudaMemPoolDestroy(t->pool);
  if (t->host_word) cudaFreeHost(t->host_word);
  delete t;
}

// Latched device error, read and cleared (stream-ordered).
hkv_status take_device_error(hkv_table_s* t, cudaStream_t s) {
  uint32_t e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, t->dev.err, 4, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_status(ce, "sync");
  if (e) {
    cudaMemsetAsync(t->dev.err, 0, 4, s);
    cudaStreamSynchronize(s);
    const char* what = e == HKV_ERR_RESERVED_KEY    ? "a batch held a reserved key (>= 2^63)"
                       : e == HKV_ERR_DUPLICATE_KEY ? "deterministic mode: a batch held a key twice"
                       : e == HKV_ERR_TIMEOUT       ? "a bounded slot-claim wait ran out"
                                                    : "device error";
    set_last_error(what);
    return (hkv_status)e;
  }
  return HKV_OK;
}

bool bad(hkv_table_t t) { return t == nullptr; }

}  // namespace

extern "C" {

const char* hkv_last_error(void) { return g_last_error.c_str(); }

hkv_status hkv_create(const hkv_options* o, hkv_table_t* out) {
  if (!o || !out) return fail(HKV_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (o->dim == 0 || o->capacity == 0 || o->policy < HKV_LRU || o->policy > HKV_CUSTOM_TS_FREQ)
    return fail(HKV_ERR_INVALID_ARG, "capacity, dim and policy must be valid");
  uint64_t nb = 1;
  while (nb * kSlots < o->capacity) nb <<= 1;
  if (nb > (1ull << 32)) return fail(HKV_ERR_INVALID_ARG, "capacity above 2^39 slots");

  hkv_table_s* t = new hkv_table_s();
  t->opts = *o;
  t->num_buckets = nb;
  t->capacity = nb * kSlots;
  cudaGetDevice(&t->device);
  cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
  const uint64_t slots = t->capacity;
  const uint64_t dim = o->dim;

  // metadata: digests | (key, score) pairs | sizes | err | counters
  const uint64_t off_kv = slots;                      // digests: slots bytes (multiple of 128)
  const uint64_t off_sizes = off_kv + slots * 16;
  const uint64_t off_err = off_sizes + ((nb * 4 + 255) & ~255ull);
  const uint64_t off_cnt = off_err + 256;
  const uint64_t meta_bytes = off_cnt + 256;
  cudaError_t e = cudaMalloc(&t->meta, meta_bytes);
  if (e != cudaSuccess) {
    free_table(t);
    return cuda_status(e, "metadata allocation");
  }
  char* m = static_cast<char*>(t->meta);
  t->dev.digests = reinterpret_cast<uint8_t*>(m);
  t->dev.kv = reinterpret_cast<uint64_t*>(m + off_kv);
  t->dev.sizes = reinterpret_cast<uint32_t*>(m + off_sizes);
  t->dev.err = reinterpret_cast<uint32_t*>(m + off_err);
  t->dev.counters = reinterpret_cast<unsigned long long*>(m + off_cnt);
  t->dev.bucket_mask = nb - 1;
  t->dev.dim = o->dim;
  t->dev.policy = o->policy;
  t->dev.dual = o->dual_bucket ? 1 : 0;
  t->dev.vec8 = 1;  // 8-byte copies where 16-byte ones are not possible

  // value slices: a power-of-two number of buckets each
  const uint64_t want_slice = o->slice_bytes ? o->slice_bytes : kDefaultSlice;
  uint64_t bps = 1;
  while (bps * 2 <= nb && bps * 2 * kSlots * dim * 4 <= want_slice) bps <<= 1;
  t->slots_per_slice = bps * kSlots;
  int shift = 0;
  while ((1ull << shift) < t->slots_per_slice) ++shift;
  t->dev.slice_shift = (uint32_t)shift;
  const uint64_t n_slices = nb / bps;
  const uint64_t slice_bytes = t->slots_per_slice * dim * 4;
  uint64_t budget = o->hbm_value_budget_bytes ? o->hbm_value_budget_bytes : ~0ull;
  const uint64_t n_hbm = std::min<uint64_t>(n_slices, budget / slice_bytes);
  // host slices: one huge-page-advised mapping registered with CUDA, else
  // cudaHostAlloc per slice
  char* host_dev = nullptr;
  if (n_hbm < n_slices) {
    const uint64_t host_bytes = (n_slices - n_hbm) * slice_bytes;
    const uint64_t align = 1ull << 30;  // whole huge pages of either granule
    void* m = mmap(nullptr, host_bytes + align, PROT_READ | PROT_WRITE,
                   MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE, -1, 0);
    if (m != MAP_FAILED) {
      char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(m) + align - 1) &
                                           ~(uintptr_t)(align - 1));
      madvise(base, host_bytes, MADV_HUGEPAGE);  // advice only: failure is harmless
      void* dp = nullptr;
      const bool reg = cudaHostRegister(base, host_bytes, cudaHostRegisterMapped |
                                                              cudaHostRegisterPortable) == cudaSuccess;
      if (reg && cudaHostGetDevicePointer(&dp, base, 0) == cudaSuccess) {
        t->host_map = m;
        t->host_map_bytes = host_bytes + align;
        t->host_base = base;
        t->host_huge_bytes = huge_page_bytes(base, host_bytes);
        host_dev = static_cast<char*>(dp);
      } else {
        if (reg) cudaHostUnregister(base);
        cudaGetLastError();
        munmap(m, host_bytes + align);
      }
    }
  }
  std::vector<float*> bases;
  for (uint64_t i = 0; i < n_slices; ++i) {
    void* p = nullptr;
    if (i < n_hbm) {
      e = cudaMalloc(&p, slice_bytes);
      if (e != cudaSuccess) break;
      t->hbm_slices.push_back(p);
      t->hbm_value_slots += t->slots_per_slice;
    } else if (t->host_map) {
      const uint64_t k = i - n_hbm;
      t->host_slices.push_back(static_cast<char*>(t->host_base) + k * slice_bytes);
      p = host_dev + k * slice_bytes;
    } else {
      e = cudaHostAlloc(&p, slice_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
      if (e != cudaSuccess) break;
      t->host_slices.push_back(p);
      void* dp = nullptr;
      e = cudaHostGetDevicePointer(&dp, p, 0);
      if (e != cudaSuccess) break;
      p = dp;
    }
    bases.push_back(static_cast<float*>(p));
  }
  if (e != cudaSuccess) {
    free_table(t);
    return cuda_status(e, "value slice allocation");
  }
  e = cudaMalloc(&t->slices_dev, n_slices * sizeof(float*));
  if (e == cudaSuccess)
    e = cudaMemcpy(t->slices_dev, bases.data(), n_slices * sizeof(float*), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_table(t);
    return cuda_status(e, "slice table");
  }
  t->dev.values0 = bases[0];
  t->dev.slices = t->slices_dev;
  for (size_t i = 0; i < t->hbm_slices.size(); ++i) cudaMemset(t->hbm_slices[i], 0, slice_bytes);

  // stream-ordered pool for per-call scratch; keep freed blocks cached
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = t->device;
  e = cudaMemPoolCreate(&t->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(t->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e != cudaSuccess) {
    free_table(t);
    return cuda_status(e, "scratch pool");
  }

  e = cudaHostAlloc(reinterpret_cast<void**>(&t->host_word), 64, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    t->host_word = nullptr;
    free_table(t);
    return cuda_status(e, "pinned word");
  }
  init_meta_kernel<<<std::max(1, t->num_sms * 8), 256>>>(t->dev.digests, t->dev.kv, slots);
  cudaMemset(t->dev.sizes, 0, nb * 4);
  cudaMemset(t->dev.err, 0, 256);
  cudaMemset(t->dev.counters, 0, 256);
  // Default launch shape (the autotuner refines it per table): few threads
  // per key keep the probe kernels from being issue-bound; wide values get
  // more lanes for the row copy.
  t->launch.find_tpk = t->opts.dim <= 32 ? 2 : (t->opts.dim <= 128 ? 4 : 8);
  t->launch.update_tpk = t->opts.dim <= 128 ? 2 : 4;
  // No L2 window by default: on the four-table workload a window over each
  // table's digest array made every probe kernel slower (hkv_set_l2_residency
  // turns it on per table).
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_table(t);
    return cuda_status(e, "table initialisation");
  }
  *out = t;
  return HKV_OK;
}

hkv_status hkv_set_concurrency(hkv_table_t t, int mode) {
  if (bad(t) || (mode != HKV_CC_TRIPLE_GROUP && mode != HKV_CC_RW_LOCK))
    return fail(HKV_ERR_INVALID_ARG, "concurrency mode");
  t->sched.set_rw_lock(mode == HKV_CC_RW_LOCK);
  return HKV_OK;
}

hkv_status hkv_set_l2_residency(hkv_table_t t, uint64_t digest_bytes) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(t->device);
  set_l2_window(t, digest_bytes);
  cudaSetDevice(dev);
  return HKV_OK;
}

uint64_t hkv_l2_residency(hkv_table_t t) { return bad(t) ? 0 : t->l2win.num_bytes; }

hkv_status hkv_destroy(hkv_table_t t) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  cudaDeviceSynchronize();
  t->sched.clear();
  free_table(t);
  return HKV_OK;
}

uint64_t hkv_capacity(hkv_table_t t) { return t ? t->capacity : 0; }
uint64_t hkv_num_buckets(hkv_table_t t) { return t ? t->num_buckets : 0; }
uint32_t hkv_dim(hkv_table_t t) { return t ? t->opts.dim : 0; }
uint64_t hkv_hbm_value_slots(hkv_table_t t) { return t ? t->hbm_value_slots : 0; }

hkv_status hkv_host_memory_info(hkv_table_t t, uint64_t* host_bytes, uint64_t* huge_bytes,
                                int* one_mapping) {
  if (bad(t) || !host_bytes || !huge_bytes || !one_mapping)
    return fail(HKV_ERR_INVALID_ARG, "host memory info arguments");
  *host_bytes = (t->capacity - t->hbm_value_slots) * (uint64_t)t->opts.dim * 4;
  *huge_bytes = t->host_huge_bytes;
  *one_mapping = t->host_map ? 1 : 0;
  return HKV_OK;
}

hkv_status hkv_find(hkv_table_t t, uint64_t n, const uint64_t* keys, float* values_out,
                    uint8_t* found, uint64_t* scores_out, hkv_stream_t stream) {
  if (bad(t) || (n && (!keys || !values_out))) return fail(HKV_ERR_INVALID_ARG, "find arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  hkv_status rc = launch_find(t, n, keys, values_out, found, scores_out, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_contains(hkv_table_t t, uint64_t n, const uint64_t* keys, uint8_t* found,
                        hkv_stream_t stream) {
  if (bad(t) || (n && (!keys || !found))) return fail(HKV_ERR_INVALID_ARG, "contains arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  hkv_status rc = launch_find(t, n, keys, nullptr, found, nullptr, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_insert_or_assign(hkv_table_t t, uint64_t n, const uint64_t* keys,
                                const float* values, const uint64_t* scores,
                                uint8_t* status_out, uint64_t* evicted_keys,
                                uint64_t* evicted_scores, float* evicted_values,
                                uint64_t* n_evicted, hkv_stream_t stream) {
  if (bad(t) || (n && (!keys || !values))) return fail(HKV_ERR_INVALID_ARG, "upsert arguments");
  if (n && t->opts.policy == HKV_CUSTOM && !scores)
    return fail(HKV_ERR_INVALID_ARG, "HKV_CUSTOM needs scores");
  if (n >= (1ull << 31)) return fail(HKV_ERR_INVALID_ARG, "batch above 2^31 keys");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kInserter, s);
  ScoreCtx ctx{n ? t->step.load() + 1 : t->step.load(), t->epoch.load()};
  hkv_status rc = launch_upsert(t, n, keys, values,
                                (t->opts.policy == HKV_CUSTOM) ? scores : nullptr, status_out,
                                evicted_keys, evicted_scores, evicted_values, n_evicted, ctx, s);
  if (rc == HKV_OK && n) t->step++;
  t->sched.release(s);
  return rc;
}

hkv_status hkv_find_or_insert(hkv_table_t t, uint64_t n, const uint64_t* keys, float* values_io,
                              const uint64_t* scores, uint8_t* found_out, hkv_stream_t stream) {
  if (bad(t) || (n && (!keys || !values_io)))
    return fail(HKV_ERR_INVALID_ARG, "find_or_insert arguments");
  if (n && t->opts.policy == HKV_CUSTOM && !scores)
    return fail(HKV_ERR_INVALID_ARG, "HKV_CUSTOM needs scores");
  if (n >= (1ull << 31)) return fail(HKV_ERR_INVALID_ARG, "batch above 2^31 keys");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kInserter, s);
  ScoreCtx ctx{n ? t->step.load() + 1 : t->step.load(), t->epoch.load()};
  hkv_status rc = launch_find_or_insert(t, n, keys, values_io,
                                        (t->opts.policy == HKV_CUSTOM) ? scores : nullptr,
                                        found_out, ctx, s);
  if (rc == HKV_OK && n) t->step++;
  t->sched.release(s);
  return rc;
}

hkv_status hkv_assign(hkv_table_t t, uint64_t n, const uint64_t* keys, const float* values,
                      const uint64_t* scores, hkv_stream_t stream) {
  if (bad(t) || (n && !keys)) return fail(HKV_ERR_INVALID_ARG, "assign arguments");
  if (n >= (1ull << 31)) return fail(HKV_ERR_INVALID_ARG, "batch above 2^31 keys");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kUpdater, s);
  // updaters run concurrently: each reserves its step (a failed launch
  // still advances it)
  ScoreCtx ctx{n ? t->step.fetch_add(1) + 1 : t->step.load(), t->epoch.load()};
  hkv_status rc = launch_assign(t, n, keys, values,
                                (t->opts.policy == HKV_CUSTOM) ? scores : nullptr, ctx, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_erase(hkv_table_t t, uint64_t n, const uint64_t* keys, hkv_stream_t stream) {
  if (bad(t) || (n && !keys)) return fail(HKV_ERR_INVALID_ARG, "erase arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kInserter, s);
  hkv_status rc = launch_erase(t, n, keys, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_copy_state(hkv_table_t dst, hkv_table_t src, hkv_stream_t stream) {
  if (bad(dst) || bad(src) || dst == src)
    return fail(HKV_ERR_INVALID_ARG, "copy_state: two distinct tables");
  const hkv_options &a = dst->opts, &b = src->opts;
  if (dst->capacity != src->capacity || a.dim != b.dim || a.policy != b.policy ||
      a.dual_bucket != b.dual_bucket || a.deterministic != b.deterministic ||
      dst->slots_per_slice != src->slots_per_slice ||
      dst->hbm_slices.size() != src->hbm_slices.size() ||
      dst->host_slices.size() != src->host_slices.size() || dst->device != src->device)
    return fail(HKV_ERR_INVALID_ARG, "copy_state: tables of different shapes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Take the two roles in address order, so that two threads copying in
  // opposite directions cannot wait on each other.
  hkv_table_s* first = dst < src ? dst : src;
  hkv_table_s* second = dst < src ? src : dst;
  first->sched.acquire(first == dst ? kInserter : kReader, s);
  second->sched.acquire(second == dst ? kInserter : kReader, s);
  // digests, (key, score) pairs and occupancy counters: the metadata up to
  // the error word, which sits at the same offset in both tables
  const uint64_t meta = reinterpret_cast<const char*>(src->dev.err) -
                        reinterpret_cast<const char*>(src->meta);
  cudaMemcpyAsync(dst->meta, src->meta, meta, cudaMemcpyDeviceToDevice, s);
  const uint64_t slice_bytes = src->slots_per_slice * (uint64_t)b.dim * 4;
  for (size_t i = 0; i < src->hbm_slices.size(); ++i)
    cudaMemcpyAsync(dst->hbm_slices[i], src->hbm_slices[i], slice_bytes,
                    cudaMemcpyDeviceToDevice, s);
  for (size_t i = 0; i < src->host_slices.size(); ++i)
    cudaMemcpyAsync(dst->host_slices[i], src->host_slices[i], slice_bytes, cudaMemcpyDefault, s);
  dst->step = src->step.load();
  dst->epoch = src->epoch.load();
  const hkv_status rc = cuda_status(cudaGetLastError(), "copy_state");
  second->sched.release(s);
  first->sched.release(s);
  return rc;
}

hkv_status hkv_size(hkv_table_t t, uint64_t* out, hkv_stream_t stream) {
  if (bad(t) || !out) return fail(HKV_ERR_INVALID_ARG, "size arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* d = t->dev.counters + 28;  // spare words after the counters
  {
    t->sched.acquire(kReader, s);
    hkv_status rc = launch_size(t, d, s);
    t->sched.release(s);
    if (rc) return rc;
  }
  unsigned long long h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "size");
  *out = h;
  return take_device_error(t, s);
}

hkv_status hkv_export_batch(hkv_table_t t, uint64_t slot_offset, uint64_t n_slots,
                            uint64_t* count_out, uint64_t* keys, float* values, uint64_t* scores,
                            uint64_t* slots, hkv_stream_t stream) {
  if (bad(t) || !count_out) return fail(HKV_ERR_INVALID_ARG, "export arguments");
  if (slot_offset > t->capacity || n_slots > t->capacity - slot_offset)
    return fail(HKV_ERR_INVALID_ARG, "slot range outside the table");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  hkv_status rc = launch_export(t, slot_offset, n_slots, count_out, keys, values, scores, slots, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_export_batch_if(hkv_table_t t, uint64_t slot_offset, uint64_t n_slots,
                               uint64_t score_min, uint64_t score_max, uint64_t* count_out,
                               uint64_t* keys, float* values, uint64_t* scores, uint64_t* slots,
                               hkv_stream_t stream) {
  if (bad(t) || !count_out) return fail(HKV_ERR_INVALID_ARG, "export arguments");
  if (slot_offset > t->capacity || n_slots > t->capacity - slot_offset)
    return fail(HKV_ERR_INVALID_ARG, "slot range outside the table");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  hkv_status rc = launch_export(t, slot_offset, n_slots, count_out, keys, values, scores, slots,
                                s, score_min, score_max);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_find_ptr(hkv_table_t t, uint64_t n, const uint64_t* keys, const float** ptrs_out,
                        uint8_t* found, hkv_stream_t stream) {
  if (bad(t) || (n && (!keys || !ptrs_out))) return fail(HKV_ERR_INVALID_ARG, "find* arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  hkv_status rc = launch_find_ptr(t, n, keys, ptrs_out, found, s);
  t->sched.release(s);
  return rc;
}

hkv_status hkv_gather_rows(const float* const* ptrs, uint64_t n, uint32_t dim, float* out,
                           hkv_stream_t stream) {
  if ((n && (!ptrs || !out)) || dim == 0) return fail(HKV_ERR_INVALID_ARG, "gather arguments");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return launch_gather(ptrs, n, dim, out, sms, static_cast<cudaStream_t>(stream));
}

hkv_status hkv_set_step(hkv_table_t t, uint64_t step) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  t->step = step;
  return HKV_OK;
}

uint64_t hkv_get_step(hkv_table_t t) { return t ? t->step.load() : 0; }

hkv_status hkv_set_epoch(hkv_table_t t, uint64_t epoch) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  t->epoch = epoch;
  return HKV_OK;
}

hkv_status hkv_sync(hkv_table_t t, hkv_stream_t stream) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  return take_device_error(t, static_cast<cudaStream_t>(stream));
}

hkv_status hkv_read_counters(hkv_table_t t, uint64_t* out, hkv_stream_t stream) {
  if (bad(t) || !out) return fail(HKV_ERR_INVALID_ARG, "counters arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, t->dev.counters, HKV_COUNTER_COUNT * 8,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e, "read counters");
}

hkv_status hkv_reset_counters(hkv_table_t t, hkv_stream_t stream) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  return cuda_status(cudaMemsetAsync(t->dev.counters, 0, HKV_COUNTER_COUNT * 8,
                                     static_cast<cudaStream_t>(stream)),
                     "reset counters");
}

hkv_status hkv_profile_enable(hkv_table_t t, int on) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  std::lock_guard<std::mutex> lk(t->prof.mu);
  t->prof.on = on != 0;
  return HKV_OK;
}

hkv_status hkv_profile_read(hkv_table_t t, double* ms_out, uint64_t* launches_out) {
  if (bad(t) || !ms_out || !launches_out) return fail(HKV_ERR_INVALID_ARG, "profile arguments");
  std::lock_guard<std::mutex> lk(t->prof.mu);
  for (int k = 0; k < HKV_KERNEL_KINDS; ++k) {
    ms_out[k] = 0;
    launches_out[k] = 0;
  }
  hkv_status rc = HKV_OK;
  for (auto& r : t->prof.recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess && rc == HKV_OK) rc = cuda_status(e, "profile events");
    ms_out[r.kind] += ms;
    launches_out[r.kind] += 1;
    t->prof.pool.push_back(r.a);
    t->prof.pool.push_back(r.b);
  }
  t->prof.recs.clear();
  return rc;
}

hkv_status hkv_set_value_vector(hkv_table_t t, int bytes) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  if (bytes != 0 && bytes != 4 && bytes != 8 && bytes != 16)
    return fail(HKV_ERR_INVALID_ARG, "value vector width must be 4, 8 or 16 bytes");
  t->launch.vec_bytes = bytes ? bytes : 16;
  t->dev.vec8 = t->launch.vec_bytes >= 8 ? 1 : 0;
  return HKV_OK;
}

hkv_status hkv_set_launch(hkv_table_t t, int find_tpk, int update_tpk) {
  if (bad(t)) return fail(HKV_ERR_INVALID_ARG, "null table");
  auto ok = [](int v) { return v == 0 || v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; };
  if (!ok(find_tpk) || !ok(update_tpk)) return fail(HKV_ERR_INVALID_ARG, "threads per key");
  if (find_tpk) t->launch.find_tpk = find_tpk;
  if (update_tpk) t->launch.update_tpk = update_tpk;
  return HKV_OK;
}

}  // extern "C"

namespace hkv {

hkv_status insert_or_assign_gathered(hkv_table_s* t, uint64_t n, const uint64_t* keys,
                                     const float* rows_src, float* rows_stage,
                                     const uint64_t* scores, uint8_t* status_out,
                                     cudaStream_t s) {
  if (!t || (n && (!keys || !rows_src || !rows_stage)))
    return fail(HKV_ERR_INVALID_ARG, "upsert arguments");
  if (n && t->opts.policy == HKV_CUSTOM && !scores)
    return fail(HKV_ERR_INVALID_ARG, "HKV_CUSTOM needs scores");
  if (n >= (1ull << 31)) return fail(HKV_ERR_INVALID_ARG, "batch above 2^31 keys");
  t->sched.acquire(kInserter, s);
  ScoreCtx ctx{n ? t->step.load() + 1 : t->step.load(), t->epoch.load()};
  hkv_status rc = launch_upsert(t, n, keys, rows_stage,
                                (t->opts.policy == HKV_CUSTOM) ? scores : nullptr, status_out,
                                nullptr, nullptr, nullptr, nullptr, ctx, s, false, rows_src);
  if (rc == HKV_OK && n) t->step++;
  t->sched.release(s);
  return rc;
}

}  // namespace hkv
