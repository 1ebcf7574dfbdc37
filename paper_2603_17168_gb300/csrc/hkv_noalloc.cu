// insert_or_assign for callers that cannot allocate device memory.
//
// hkv_insert_or_assign takes its per-call scratch (dedup table, miss
// records, victims: about 75 bytes per key) from a stream-ordered pool, which
// may allocate on a call. Some callers cannot allow that: a serving process
// whose device memory is all reserved up front by its framework's allocator,
// or a latency-critical path that must not meet an allocation's possible
// implicit synchronisation or an out-of-memory failure in the middle of a
// request. This variant runs the same kernels in one fixed scratch array
// that lives in the library's own device image, so a call allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits. Host code
// cannot pass the array's name to a kernel (on the host that name is only a
// stand-in symbol, not a device address), so every call looks its device
// address up with cudaGetSymbolAddress, with the table's device current.
// The address is not cached: a context torn down by cudaDeviceReset and
// created again maps the array elsewhere, and a cached address would then
// point at memory the new context does not own. The lookup costs far less
// than the launches it precedes. The first lookup on a device may load the
// library's device code there, which stream capture does not allow, so the
// first call on each device must come before any capture.
#include "hkv_internal.h"

namespace {

constexpr uint64_t kNoAllocScratchBytes = 5ull << 20;  // 5 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current context.
hkv_status scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return hkv::cuda_status(e, "no-alloc scratch address");
  *out = p;
  return HKV_OK;
}

}  // namespace

extern "C" hkv_status hkv_insert_or_assign_noalloc(hkv_table_t t, uint64_t n,
                                                   const uint64_t* keys, const float* values,
                                                   const uint64_t* scores, uint8_t* status_out,
                                                   uint64_t* evicted_keys,
                                                   uint64_t* evicted_scores, uint64_t* n_evicted,
                                                   hkv_stream_t stream) {
  if (!t || (n && (!keys || !values))) {
    hkv::set_last_error("upsert arguments");
    return HKV_ERR_INVALID_ARG;
  }
  if (n > HKV_NOALLOC_MAX_KEYS) {
    hkv::set_last_error("hkv_insert_or_assign_noalloc: batch of more than HKV_NOALLOC_MAX_KEYS "
                        "(65536) keys; split it or use hkv_insert_or_assign");
    return HKV_ERR_INVALID_ARG;
  }
  if (n && t->opts.policy == HKV_CUSTOM && !scores) {
    hkv::set_last_error("HKV_CUSTOM needs scores");
    return HKV_ERR_INVALID_ARG;
  }
  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return hkv::cuda_status(e, "current device");
  if (device != t->device) {
    hkv::set_last_error("make the table's device current before calling");
    return HKV_ERR_INVALID_ARG;
  }
  if (t->opts.dual_bucket && t->opts.deterministic) {
    hkv::set_last_error("hkv_insert_or_assign_noalloc: deterministic dual-bucket tables need "
                        "the ordered waves of hkv_insert_or_assign");
    return HKV_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  hkv_status rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(hkv::kInserter, s);
  hkv::ScoreCtx ctx{n ? t->step.load() + 1 : t->step.load(), t->epoch.load()};
  rc = hkv::launch_upsert_in(t, n, keys, values, (t->opts.policy == HKV_CUSTOM) ? scores : nullptr,
                             status_out, evicted_keys, evicted_scores, n_evicted, ctx, scratch,
                             kNoAllocScratchBytes, s);
  if (rc == HKV_OK && n) t->step++;
  t->sched.release(s);
  return rc;
}
