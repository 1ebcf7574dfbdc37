// Digest ablation (Sec. 5.4, Exp 3a): find without the digest line.
//
// The table's find reads a bucket's 128-byte digest line and confirms only
// the slots whose 8-bit digest matches (Algorithm 1). This entry point finds
// the same keys the way a table without digests must: a warp reads the
// bucket's whole 2 KiB run of (key, score) pairs, 16 bytes per slot, and
// compares every key. Results are identical to hkv_find; only the bytes
// moved differ (2 KiB per probed bucket instead of 128 B plus one key
// sector per digest match). It exists to measure what the digest line buys
// on this GPU and is not used by any other path.
#include "hkv_internal.h"

namespace hkv {
namespace {

constexpr int kAblThreads = 256;

// Slot of the warp's key in bucket b, or -1: every lane compares the keys of
// its slots 2l, 2l+1, 64+2l, 65+2l (coalesced 16-byte pair loads).
__device__ __forceinline__ int scan_bucket_keys(const TableDev& t, uint64_t b, uint64_t key,
                                                int lane) {
  const ulonglong2* pp = reinterpret_cast<const ulonglong2*>(key_ptr(t, b * kSlots));
  const ulonglong2 p0 = __ldg(pp + 2 * lane), p1 = __ldg(pp + 2 * lane + 1);
  const ulonglong2 p2 = __ldg(pp + 64 + 2 * lane), p3 = __ldg(pp + 65 + 2 * lane);
  int my = -1;
  if (p0.x == key) my = 2 * lane;
  if (p1.x == key) my = 2 * lane + 1;
  if (p2.x == key) my = 64 + 2 * lane;
  if (p3.x == key) my = 65 + 2 * lane;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, my >= 0);
  return bal ? __shfl_sync(0xFFFFFFFFu, my, __ffs(bal) - 1) : -1;
}

template <bool VEC16, bool VALUES>
__global__ void __launch_bounds__(kAblThreads)
    find_full_keys_kernel(TableDev t, uint64_t n, const uint64_t* __restrict__ keys,
                          float* __restrict__ out, uint8_t* __restrict__ found) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)kAblThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kAblThreads) >> 5;
  for (uint64_t i = warp; i < n; i += nwarps) {  // one key per warp
    const uint64_t key = __ldg(keys + i);
    const bool active = key < kFirstReserved;  // reserved keys are never resident
    uint64_t b = fmix64(key) & t.bucket_mask;
    int slot = active ? scan_bucket_keys(t, b, key, lane) : -1;
    if (active && slot < 0 && t.dual) {
      const uint64_t b2 = second_bucket(t, key);
      if (b2 != b) {
        slot = scan_bucket_keys(t, b2, key, lane);
        b = b2;
      }
    }
    const bool hit = slot >= 0;
    if (VALUES && hit)
      copy_row<32, VEC16, true>(out + i * t.dim, value_ptr(t, b * kSlots + (uint64_t)slot), t.dim,
                                lane, t.vec8);
    if (lane == 0 && found) found[i] = hit ? 1 : 0;
  }
}

}  // namespace
}  // namespace hkv

using namespace hkv;

extern "C" hkv_status hkv_find_full_keys(hkv_table_t t, uint64_t n, const uint64_t* keys,
                                         float* values_out, uint8_t* found, hkv_stream_t stream) {
  if (!t || (n && (!keys || (!values_out && !found)))) {
    set_last_error("find_full_keys arguments");
    return HKV_ERR_INVALID_ARG;
  }
  if (n == 0) return HKV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  t->sched.acquire(kReader, s);
  const bool vec16 = row_vector_bytes(t, values_out) == 16;
  uint64_t blocks = (n * 32 + kAblThreads - 1) / kAblThreads;
  const uint64_t cap = (uint64_t)t->num_sms * (2048 / kAblThreads);
  if (blocks > cap) blocks = cap;
  if (!values_out)
    find_full_keys_kernel<false, false><<<(unsigned)blocks, kAblThreads, 0, s>>>(
        t->dev, n, keys, values_out, found);
  else if (vec16)
    find_full_keys_kernel<true, true><<<(unsigned)blocks, kAblThreads, 0, s>>>(
        t->dev, n, keys, values_out, found);
  else
    find_full_keys_kernel<false, true><<<(unsigned)blocks, kAblThreads, 0, s>>>(
        t->dev, n, keys, values_out, found);
  const hkv_status rc = cuda_status(cudaGetLastError(), "find_full_keys launch");
  t->sched.release(s);
  return rc;
}
