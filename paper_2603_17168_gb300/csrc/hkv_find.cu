// find / contains: digest-probe kernels (Algorithm 1, Sec. 3.2; reader
// group of Sec. 3.5).
//
// A group of G lanes serves one key: every lane loads 128/G bytes of the
// bucket's digest line (16-byte vector loads for G <= 8, so one group issues
// exactly one 128-byte line), compares them four at a time with __vcmpeq4,
// confirms each digest match against the full key, and the group agrees on
// the hit through one warp ballot. The hit's value row is then copied by the
// same G lanes with 16-byte loads and streaming stores. Dual-bucket tables
// read the second line only when the first bucket missed.
//
// Tables with value slices in host memory (HOST): a hit whose row lives in
// host memory is not copied by the probe; its slot goes to a per-key list,
// which is grouped by host region and copied in that order afterwards
// (hkv_hostrows.cu), since scattered host rows are bound by the device's
// address translation.
#include <algorithm>

#include "hkv_internal.h"

namespace hkv {
namespace {

constexpr int kFindThreads = 256;

template <int G, bool VEC16, bool VALUES, bool HOST = false>
__global__ void __launch_bounds__(kFindThreads, 8)
    find_kernel(TableDev t, uint64_t n, const uint64_t* __restrict__ keys,
                float* __restrict__ out, uint8_t* __restrict__ found,
                uint64_t* __restrict__ scores_out, const OpDesc* __restrict__ d,
                const float** __restrict__ ptrs_out, uint64_t* __restrict__ hslot = nullptr,
                uint64_t host0 = 0) {
  if (d) {
    n = d->n;
    keys = d->keys;
    out = d->values_out;
    found = d->flags;
  }
  constexpr int KPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int lane_g = lane & (G - 1);
  const int group_base = lane & ~(G - 1);
  const unsigned group_bits = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << group_base);
  const uint64_t warp = (blockIdx.x * (uint64_t)kFindThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kFindThreads) >> 5;
  unsigned hits = 0, misses = 0, lines = 0, kreads = 0;

  for (uint64_t base = warp * KPW; base < n; base += nwarps * KPW) {
    const uint64_t i = base + (lane / G);
    bool in = i < n;
    uint64_t key = in ? __ldg(keys + i) : kEmptyKey;
    bool active = in && key < kFirstReserved;
    uint64_t h = fmix64(key);
    uint64_t b = h & t.bucket_mask;
    uint32_t pat4 = digest_from_hash(h) * 0x01010101u;
    int slot = probe_bucket<G, false, false>(t, b, key, pat4, active, lane_g, group_bits,
                                             group_base, kreads);
    lines += active && lane_g == 0;
    if (t.dual) {
      uint64_t b2 = second_bucket(t, key);
      bool need = active && slot < 0 && b2 != b;
      lines += need && lane_g == 0;
      if (__any_sync(0xFFFFFFFFu, need)) {
        int s2 = probe_bucket<G, false, false>(t, b2, key, pat4, need, lane_g, group_bits,
                                               group_base, kreads);
        if (need && s2 >= 0) {
          slot = s2;
          b = b2;
        }
      }
    }
    const bool hit = active && slot >= 0;
    const uint64_t g = b * kSlots + (uint64_t)slot;
    const bool later = HOST && hit && g >= host0;  // a host row: copied in region order
    if (hit) {
      if (VALUES && !later)
        copy_row<G, VEC16, true>(out + i * t.dim, value_ptr(t, g), t.dim, lane_g, t.vec8);
      if (scores_out && lane_g == 0) scores_out[i] = __ldg(score_ptr(t, g));
    }
    if (HOST && in && lane_g == 0) hslot[i] = later ? g : kNoHostSlot;
    if (in && lane_g == 0) {
      if (found) found[i] = hit ? 1 : 0;
      if (ptrs_out) ptrs_out[i] = hit ? value_ptr(t, b * kSlots + (uint64_t)slot) : nullptr;
      hits += hit;
      misses += !hit;
    }
  }
  const int which[4] = {HKV_CNT_FIND_HIT, HKV_CNT_FIND_MISS, HKV_CNT_FIND_LINES, HKV_CNT_FIND_KEYS};
  const unsigned vals[4] = {hits, misses, lines, kreads};
  flush_counts(t, which, vals);
}

template <int G>
void launch_g(const hkv_table_s* t, uint64_t n, const uint64_t* keys, float* out, uint8_t* found,
              uint64_t* scores_out, bool vec16, cudaStream_t s, const OpDesc* d = nullptr,
              bool values_if_desc = false, const float** ptrs = nullptr,
              uint64_t* hslot = nullptr) {
  const bool values = d ? values_if_desc : out != nullptr;
  uint64_t warps_needed = (n + (32 / G) - 1) / (32 / G);
  uint64_t blocks = (warps_needed * 32 + kFindThreads - 1) / kFindThreads;
  uint64_t cap = (uint64_t)t->num_sms * (2048 / kFindThreads);
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (hslot)  // values with host rows listed (vec16 only)
    launch_table_kernel(t, find_kernel<G, true, true, true>, (unsigned)blocks, kFindThreads, 0,
                        s, t->dev, n, keys, out, found, scores_out, d, ptrs, hslot,
                        t->hbm_value_slots);
  else if (!values)
    launch_table_kernel(t, find_kernel<G, false, false>, (unsigned)blocks, kFindThreads, 0, s,
                        t->dev, n, keys, out, found, scores_out, d, ptrs, nullptr,
                        (uint64_t)0);
  else if (vec16)
    launch_table_kernel(t, find_kernel<G, true, true>, (unsigned)blocks, kFindThreads, 0, s,
                        t->dev, n, keys, out, found, scores_out, d, ptrs, nullptr,
                        (uint64_t)0);
  else
    launch_table_kernel(t, find_kernel<G, false, true>, (unsigned)blocks, kFindThreads, 0, s,
                        t->dev, n, keys, out, found, scores_out, d, ptrs, nullptr,
                        (uint64_t)0);
}

}  // namespace

hkv_status launch_find(hkv_table_s* t, uint64_t n, const uint64_t* keys, float* values_out,
                       uint8_t* found, uint64_t* scores_out, cudaStream_t s) {
  if (n == 0) return HKV_OK;
  const bool vec16 = row_vector_bytes(t, values_out) == 16;
  // host rows of a tiered table: listed by the probe, copied in region order
  void* scratch = nullptr;
  uint64_t* hslot = nullptr;
  // (the region order holds 32-bit batch indices: larger finds copy in place)
  if (values_out && vec16 && !t->host_slices.empty() && n < (1ull << 32)) {
    const uint64_t hb = (n * 8 + 255) & ~255ull;
    if (cudaMallocFromPoolAsync(&scratch, hb + region_sort_bytes(t, n), t->pool, s) !=
        cudaSuccess) {
      cudaGetLastError();
      set_last_error("find scratch allocation failed");
      return HKV_ERR_OOM;
    }
    hslot = static_cast<uint64_t*>(scratch);
  }
  {
  KernelTimer timer(t->prof, HKV_K_FIND, s);
  switch (t->launch.find_tpk) {
    case 1: launch_g<1>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
    case 2: launch_g<2>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
    case 4: launch_g<4>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
    case 16: launch_g<16>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
    case 32: launch_g<32>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
    default: launch_g<8>(t, n, keys, values_out, found, scores_out, vec16, s, nullptr, false, nullptr, hslot); break;
  }
  }
  if (hslot) {
    KernelTimer timer(t->prof, HKV_K_HOSTROWS, s);
    RegionOrder ro;
    const uint64_t hb = (n * 8 + 255) & ~255ull;
    hkv_status rc = region_sort(t, hslot, n, nullptr, static_cast<char*>(scratch) + hb, &ro, s);
    if (rc == HKV_OK) rc = launch_host_rows_gather(t, n, hslot, ro, values_out, true, s);
    cudaFreeAsync(scratch, s);
    if (rc) return rc;
  }
  return cuda_status(cudaGetLastError(), "find launch");
}

hkv_status launch_find_ptr(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float** ptrs,
                           uint8_t* found, cudaStream_t s) {
  if (n == 0) return HKV_OK;
  KernelTimer timer(t->prof, HKV_K_FIND, s);
  switch (t->launch.find_tpk) {
    case 1: launch_g<1>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs); break;
    case 2: launch_g<2>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs); break;
    case 4: launch_g<4>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs); break;
    case 16:
      launch_g<16>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs);
      break;
    case 32:
      launch_g<32>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs);
      break;
    default: launch_g<8>(t, n, keys, nullptr, found, nullptr, false, s, nullptr, false, ptrs);
  }
  return cuda_status(cudaGetLastError(), "find* launch");
}

namespace {

// Gather rows through pointers: one warp per row, 16-byte vectors when the
// row and the output are 16-byte aligned. A null pointer leaves its row.
__global__ void gather_rows_kernel(const float* const* __restrict__ ptrs, uint64_t n, uint32_t dim,
                                   float* __restrict__ out, int vec16) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n; i += nwarps) {
    const float* src = ptrs[i];
    if (!src) continue;
    float* dst = out + i * dim;
    if (vec16) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
      float4* d4 = reinterpret_cast<float4*>(dst);
      for (uint32_t j = lane; j < dim / 4; j += 32) __stcs(d4 + j, __ldcg(s4 + j));
    } else {
      for (uint32_t j = lane; j < dim; j += 32) __stcs(dst + j, __ldcg(src + j));
    }
  }
}

}  // namespace

hkv_status launch_gather(const float* const* ptrs, uint64_t n, uint32_t dim, float* out,
                         int num_sms, cudaStream_t s) {
  if (n == 0) return HKV_OK;
  const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, (uint64_t)num_sms * 8);
  const int vec16 = dim % 4 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  gather_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(ptrs, n, dim, out, vec16);
  return cuda_status(cudaGetLastError(), "gather launch");
}

hkv_status launch_find_desc(hkv_table_s* t, uint64_t n_max, const OpDesc* d, bool values,
                            cudaStream_t s) {
  // Sized for n_max; the kernel reads the round's size and buffers from d,
  // whose value rows the batch object keeps 16-byte aligned.
  const uint64_t n = n_max ? n_max : 1;
  const bool vec16 = row_vector_bytes(t, nullptr) == 16;  // rows checked 16-byte aligned
  switch (t->launch.find_tpk) {
    case 1: launch_g<1>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
    case 2: launch_g<2>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
    case 4: launch_g<4>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
    case 16: launch_g<16>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
    case 32: launch_g<32>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
    default: launch_g<8>(t, n, nullptr, nullptr, nullptr, nullptr, vec16, s, d, values); break;
  }
  return cuda_status(cudaGetLastError(), "batched find launch");
}

}  // namespace hkv
