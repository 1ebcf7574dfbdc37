// Value rows in host memory, moved in address order (tiered tables,
// Sec. 4.2 "Tiered Storage Engine").
//
// A kernel reading or writing 512-byte rows scattered over tens of GiB of
// mapped host memory is limited by the device's address translation, not by
// the link: on GB300, random rows over 64 GiB ran 19-41 M rows/s, the same
// rows visited in address order 228-365 M rows/s (the link's 210 GB/s is
// about 410 M rows/s). So the paths that touch many host rows (find with
// values, and the rows an upsert writes) first list the host slots they
// need, group the list by 2 MiB region of host memory with a counting sort
// (histogram, one-block scan, scatter), and then move the rows region by
// region. The order inside a region is whatever the scatter's atomics gave:
// only the region matters for translation.
#include "hkv_internal.h"

namespace hkv {
namespace {

constexpr int kRegionLog2Bytes = 21;  // 2 MiB of values per region
constexpr int kSortThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kRowLanes = 8;          // lanes per row in the ordered copies

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

__device__ __forceinline__ uint64_t items(uint64_t m_max, const unsigned long long* m_dev) {
  return m_dev ? (uint64_t)*m_dev : m_max;
}

__global__ void __launch_bounds__(kSortThreads)
    region_hist_kernel(const uint64_t* __restrict__ slot, uint64_t m_max,
                       const unsigned long long* m_dev, uint64_t host0, int rshift,
                       uint32_t* __restrict__ hist) {
  const uint64_t m = items(m_max, m_dev);
  for (uint64_t j = blockIdx.x * (uint64_t)kSortThreads + threadIdx.x; j < m;
       j += (uint64_t)gridDim.x * kSortThreads) {
    const uint64_t g = slot[j];
    if (g != kNoHostSlot) atomicAdd(hist + ((g - host0) >> rshift), 1u);
  }
}

// Exclusive prefix sum of hist[0..nreg) in place by one block; *total gets
// the sum.
__global__ void __launch_bounds__(kScanThreads)
    region_scan_kernel(uint32_t* __restrict__ hist, uint64_t nreg,
                       unsigned long long* __restrict__ total) {
  __shared__ uint32_t part[kScanThreads];
  const uint64_t per = (nreg + kScanThreads - 1) / kScanThreads;
  const uint64_t lo = threadIdx.x * per;
  const uint64_t hi = lo + per < nreg ? lo + per : nreg;
  uint32_t sum = 0;
  for (uint64_t r = lo; r < hi; ++r) sum += hist[r];
  part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const uint32_t y = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (uint64_t r = lo; r < hi; ++r) {
    const uint32_t c = hist[r];
    hist[r] = run;
    run += c;
  }
  if (threadIdx.x == kScanThreads - 1) *total = part[kScanThreads - 1];
}

__global__ void __launch_bounds__(kSortThreads)
    region_scatter_kernel(const uint64_t* __restrict__ slot, uint64_t m_max,
                          const unsigned long long* m_dev, uint64_t host0, int rshift,
                          uint32_t* __restrict__ next, uint32_t* __restrict__ order) {
  const uint64_t m = items(m_max, m_dev);
  for (uint64_t j = blockIdx.x * (uint64_t)kSortThreads + threadIdx.x; j < m;
       j += (uint64_t)gridDim.x * kSortThreads) {
    const uint64_t g = slot[j];
    if (g != kNoHostSlot) order[atomicAdd(next + ((g - host0) >> rshift), 1u)] = (uint32_t)j;
  }
}

// find's host rows: out[i] = the row of slot hslot[i], for the listed i.
template <bool VEC16>
__global__ void __launch_bounds__(kSortThreads)
    host_rows_gather_kernel(TableDev t, const uint64_t* __restrict__ hslot, RegionOrder ro,
                            float* __restrict__ out) {
  const uint64_t m = *ro.count;
  const int lane_g = threadIdx.x & (kRowLanes - 1);
  const uint64_t grp = (blockIdx.x * (uint64_t)kSortThreads + threadIdx.x) / kRowLanes;
  const uint64_t ngrp = (uint64_t)gridDim.x * kSortThreads / kRowLanes;
  for (uint64_t p = grp; p < m; p += ngrp) {
    const uint64_t i = ro.order[p];
    copy_row<kRowLanes, VEC16, true>(out + i * t.dim, value_ptr(t, hslot[i]), t.dim, lane_g,
                                     t.vec8);
  }
}

unsigned grid_of(const hkv_table_s* t, uint64_t threads, int block, int per_sm) {
  uint64_t b = (threads + block - 1) / block;
  const uint64_t cap = (uint64_t)t->num_sms * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b ? b : 1);
}

}  // namespace

int region_shift(const hkv_table_s* t) {
  const uint64_t row = (uint64_t)t->dev.dim * 4;
  int s = 0;
  while ((row << (s + 1)) <= (1ull << kRegionLog2Bytes)) ++s;
  return s;
}

uint64_t region_count(const hkv_table_s* t) {
  const uint64_t host_slots = t->capacity - t->hbm_value_slots;
  const int s = region_shift(t);
  return (host_slots + (1ull << s) - 1) >> s;
}

uint64_t region_sort_bytes(const hkv_table_s* t, uint64_t m_max) {
  return align256(region_count(t) * 4) + align256(m_max * 4) + 256;
}

hkv_status region_sort(const hkv_table_s* t, const uint64_t* slot, uint64_t m_max,
                       const unsigned long long* m_dev, void* scratch, RegionOrder* out,
                       cudaStream_t st) {
  const uint64_t nreg = region_count(t);
  const int rshift = region_shift(t);
  const uint64_t host0 = t->hbm_value_slots;
  char* p = static_cast<char*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(p);
  p += align256(nreg * 4);
  out->order = reinterpret_cast<uint32_t*>(p);
  p += align256(m_max * 4);
  out->count = reinterpret_cast<unsigned long long*>(p);
  cudaMemsetAsync(hist, 0, nreg * 4, st);
  const unsigned grid = grid_of(t, m_max, kSortThreads, 8);
  region_hist_kernel<<<grid, kSortThreads, 0, st>>>(slot, m_max, m_dev, host0, rshift, hist);
  region_scan_kernel<<<1, kScanThreads, 0, st>>>(hist, nreg, out->count);
  region_scatter_kernel<<<grid, kSortThreads, 0, st>>>(slot, m_max, m_dev, host0, rshift, hist,
                                                       out->order);
  return cuda_status(cudaGetLastError(), "host row ordering");
}

hkv_status launch_host_rows_gather(const hkv_table_s* t, uint64_t n, const uint64_t* hslot,
                                   const RegionOrder& ro, float* out, bool vec16,
                                   cudaStream_t st) {
  const unsigned grid = grid_of(t, n * kRowLanes, kSortThreads, 8);
  if (vec16)
    host_rows_gather_kernel<true><<<grid, kSortThreads, 0, st>>>(t->dev, hslot, ro, out);
  else
    host_rows_gather_kernel<false><<<grid, kSortThreads, 0, st>>>(t->dev, hslot, ro, out);
  return cuda_status(cudaGetLastError(), "host row gather");
}

}  // namespace hkv
