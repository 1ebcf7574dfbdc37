// Host-side table object and the internal launchers shared by the
// translation units of the library (no scheduling inside the launchers; the
// C-ABI entry points wrap them in the triple-group scheduler).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "hkv_common.cuh"
#include "sched.hpp"

namespace hkv {

// CUDA-event backend of the triple-group scheduler.
struct CudaEvents {
  using Stream = cudaStream_t;
  using Event = cudaEvent_t;
  std::vector<cudaEvent_t> pool;
  Event record(Stream s) {
    cudaEvent_t e;
    if (pool.empty()) {
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    } else {
      e = pool.back();
      pool.pop_back();
    }
    cudaEventRecord(e, s);
    return e;
  }
  void wait(Stream s, Event e) { cudaStreamWaitEvent(s, e, 0); }
  bool same(Stream a, Stream b) const { return a == b; }
  void recycle(Event e) { pool.push_back(e); }
  ~CudaEvents() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Per-table kernel timer (hkv_profile_*): event pairs on the launching stream.
struct Profiler {
  bool on = false;
  std::mutex mu;
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  cudaEvent_t get() {
    cudaEvent_t e;
    if (pool.empty()) {
      cudaEventCreate(&e);
    } else {
      e = pool.back();
      pool.pop_back();
    }
    return e;
  }
  ~Profiler() {
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Brackets one kernel launch with profiling events when profiling is on.
class KernelTimer {
 public:
  KernelTimer(Profiler& p, int kind, cudaStream_t s) : p_(p), kind_(kind), s_(s) {
    if (!p_.on) return;
    std::lock_guard<std::mutex> lk(p_.mu);
    a_ = p_.get();
    cudaEventRecord(a_, s_);
  }
  ~KernelTimer() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(p_.mu);
    cudaEvent_t b = p_.get();
    cudaEventRecord(b, s_);
    p_.recs.push_back({kind_, a_, b});
  }

 private:
  Profiler& p_;
  int kind_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr;
};

// Launch shape chosen for the probe kernels.
struct LaunchCfg {
  int find_tpk = 8;    // threads per key, find / contains
  int update_tpk = 8;  // threads per key, update phase of upsert / assign
  int vec_bytes = 16;  // widest value-row copy vector (16, 8 or 4)
};

}  // namespace hkv

struct hkv_table_s {
  hkv::TableDev dev{};
  hkv_options opts{};
  int device = 0;
  int num_sms = 0;
  uint64_t num_buckets = 0;
  uint64_t capacity = 0;
  uint64_t slots_per_slice = 0;
  uint64_t hbm_value_slots = 0;
  // Table step and epoch: atomic, since calls of a compatible group (assign
  // from several threads) run their host code concurrently.
  std::atomic<uint64_t> step{0};
  std::atomic<uint64_t> epoch{0};
  hkv::LaunchCfg launch;
  void* meta = nullptr;                 // digests + keys + scores + err + counters
  std::vector<void*> hbm_slices;
  std::vector<void*> host_slices;
  // The host slices, when they were carved from one mapping registered with
  // CUDA (huge-page advised) rather than allocated one by one.
  void* host_map = nullptr;
  uint64_t host_map_bytes = 0;
  void* host_base = nullptr;            // first host slice inside host_map
  uint64_t host_huge_bytes = 0;         // of it backed by huge pages at creation
  float** slices_dev = nullptr;
  cudaMemPool_t pool = nullptr;         // stream-ordered scratch allocations
  hkv::TripleGroup<hkv::CudaEvents> sched;
  hkv::Profiler prof;
  // L2 residency of the digest array: the access-policy window its probe
  // kernels launch with (num_bytes 0: none).
  cudaAccessPolicyWindow l2win{};
  unsigned long long* host_word = nullptr;  // pinned word for device-to-host counts
};

namespace hkv {

// Launch a kernel that probes or fills t's buckets with the table's L2
// window on its digest array as a per-launch attribute, so the caller's
// stream keeps its own attributes.
template <typename... KArgs, typename... Args>
inline void launch_table_kernel(const hkv_table_s* t, void (*kernel)(KArgs...), unsigned grid,
                                unsigned block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr{};
  if (t->l2win.num_bytes) {
    attr.id = cudaLaunchAttributeAccessPolicyWindow;
    attr.val.accessPolicyWindow = t->l2win;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Window covering the first `want` bytes of t's digest array (0: none),
// sized to the device's window limit and to the persisting L2 set-aside,
// which it raises as far as the device allows (a per-context limit).
void set_l2_window(hkv_table_s* t, uint64_t want);

}  // namespace hkv

namespace hkv {

// Widest vector (16, 8 or 4 bytes) a value-row copy between rows of `dim`
// floats at the given row arrays (null: not involved) may use under t's
// vec_bytes setting; table rows are 16-byte aligned.
int row_vector_bytes(const hkv_table_s* t, const void* a, const void* b = nullptr);

void set_last_error(const std::string& msg);
hkv_status cuda_status(cudaError_t e, const char* what);

// Raw launchers (asynchronous on `s`); each returns HKV_OK or an error after
// checking its launches.
hkv_status launch_find(hkv_table_s* t, uint64_t n, const uint64_t* keys, float* values_out,
                       uint8_t* found, uint64_t* scores_out, cudaStream_t s);
// find* (Sec. 5.2): value-row pointers instead of copies.
hkv_status launch_find_ptr(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float** ptrs,
                           uint8_t* found, cudaStream_t s);
hkv_status launch_gather(const float* const* ptrs, uint64_t n, uint32_t dim, float* out,
                         int num_sms, cudaStream_t s);
hkv_status launch_upsert(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                         const uint64_t* scores, uint8_t* status_out, uint64_t* ev_keys,
                         uint64_t* ev_scores, float* ev_values, uint64_t* n_evicted,
                         ScoreCtx ctx, cudaStream_t s, bool keep_hits = false,
                         const float* gather_src = nullptr);
// insert_or_assign whose rows sit in memory the kernels read slowly (mapped
// page-locked host memory, `rows_src`): after dedup, the rows of the
// batch's distinct keys (their last occurrences) are gathered into
// `rows_stage` (device, n x dim) by one streaming kernel, and the update and
// insert phases read them there. Results as hkv_insert_or_assign with
// values = rows_src; evictions are not reported.
hkv_status insert_or_assign_gathered(hkv_table_s* t, uint64_t n, const uint64_t* keys,
                                     const float* rows_src, float* rows_stage,
                                     const uint64_t* scores, uint8_t* status_out,
                                     cudaStream_t s);
// find_or_insert (Sec. 4.1): upsert that leaves residents' values alone,
// then a find into values_io; found_out from the statuses.
hkv_status launch_find_or_insert(hkv_table_s* t, uint64_t n, const uint64_t* keys,
                                 float* values_io, const uint64_t* scores, uint8_t* found_out,
                                 ScoreCtx ctx, cudaStream_t s);
// The upsert pipeline run in a caller-provided scratch block of
// scratch_bytes (device memory); no allocation. Evicted values not kept.
hkv_status launch_upsert_in(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                            const uint64_t* scores, uint8_t* status_out, uint64_t* ev_keys,
                            uint64_t* ev_scores, uint64_t* n_evicted, ScoreCtx ctx,
                            void* scratch, uint64_t scratch_bytes, cudaStream_t s);
// Host-memory value rows in address order (tiered tables, hkv_hostrows.cu).
// region_sort groups the items j < m (m = *m_dev when given, else m_max)
// with slot[j] != kNoHostSlot, all of them slots in host memory, by 2 MiB
// region; scratch is region_sort_bytes(t, m_max) bytes of device memory.
uint64_t region_sort_bytes(const hkv_table_s* t, uint64_t m_max);
hkv_status region_sort(const hkv_table_s* t, const uint64_t* slot, uint64_t m_max,
                       const unsigned long long* m_dev, void* scratch, RegionOrder* out,
                       cudaStream_t st);
// out[i] = the row of slot hslot[i] for every listed i (find with values).
hkv_status launch_host_rows_gather(const hkv_table_s* t, uint64_t n, const uint64_t* hslot,
                                   const RegionOrder& ro, float* out, bool vec16,
                                   cudaStream_t st);
// Batched rounds: size, buffers and score context come from a device
// OpDesc; grids are sized for n_max, scratch is the caller's block of
// upsert_scratch_bytes(n_max) bytes. No allocation, no profiling events.
uint64_t upsert_scratch_bytes(uint64_t n_max);
// True iff p points into device memory of the current device. Input rows
// anywhere else (page-locked host memory that kernels read in place) get
// plain loads only: no bulk L2 prefetch is issued on them.
bool in_device_memory(const void* p);
hkv_status launch_find_desc(hkv_table_s* t, uint64_t n_max, const OpDesc* d, bool values,
                            cudaStream_t s);
hkv_status launch_upsert_desc(hkv_table_s* t, uint64_t n_max, const OpDesc* d, void* scratch,
                              uint64_t scratch_bytes, cudaStream_t s);
hkv_status launch_assign(hkv_table_s* t, uint64_t n, const uint64_t* keys, const float* values,
                         const uint64_t* scores, ScoreCtx ctx, cudaStream_t s);
hkv_status launch_erase(hkv_table_s* t, uint64_t n, const uint64_t* keys, cudaStream_t s);
hkv_status launch_export(hkv_table_s* t, uint64_t offset, uint64_t n_slots, uint64_t* count_out,
                         uint64_t* keys, float* values, uint64_t* scores, uint64_t* slots,
                         cudaStream_t s, uint64_t score_min = 0, uint64_t score_max = ~0ull);
hkv_status launch_size(hkv_table_s* t, unsigned long long* out_dev, cudaStream_t s);

}  // namespace hkv
