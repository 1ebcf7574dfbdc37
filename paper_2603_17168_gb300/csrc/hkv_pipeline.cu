// Host-buffer pipeline: the end-to-end path from host memory through the
// table and back, with copies overlapped with kernels.
//
// Each operation takes the next of `depth` staging slots in HBM and is
// queued as three stream-ordered pieces:
//
//   copy-in   stream: wait until the slot's previous results left the
//             device, copy the inputs (keys, scores; rows if staged) into
//             the slot;
//   compute   stream: wait for the copy-in, run hkv_find /
//             hkv_insert_or_assign on the slot's buffers;
//   copy-out  stream: wait for the compute, copy the results (rows and
//             found flags, or statuses) to the caller's host buffers and
//             mark the slot free.
//
// An upsert's rows are not copied whole: when the caller's buffer is memory
// the device can address (page-locked host memory), one streaming kernel on
// the compute stream gathers, right after dedup, only the rows the table
// can store (the last occurrence of each distinct key) into the slot, and
// the update and insert phases read them there. Duplicates' rows never
// cross the link. Other host memory is staged whole by the copy engine.
// A find's rows go back whole by the copy engine (kernels storing into host
// memory beside the probe kernels took their block slots and lost).
//
// The compute stream runs operations in call order (they may share a
// table), while the copy streams work on the neighbouring operations: with
// three slots, operation k's inputs arrive while operation k-1 computes and
// operation k-2's results leave. The two directions of the link are used at
// once.
#include <vector>

#include "hkv_internal.h"

namespace {

struct PipeSlot {
  uint64_t* keys = nullptr;   // [max_keys]
  float* rows = nullptr;      // [max_keys][max_dim]: upsert input or find output
  uint64_t* scores = nullptr; // [max_keys]
  uint8_t* flags = nullptr;   // [max_keys]: found or status
  cudaEvent_t in_done = nullptr, compute_done = nullptr, free = nullptr;
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Device address of a host range [p, p + bytes) if every byte of it can be
// read and written by kernels of the current device (page-locked host
// memory mapped into its address space, or device or managed memory), else
// null: then the range is reached by staging copies only.
void* device_view(const void* p, uint64_t bytes) {
  if (!p || bytes == 0) return nullptr;
  const char* first = static_cast<const char*>(p);
  const char* last = first + bytes - 1;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, first) != cudaSuccess ||
      cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  auto usable = [](const cudaPointerAttributes& x) {
    return (x.type == cudaMemoryTypeHost || x.type == cudaMemoryTypeDevice ||
            x.type == cudaMemoryTypeManaged) &&
           x.devicePointer != nullptr;
  };
  if (!usable(a) || !usable(b)) return nullptr;
  // one contiguous mapping from the first byte to the last
  if (static_cast<char*>(b.devicePointer) != static_cast<char*>(a.devicePointer) + (bytes - 1))
    return nullptr;
  return a.devicePointer;
}

}  // namespace

struct hkv_pipeline_s {
  int device = 0;
  uint64_t max_keys = 0;
  uint32_t max_dim = 0;
  void* block = nullptr;
  std::vector<PipeSlot> slots;
  uint64_t next = 0;
  cudaStream_t in = nullptr, compute = nullptr, out = nullptr;
};

namespace {

void free_pipeline(hkv_pipeline_s* p) {
  if (p->in) cudaStreamSynchronize(p->in);
  if (p->compute) cudaStreamSynchronize(p->compute);
  if (p->out) cudaStreamSynchronize(p->out);
  for (auto& s : p->slots) {
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.compute_done) cudaEventDestroy(s.compute_done);
    if (s.free) cudaEventDestroy(s.free);
  }
  if (p->block) cudaFree(p->block);
  if (p->in) cudaStreamDestroy(p->in);
  if (p->compute) cudaStreamDestroy(p->compute);
  if (p->out) cudaStreamDestroy(p->out);
  delete p;
}

hkv_status bad_arg(const char* msg) {
  hkv::set_last_error(msg);
  return HKV_ERR_INVALID_ARG;
}

// Take the next slot: its input copy waits until its previous results
// have been copied out.
PipeSlot& take_slot(hkv_pipeline_s* p) {
  PipeSlot& s = p->slots[p->next % p->slots.size()];
  ++p->next;
  cudaStreamWaitEvent(p->in, s.free, 0);
  return s;
}

}  // namespace

extern "C" {

hkv_status hkv_pipeline_create(uint64_t max_keys, uint32_t max_dim, int depth,
                               hkv_pipeline_t* out) {
  if (!out || max_keys == 0 || max_keys >= (1ull << 31) || max_dim == 0 || depth < 2 ||
      depth > 8)
    return bad_arg("pipeline arguments");
  auto* p = new hkv_pipeline_s();
  cudaGetDevice(&p->device);
  p->max_keys = max_keys;
  p->max_dim = max_dim;
  const uint64_t sz_keys = align256(max_keys * 8);
  const uint64_t sz_rows = align256(max_keys * max_dim * 4ull);
  const uint64_t sz_flags = align256(max_keys);
  const uint64_t per_slot = 2 * sz_keys + sz_rows + sz_flags;
  cudaError_t e = cudaMalloc(&p->block, per_slot * (uint64_t)depth);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking);
  p->slots.resize(depth);
  char* base = static_cast<char*>(p->block);
  for (int i = 0; i < depth && e == cudaSuccess; ++i) {
    PipeSlot& s = p->slots[i];
    char* c = base + per_slot * i;
    s.keys = reinterpret_cast<uint64_t*>(c);
    s.scores = reinterpret_cast<uint64_t*>(c + sz_keys);
    s.rows = reinterpret_cast<float*>(c + 2 * sz_keys);
    s.flags = reinterpret_cast<uint8_t*>(c + 2 * sz_keys + sz_rows);
    e = cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.compute_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.free, cudaEventDisableTiming);
    // a fresh slot is free: record once so the first wait has an event
    if (e == cudaSuccess) e = cudaEventRecord(s.free, p->out);
  }
  if (e != cudaSuccess) {
    free_pipeline(p);
    return hkv::cuda_status(e, "pipeline creation");
  }
  *out = p;
  return HKV_OK;
}

hkv_status hkv_pipeline_find(hkv_pipeline_t p, hkv_table_t t, uint64_t n, const uint64_t* keys,
                             float* values, uint8_t* found) {
  if (!p || !t) return bad_arg("null pipeline or table");
  if (n > p->max_keys || t->opts.dim > p->max_dim)
    return bad_arg("find larger than the pipeline");
  if (t->device != p->device) return bad_arg("table on another device");
  if (n && (!keys || !values)) return bad_arg("pipeline find buffers");
  if (n == 0) return HKV_OK;
  const uint64_t row_bytes = n * t->opts.dim * 4ull;
  PipeSlot& s = take_slot(p);
  cudaMemcpyAsync(s.keys, keys, n * 8, cudaMemcpyHostToDevice, p->in);
  cudaEventRecord(s.in_done, p->in);
  cudaStreamWaitEvent(p->compute, s.in_done, 0);
  // Rows of misses come back as zeros: cleared on the device (on the compute
  // stream, which has slack, not on the copy-in stream, which is the link's
  // critical path), not sent.
  cudaMemsetAsync(s.rows, 0, row_bytes, p->compute);
  hkv_status rc = hkv_find(t, n, s.keys, s.rows, s.flags, nullptr, p->compute);
  cudaEventRecord(s.compute_done, p->compute);
  cudaStreamWaitEvent(p->out, s.compute_done, 0);
  cudaMemcpyAsync(values, s.rows, row_bytes, cudaMemcpyDeviceToHost, p->out);
  if (found) cudaMemcpyAsync(found, s.flags, n, cudaMemcpyDeviceToHost, p->out);
  cudaEventRecord(s.free, p->out);
  if (rc != HKV_OK) return rc;
  return hkv::cuda_status(cudaGetLastError(), "pipeline find");
}

hkv_status hkv_pipeline_insert_or_assign(hkv_pipeline_t p, hkv_table_t t, uint64_t n,
                                         const uint64_t* keys, const float* values,
                                         const uint64_t* scores, uint8_t* status) {
  if (!p || !t) return bad_arg("null pipeline or table");
  if (n > p->max_keys || t->opts.dim > p->max_dim)
    return bad_arg("upsert larger than the pipeline");
  if (t->device != p->device) return bad_arg("table on another device");
  if (n && (!keys || !values)) return bad_arg("pipeline upsert buffers");
  if (n && t->opts.policy == HKV_CUSTOM && !scores) return bad_arg("HKV_CUSTOM needs scores");
  if (n == 0) return HKV_OK;
  const uint64_t row_bytes = n * t->opts.dim * 4ull;
  // Rows the device can address are gathered after dedup (only the distinct
  // keys' last occurrences); other rows are staged whole.
  const float* rows_dev = static_cast<const float*>(device_view(values, row_bytes));
  PipeSlot& s = take_slot(p);
  cudaMemcpyAsync(s.keys, keys, n * 8, cudaMemcpyHostToDevice, p->in);
  if (!rows_dev) cudaMemcpyAsync(s.rows, values, row_bytes, cudaMemcpyHostToDevice, p->in);
  const bool custom = t->opts.policy == HKV_CUSTOM;
  if (custom) cudaMemcpyAsync(s.scores, scores, n * 8, cudaMemcpyHostToDevice, p->in);
  cudaEventRecord(s.in_done, p->in);
  cudaStreamWaitEvent(p->compute, s.in_done, 0);
  hkv_status rc =
      rows_dev ? hkv::insert_or_assign_gathered(t, n, s.keys, rows_dev, s.rows,
                                                custom ? s.scores : nullptr,
                                                status ? s.flags : nullptr, p->compute)
               : hkv_insert_or_assign(t, n, s.keys, s.rows, custom ? s.scores : nullptr,
                                      status ? s.flags : nullptr, nullptr, nullptr, nullptr,
                                      nullptr, p->compute);
  cudaEventRecord(s.compute_done, p->compute);
  cudaStreamWaitEvent(p->out, s.compute_done, 0);
  if (status) cudaMemcpyAsync(status, s.flags, n, cudaMemcpyDeviceToHost, p->out);
  cudaEventRecord(s.free, p->out);
  if (rc != HKV_OK) return rc;
  return hkv::cuda_status(cudaGetLastError(), "pipeline upsert");
}

hkv_status hkv_pipeline_sync(hkv_pipeline_t p) {
  if (!p) return bad_arg("null pipeline");
  cudaError_t e = cudaStreamSynchronize(p->in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->compute);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->out);
  return hkv::cuda_status(e, "pipeline sync");
}

hkv_status hkv_pipeline_destroy(hkv_pipeline_t p) {
  if (!p) return bad_arg("null pipeline");
  free_pipeline(p);
  return HKV_OK;
}

}  // extern "C"
