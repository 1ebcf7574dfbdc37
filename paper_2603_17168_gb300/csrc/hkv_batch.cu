// Batched multi-table rounds: one launch of a captured CUDA graph per round.
//
// A batch object binds a set of tables (one slot each) with the largest
// round each slot accepts. For every round it writes one small descriptor
// per slot (size, buffers, score context) to device memory with a single
// host-to-device copy, then replays a CUDA graph captured once per
// combination of operations: the graph forks one branch per busy slot onto
// its own stream, so tables of different sizes and value widths run side by
// side, and joins them back into the caller's stream. The kernels read the
// round's sizes from the descriptors, so one captured graph serves every
// round of that combination. Each table keeps its triple-group role for the
// round (find: reader, insert_or_assign: inserter; Sec. 3.5), taken on the
// caller's stream around the graph launch.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "hkv_internal.h"

using hkv::OpDesc;

struct hkv_batch_s {
  int device = 0;
  int n = 0;
  std::vector<hkv_table_t> tables;
  std::vector<uint64_t> max_keys;
  std::vector<void*> scratch;
  std::vector<uint64_t> scratch_bytes;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // captures rounds (the caller's stream may be the legacy one)
  OpDesc* desc_dev = nullptr;
  static constexpr int kRing = 4;
  OpDesc* desc_host[kRing] = {};
  cudaEvent_t ring_ev[kRing] = {};
  int ring = 0;
  std::map<std::vector<int>, cudaGraphExec_t> graphs;
  // per slot: the last upsert row pointer and whether it is device memory
  // (input rows get a bulk L2 prefetch only there); asked again only when
  // the pointer changes, since a pointer query costs more host time than a
  // round's other bookkeeping
  std::vector<const float*> rows_seen;
  std::vector<int> rows_on_device;
  std::mutex mu;
};

namespace {

void free_batch(hkv_batch_s* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  for (void* p : b->scratch) cudaFree(p);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->desc_dev) cudaFree(b->desc_dev);
  for (int r = 0; r < hkv_batch_s::kRing; ++r) {
    if (b->desc_host[r]) cudaFreeHost(b->desc_host[r]);
    if (b->ring_ev[r]) cudaEventDestroy(b->ring_ev[r]);
  }
  delete b;
}

hkv_status bad_arg(const char* msg) {
  hkv::set_last_error(msg);
  return HKV_ERR_INVALID_ARG;
}

// Fork one branch per busy slot from `s`, launch its operation, join back.
hkv_status enqueue_round(hkv_batch_s* b, const hkv_batch_op* ops, cudaStream_t s) {
  cudaEventRecord(b->fork, s);
  for (int i = 0; i < b->n; ++i) {
    if (ops[i].op == HKV_OP_NONE) continue;
    cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    hkv_table_t t = b->tables[i];
    hkv_status rc = ops[i].op == HKV_OP_FIND
                        ? hkv::launch_find_desc(t, b->max_keys[i], b->desc_dev + i, true,
                                                b->streams[i])
                        : hkv::launch_upsert_desc(t, b->max_keys[i], b->desc_dev + i,
                                                  b->scratch[i], b->scratch_bytes[i],
                                                  b->streams[i]);
    if (rc) return rc;
    cudaEventRecord(b->done[i], b->streams[i]);
    cudaStreamWaitEvent(s, b->done[i], 0);
  }
  return hkv::cuda_status(cudaGetLastError(), "batched round");
}

}  // namespace

extern "C" {

hkv_status hkv_batch_create(int n_slots, const hkv_table_t* tables, const uint64_t* max_keys,
                            hkv_batch_t* out) {
  if (!out || !tables || !max_keys || n_slots <= 0) return bad_arg("batch arguments");
  *out = nullptr;
  for (int i = 0; i < n_slots; ++i) {
    if (!tables[i] || max_keys[i] == 0 || max_keys[i] >= (1ull << 31))
      return bad_arg("each slot needs a table and 0 < max_keys < 2^31");
    for (int j = 0; j < i; ++j)
      if (tables[j] == tables[i]) return bad_arg("a table may appear in one slot only");
    // their ordered phase I is driven from the host, which a graph cannot do
    if (tables[i]->opts.deterministic && tables[i]->dev.dual)
      return bad_arg("deterministic dual-bucket tables take hkv_insert_or_assign only");
  }
  hkv_batch_s* b = new hkv_batch_s();
  cudaGetDevice(&b->device);
  b->n = n_slots;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_slots && e == cudaSuccess; ++i) {
    b->tables.push_back(tables[i]);
    b->max_keys.push_back(max_keys[i]);
    b->rows_seen.push_back(nullptr);
    b->rows_on_device.push_back(0);
    const uint64_t bytes = hkv::upsert_scratch_bytes(max_keys[i]);
    void* p = nullptr;
    e = cudaMalloc(&p, bytes);
    b->scratch.push_back(p);
    b->scratch_bytes.push_back(bytes);
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    b->streams.push_back(st);
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    b->done.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->desc_dev, n_slots * sizeof(OpDesc));
  for (int r = 0; r < hkv_batch_s::kRing && e == cudaSuccess; ++r) {
    e = cudaHostAlloc(&b->desc_host[r], n_slots * sizeof(OpDesc), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ring_ev[r], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return hkv::cuda_status(e, "batch creation");
  }
  *out = b;
  return HKV_OK;
}

hkv_status hkv_batch_destroy(hkv_batch_t b) {
  if (!b) return bad_arg("null batch");
  cudaDeviceSynchronize();
  free_batch(b);
  return HKV_OK;
}

hkv_status hkv_batch_run(hkv_batch_t b, const hkv_batch_op* ops, int use_graph,
                         hkv_stream_t stream) {
  if (!b || !ops) return bad_arg("batch run arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> guard(b->mu);
  // validate the round
  for (int i = 0; i < b->n; ++i) {
    const hkv_batch_op& o = ops[i];
    hkv_table_t t = b->tables[i];
    if (o.op < HKV_OP_NONE || o.op > HKV_OP_UPSERT) return bad_arg("unknown batch operation");
    if (o.op == HKV_OP_NONE) continue;
    if (o.n > b->max_keys[i]) return bad_arg("round larger than the slot's max_keys");
    if (o.n && !o.keys) return bad_arg("batch keys missing");
    const float* rows = o.op == HKV_OP_FIND ? o.values_out : o.values_in;
    if (o.n && !rows) return bad_arg("batch value rows missing");
    if (reinterpret_cast<uintptr_t>(rows) & 15) return bad_arg("batch value rows must be 16-byte aligned");
    if (o.op == HKV_OP_UPSERT && t->opts.policy == HKV_CUSTOM && o.n && !o.scores)
      return bad_arg("HKV_CUSTOM needs scores");
  }
  // descriptors for this round, through a ring of pinned buffers
  const int r = b->ring;
  b->ring = (r + 1) % hkv_batch_s::kRing;
  cudaEventSynchronize(b->ring_ev[r]);
  OpDesc* hd = b->desc_host[r];
  for (int i = 0; i < b->n; ++i) {
    const hkv_batch_op& o = ops[i];
    hkv_table_t t = b->tables[i];
    OpDesc d{};
    d.n = o.op == HKV_OP_NONE ? 0 : o.n;
    d.keys = o.keys;
    d.values_in = o.values_in;
    d.values_out = o.values_out;
    d.flags = o.flags;
    d.scores = t->opts.policy == HKV_CUSTOM ? o.scores : nullptr;
    if (o.op == HKV_OP_UPSERT && o.values_in && o.values_in != b->rows_seen[i]) {
      b->rows_seen[i] = o.values_in;
      b->rows_on_device[i] = hkv::in_device_memory(o.values_in) ? 1 : 0;
    }
    d.row_prefetch = o.op == HKV_OP_UPSERT && o.values_in ? b->rows_on_device[i] : 0;
    d.step = t->step;
    d.epoch = t->epoch;
    if (o.op == HKV_OP_UPSERT && o.n) d.step = ++t->step;
    hd[i] = d;
  }
  // take every table's role on the caller's stream (tables taken in address
  // order, so concurrent rounds over overlapping tables cannot deadlock)
  std::vector<int> order;
  for (int i = 0; i < b->n; ++i)
    if (ops[i].op != HKV_OP_NONE) order.push_back(i);
  std::sort(order.begin(), order.end(),
            [&](int x, int y) { return b->tables[x] < b->tables[y]; });
  for (int i : order)
    b->tables[i]->sched.acquire(ops[i].op == HKV_OP_FIND ? hkv::kReader : hkv::kInserter, s);
  cudaMemcpyAsync(b->desc_dev, hd, b->n * sizeof(OpDesc), cudaMemcpyHostToDevice, s);
  cudaEventRecord(b->ring_ev[r], s);

  hkv_status rc = HKV_OK;
  if (!use_graph) {
    rc = enqueue_round(b, ops, s);
  } else {
    std::vector<int> key;
    for (int i = 0; i < b->n; ++i) {
      key.push_back(ops[i].op);
      key.push_back(b->tables[i]->launch.find_tpk);
      key.push_back(b->tables[i]->launch.update_tpk);
    }
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      // capture once; the per-table profiling hook stays off while capturing
      std::vector<bool> prof;
      for (auto t : b->tables) {
        prof.push_back(t->prof.on);
        t->prof.on = false;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        rc = enqueue_round(b, ops, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
      }
      for (int i = 0; i < b->n; ++i) b->tables[i]->prof.on = prof[i];
      cudaGraphExec_t ge = nullptr;
      if (e == cudaSuccess && rc == HKV_OK) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess && rc == HKV_OK) rc = hkv::cuda_status(e, "round capture");
      if (rc == HKV_OK) it = b->graphs.emplace(key, ge).first;
    }
    if (rc == HKV_OK) rc = hkv::cuda_status(cudaGraphLaunch(it->second, s), "round launch");
  }
  for (size_t k = 0; k < order.size(); ++k) b->tables[order[k]]->sched.release(s);
  return rc;
}

}  // extern "C"
