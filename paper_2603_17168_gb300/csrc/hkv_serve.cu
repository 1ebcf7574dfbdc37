// Serving loop with continuous batching over device-resident tables.
//
// Requests (find or insert_or_assign on one table, keys and values in
// pinned host memory) arrive over time. Each table owns a staging ring in
// HBM; a request is admitted when its keys fit in its table's ring, which
// bounds the device memory held by requests in flight. An admitted
// request's inputs are copied into the ring on a copy-in stream. Whenever
// fewer than max_inflight rounds are on the GPU, the loop forms a round:
// for every table with admitted work it takes the head of that table's
// FIFO, and merges it with the following requests when they are finds that
// sit contiguously in the ring (an upsert always runs alone, so every
// request sees exactly the table history it would see alone, in arrival
// order). A round with several busy tables runs as one batched multi-table
// launch (hkv_batch_run); a round with one busy table calls that table's
// find / insert_or_assign directly, with grids sized to the request rather
// than to the ring. The round's outputs are copied back to each request's
// host buffers on a copy-out stream, so the next round's kernels run while
// they travel, and each request gets its own completion event: the loop
// polls those, stamps completion times request by request and frees ring
// space in FIFO order. Copies in, kernels and copies out of neighbouring
// rounds overlap, and each round overlaps tables.
//
// The plain mode runs the same trace one request at a time in arrival
// order (hkv_find / hkv_insert_or_assign per request, results copied back
// on the same stream), the baseline the batched mode is compared with.
#include <chrono>
#include <deque>
#include <thread>
#include <vector>

#include "hkv_internal.h"

namespace {

struct Ring {
  uint64_t* keys = nullptr;
  float* values = nullptr;
  uint8_t* flags = nullptr;
  uint64_t cap = 0;
  struct Alloc {
    uint64_t off, n;
  };
  std::deque<Alloc> live;  // FIFO of allocations

  // Contiguous FIFO allocation of n keys; returns false if it does not fit.
  bool alloc(uint64_t n, uint64_t* off) {
    if (n > cap) return false;
    uint64_t o = 0;
    if (!live.empty()) {
      const uint64_t first = live.front().off;
      const uint64_t end = live.back().off + live.back().n;
      if (end > first) {  // one run [first, end): room after it, or wrap to 0
        if (end + n <= cap) o = end;
        else if (n <= first) o = 0;
        else return false;
      } else {            // wrapped: the free space is [end, first)
        if (end + n <= first) o = end;
        else return false;
      }
    }
    live.push_back({o, n});
    *off = o;
    return true;
  }
  void release() { live.pop_front(); }
};

uint64_t table_hbm_bytes(hkv_table_t t) {
  return t->capacity * 17 + 512 + t->hbm_value_slots * (uint64_t)t->opts.dim * 4;
}

}  // namespace

struct hkv_server_s {
  int n = 0;
  std::vector<hkv_table_t> tables;
  std::vector<Ring> rings;
  hkv_batch_t batch = nullptr;
  cudaStream_t copy_stream = nullptr;  // request inputs into the rings
  cudaStream_t out_stream = nullptr;   // batched mode: results back to the host
  int max_inflight = 2;
  uint64_t hbm_bytes = 0;
  int profile = 0;                     // time rounds on the device (hkv_serve_profile)
  hkv_serve_stats stats{};             // of the last run
};

namespace {

void free_server(hkv_server_s* s) {
  if (s->batch) hkv_batch_destroy(s->batch);
  for (auto& r : s->rings) {
    if (r.keys) cudaFree(r.keys);
    if (r.values) cudaFree(r.values);
    if (r.flags) cudaFree(r.flags);
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->out_stream) cudaStreamDestroy(s->out_stream);
  delete s;
}

hkv_status bad(const char* m) {
  hkv::set_last_error(m);
  return HKV_ERR_INVALID_ARG;
}

using Clock = std::chrono::steady_clock;

struct ReqState {
  uint64_t off = 0;
  int stage = 0;  // 0 waiting, 1 arrived, 2 admitted, 3 launched, 4 done
};

struct Round {
  cudaEvent_t ev;              // the round's last copy back has finished
  std::vector<uint64_t> reqs;
  cudaEvent_t tev[4] = {};     // timing: compute start, end; copy-out start, end
  int ntev = 0;
};

// A launched request awaiting its completion event (batched mode).
struct Pending {
  uint64_t req;
  cudaEvent_t ev;
};

double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

}  // namespace

extern "C" {

hkv_status hkv_serve_create(const hkv_table_t* tables, int n_tables, uint64_t ring_keys,
                            uint64_t hbm_budget_bytes, int max_inflight, hkv_server_t* out) {
  if (!out || !tables || n_tables <= 0 || ring_keys == 0 || ring_keys >= (1ull << 31) ||
      max_inflight <= 0)
    return bad("serve arguments");
  *out = nullptr;
  uint64_t need = 0;
  for (int i = 0; i < n_tables; ++i) {
    if (!tables[i]) return bad("null table");
    if (tables[i]->opts.policy == HKV_CUSTOM)
      return bad("served requests carry no scores: HKV_CUSTOM tables are not served");
    need += table_hbm_bytes(tables[i]);
    need += ring_keys * (9 + 4ull * tables[i]->opts.dim);
    need += hkv::upsert_scratch_bytes(ring_keys);
  }
  if (hbm_budget_bytes && need > hbm_budget_bytes) {
    hkv::set_last_error("tables plus request staging exceed the HBM budget");
    return HKV_ERR_OOM;
  }
  hkv_server_s* s = new hkv_server_s();
  s->n = n_tables;
  s->max_inflight = max_inflight;
  s->hbm_bytes = need;
  s->tables.assign(tables, tables + n_tables);
  s->rings.resize(n_tables);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_tables && e == cudaSuccess; ++i) {
    Ring& r = s->rings[i];
    r.cap = ring_keys;
    e = cudaMalloc(&r.keys, ring_keys * 8);
    if (e == cudaSuccess) e = cudaMalloc(&r.values, ring_keys * 4ull * tables[i]->opts.dim);
    if (e == cudaSuccess) e = cudaMalloc(&r.flags, ring_keys);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->out_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_server(s);
    return hkv::cuda_status(e, "server staging");
  }
  std::vector<uint64_t> mk(n_tables, ring_keys);
  hkv_status rc = hkv_batch_create(n_tables, tables, mk.data(), &s->batch);
  if (rc) {
    free_server(s);
    return rc;
  }
  *out = s;
  return HKV_OK;
}

uint64_t hkv_serve_hbm_bytes(hkv_server_t s) { return s ? s->hbm_bytes : 0; }

hkv_status hkv_serve_destroy(hkv_server_t s) {
  if (!s) return bad("null server");
  cudaDeviceSynchronize();
  free_server(s);
  return HKV_OK;
}

hkv_status hkv_serve_profile(hkv_server_t s, int on) {
  if (!s) return bad("null server");
  s->profile = on ? 1 : 0;
  return HKV_OK;
}

hkv_status hkv_serve_stats_get(hkv_server_t s, hkv_serve_stats* out) {
  if (!s || !out) return bad("serve stats arguments");
  *out = s->stats;
  return HKV_OK;
}

hkv_status hkv_serve_run(hkv_server_t s, const hkv_serve_request* reqs, uint64_t n_req,
                         int batched, int use_graph, hkv_serve_result* results,
                         hkv_stream_t stream) {
  if (!s || (n_req && (!reqs || !results))) return bad("serve run arguments");
  for (uint64_t i = 0; i < n_req; ++i) {
    const hkv_serve_request& q = reqs[i];
    if (q.table < 0 || q.table >= s->n) return bad("request table index");
    if (q.op != HKV_OP_FIND && q.op != HKV_OP_UPSERT) return bad("request operation");
    if (q.n == 0 || q.n > s->rings[q.table].cap) return bad("request size must be 1..ring_keys");
    if (!q.keys || (q.op == HKV_OP_UPSERT ? !q.values_in : !q.values_out))
      return bad("request buffers");
    if (i && q.arrival_s < reqs[i - 1].arrival_s) return bad("requests must be in arrival order");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // batched results leave on the copy-out stream; the plain path keeps
  // everything on the caller's stream
  cudaStream_t out = batched ? s->out_stream : st;
  hkv_serve_stats& S = s->stats;
  S = hkv_serve_stats{};
  std::vector<ReqState> rs(n_req);
  std::vector<std::deque<uint64_t>> arrived(s->n), admitted(s->n);
  std::deque<Round> inflight;
  std::deque<Pending> pending;  // batched: launched requests in copy-out order
  std::vector<cudaEvent_t> ev_pool, tev_pool;
  cudaEvent_t copy_ev;
  cudaEventCreateWithFlags(&copy_ev, cudaEventDisableTiming);
  auto get_ev = [&]() {
    cudaEvent_t e;
    if (ev_pool.empty()) {
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    } else {
      e = ev_pool.back();
      ev_pool.pop_back();
    }
    return e;
  };
  // device busy time: timing events around each round's compute and its
  // copies back, read and recycled when the round retires
  const bool prof = s->profile != 0;
  auto timing_ev = [&](Round& rd, cudaStream_t on) {
    if (!prof) return;
    cudaEvent_t e;
    if (tev_pool.empty()) {
      cudaEventCreate(&e);
    } else {
      e = tev_pool.back();
      tev_pool.pop_back();
    }
    cudaEventRecord(e, on);
    rd.tev[rd.ntev++] = e;
  };
  auto retire_timing = [&](Round& rd) {
    float c = 0.f, o = 0.f;
    if (rd.ntev == 4) {
      if (cudaEventElapsedTime(&c, rd.tev[0], rd.tev[1]) == cudaSuccess) S.gpu_compute_s += c * 1e-3;
      if (cudaEventElapsedTime(&o, rd.tev[2], rd.tev[3]) == cudaSuccess) S.gpu_copy_out_s += o * 1e-3;
    }
    for (int k = 0; k < rd.ntev; ++k) tev_pool.push_back(rd.tev[k]);
    rd.ntev = 0;
  };
  const auto t0 = Clock::now();
  auto now_s = [&]() { return seconds(t0, Clock::now()); };
  uint64_t next_arrival = 0, done = 0, round_id = 0;
  hkv_status rc = HKV_OK;
  std::vector<hkv_batch_op> ops(s->n);

  auto finish = [&](uint64_t r, double t_done) {
    results[r].done_s = t_done;
    rs[r].stage = 4;
    s->rings[reqs[r].table].release();
    ++done;
  };

  while (done < n_req && rc == HKV_OK) {
    bool progress = false;
    const auto ta = Clock::now();
    const double now = seconds(t0, ta);
    // 1. arrivals
    while (next_arrival < n_req && reqs[next_arrival].arrival_s <= now) {
      arrived[reqs[next_arrival].table].push_back(next_arrival);
      rs[next_arrival].stage = 1;
      ++next_arrival;
      progress = true;
    }
    // 2. admission into the staging rings (FIFO per table), inputs copied in
    bool copied = false;
    for (int t = 0; t < s->n; ++t) {
      while (!arrived[t].empty()) {
        const uint64_t r = arrived[t].front();
        const hkv_serve_request& q = reqs[r];
        Ring& ring = s->rings[t];
        uint64_t off;
        if (!ring.alloc(q.n, &off)) break;
        rs[r].off = off;
        rs[r].stage = 2;
        results[r].admit_s = now;
        const uint64_t dim = s->tables[t]->opts.dim;
        cudaMemcpyAsync(ring.keys + off, q.keys, q.n * 8, cudaMemcpyHostToDevice, s->copy_stream);
        S.h2d_bytes += q.n * 8;
        if (q.op == HKV_OP_UPSERT) {
          cudaMemcpyAsync(ring.values + off * dim, q.values_in, q.n * dim * 4,
                          cudaMemcpyHostToDevice, s->copy_stream);
          S.h2d_bytes += q.n * dim * 4;
        }
        arrived[t].pop_front();
        admitted[t].push_back(r);
        copied = progress = true;
      }
    }
    if (copied) cudaEventRecord(copy_ev, s->copy_stream);
    const auto tb = Clock::now();
    S.host_admit_s += seconds(ta, tb);
    // 3. launch work while the pipeline has room
    while ((int)inflight.size() < s->max_inflight) {
      Round rd;
      if (batched) {
        int busy_tables = 0, only = -1;
        for (int t = 0; t < s->n; ++t) {
          ops[t] = hkv_batch_op{};
          if (admitted[t].empty()) continue;
          const uint64_t first = admitted[t].front();
          const int op = reqs[first].op;
          uint64_t n = 0, end = rs[first].off;
          while (!admitted[t].empty()) {
            const uint64_t r = admitted[t].front();
            if (reqs[r].op != op || rs[r].off != end) break;
            n += reqs[r].n;
            end += reqs[r].n;
            rd.reqs.push_back(r);
            admitted[t].pop_front();
            if (op == HKV_OP_UPSERT) break;
          }
          const Ring& ring = s->rings[t];
          const uint64_t off = rs[first].off, dim = s->tables[t]->opts.dim;
          ops[t].op = op;
          ops[t].n = n;
          ops[t].keys = ring.keys + off;
          if (op == HKV_OP_FIND) ops[t].values_out = ring.values + off * dim;
          else ops[t].values_in = ring.values + off * dim;
          ops[t].flags = ring.flags + off;
          ++busy_tables;
          only = t;
        }
        if (!busy_tables) break;
        cudaStreamWaitEvent(st, copy_ev, 0);
        timing_ev(rd, st);
        if (busy_tables == 1) {
          // one table: its own call, grids sized to the request
          const hkv_batch_op& o = ops[only];
          hkv_table_t tb1 = s->tables[only];
          rc = o.op == HKV_OP_FIND
                   ? hkv_find(tb1, o.n, o.keys, o.values_out, o.flags, nullptr, st)
                   : hkv_insert_or_assign(tb1, o.n, o.keys, o.values_in, nullptr, o.flags,
                                          nullptr, nullptr, nullptr, nullptr, st);
          S.direct_rounds++;
        } else {
          rc = hkv_batch_run(s->batch, ops.data(), use_graph, st);
          S.batched_rounds++;
        }
        timing_ev(rd, st);
        if (rc) {
          retire_timing(rd);  // back to the pool (the run ends with rc)
          break;
        }
        cudaEvent_t computed = get_ev();
        cudaEventRecord(computed, st);
        cudaStreamWaitEvent(out, computed, 0);
        ev_pool.push_back(computed);  // reusable once the wait is enqueued
        timing_ev(rd, out);
      } else {
        // plain: the oldest admitted request alone
        int tb = -1;
        for (int t = 0; t < s->n; ++t)
          if (!admitted[t].empty() && (tb < 0 || admitted[t].front() < admitted[tb].front())) tb = t;
        if (tb < 0) break;
        const uint64_t r = admitted[tb].front();
        admitted[tb].pop_front();
        rd.reqs.push_back(r);
        const Ring& ring = s->rings[tb];
        const uint64_t off = rs[r].off, dim = s->tables[tb]->opts.dim;
        cudaStreamWaitEvent(st, copy_ev, 0);
        timing_ev(rd, st);
        if (reqs[r].op == HKV_OP_FIND)
          rc = hkv_find(s->tables[tb], reqs[r].n, ring.keys + off, ring.values + off * dim,
                        ring.flags + off, nullptr, st);
        else
          rc = hkv_insert_or_assign(s->tables[tb], reqs[r].n, ring.keys + off,
                                    ring.values + off * dim, nullptr, ring.flags + off, nullptr,
                                    nullptr, nullptr, nullptr, st);
        timing_ev(rd, st);
        timing_ev(rd, st);  // copies back follow on the same stream
        S.direct_rounds++;
        if (rc) {
          retire_timing(rd);
          break;
        }
      }
      // results back to each request's host buffers, each request with its
      // own completion event in batched mode
      for (uint64_t r : rd.reqs) {
        const hkv_serve_request& q = reqs[r];
        const Ring& ring = s->rings[q.table];
        const uint64_t dim = s->tables[q.table]->opts.dim;
        if (q.op == HKV_OP_FIND) {
          cudaMemcpyAsync(q.values_out, ring.values + rs[r].off * dim, q.n * dim * 4,
                          cudaMemcpyDeviceToHost, out);
          S.d2h_bytes += q.n * dim * 4;
        }
        if (q.flags) {
          cudaMemcpyAsync(q.flags, ring.flags + rs[r].off, q.n, cudaMemcpyDeviceToHost, out);
          S.d2h_bytes += q.n;
        }
        rs[r].stage = 3;
        results[r].round = round_id;
        if (batched && rd.reqs.size() > 1) {
          cudaEvent_t ev = get_ev();
          cudaEventRecord(ev, out);
          pending.push_back({r, ev});
        }
      }
      timing_ev(rd, out);
      ++round_id;
      rd.ev = get_ev();
      cudaEventRecord(rd.ev, out);
      inflight.push_back(std::move(rd));
      progress = true;
    }
    const auto tc = Clock::now();
    S.host_launch_s += seconds(tb, tc);
    // 4. retire: batched requests one by one as their copies finish, and
    // rounds (which bound the work in flight) in order
    while (batched && !pending.empty()) {
      cudaError_t q = cudaEventQuery(pending.front().ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        rc = hkv::cuda_status(q, "request completion");
        break;
      }
      finish(pending.front().req, now_s());
      ev_pool.push_back(pending.front().ev);
      pending.pop_front();
      progress = true;
    }
    while (!inflight.empty() && rc == HKV_OK) {
      cudaError_t q = cudaEventQuery(inflight.front().ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        rc = hkv::cuda_status(q, "round completion");
        break;
      }
      // a round of one request completes with the round's own event
      if (inflight.front().reqs.size() == 1) finish(inflight.front().reqs[0], now_s());
      retire_timing(inflight.front());
      ev_pool.push_back(inflight.front().ev);
      inflight.pop_front();
      progress = true;
    }
    const auto td = Clock::now();
    S.host_retire_s += seconds(tc, td);
    S.loop_iterations++;
    if (!progress) {
      std::this_thread::yield();
      S.idle_s += seconds(td, Clock::now());
    }
  }
  cudaStreamSynchronize(st);
  cudaStreamSynchronize(out);
  S.wall_s = now_s();
  S.requests = done;
  for (auto& p : pending) ev_pool.push_back(p.ev);
  for (auto& r : inflight) {
    retire_timing(r);
    ev_pool.push_back(r.ev);
  }
  for (auto e : ev_pool) cudaEventDestroy(e);
  for (auto e : tev_pool) cudaEventDestroy(e);
  cudaEventDestroy(copy_ev);
  for (auto& ring : s->rings) ring.live.clear();
  return rc;
}

}  // extern "C"
