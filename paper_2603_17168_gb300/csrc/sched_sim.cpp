// Host-only harness of the triple-group scheduler (sched.hpp) with a
// simulated stream/event backend, so the ordering rules of Sec. 3.5
// (Table 4) can be tested without a GPU. Streams are FIFO queues on a
// virtual clock; an event completes when the work queued before it does.
#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "sched.hpp"

namespace {

struct SimEvents {
  using Stream = int;
  using Event = int;
  std::vector<double> ev_time;
  std::vector<double> ready;  // per stream: time its queued work completes
  Event record(Stream s) {
    ev_time.push_back(ready[s]);
    return (int)ev_time.size() - 1;
  }
  void wait(Stream s, Event e) { ready[s] = std::max(ready[s], ev_time[e]); }
  bool same(Stream a, Stream b) const { return a == b; }
  void recycle(Event) {}
};

}  // namespace

extern "C" {

int hkv_sched_sim_mode(int n_ops, const int* group, const int* stream, const double* issue,
                       const double* dur, int n_streams, int rw_lock, double* start,
                       double* end);

// Run ops in issue order: op i of group[i] (0 reader, 1 updater, 2 inserter)
// on stream[i], issued by the host at issue[i], lasting dur[i]. Writes each
// op's start and end on the virtual clock. Returns 0, or -1 on bad input.
int hkv_sched_sim(int n_ops, const int* group, const int* stream, const double* issue,
                  const double* dur, int n_streams, double* start, double* end) {
  return hkv_sched_sim_mode(n_ops, group, stream, issue, dur, n_streams, 0, start, end);
}

// As hkv_sched_sim, with rw_lock = 1 for the reader/writer-lock rule.
int hkv_sched_sim_mode(int n_ops, const int* group, const int* stream, const double* issue,
                       const double* dur, int n_streams, int rw_lock, double* start,
                       double* end) {
  if (n_ops < 0 || n_streams <= 0) return -1;
  SimEvents be;
  be.ready.assign(n_streams, 0.0);
  hkv::TripleGroup<SimEvents> tg(be);
  tg.set_rw_lock(rw_lock != 0);
  for (int i = 0; i < n_ops; ++i) {
    if (group[i] < 0 || group[i] > 2 || stream[i] < 0 || stream[i] >= n_streams) return -1;
    tg.acquire(static_cast<hkv::Group>(group[i]), stream[i]);
    auto& b = tg.backend();
    double s = std::max(b.ready[stream[i]], issue[i]);
    start[i] = s;
    end[i] = s + dur[i];
    b.ready[stream[i]] = end[i];
    tg.release(stream[i]);
  }
  return 0;
}

// Several host threads at once, thread k issuing ops_per_thread ops on its
// own stream k: op j of thread k has group groups[k * ops_per_thread + j]
// and lasts dur[...] on the virtual clock; between acquire and release the
// thread sleeps launch_us microseconds of real time (its "launch"), so the
// threads' launch windows overlap. Writes each op's start and end. The
// backend's per-stream clock is touched only by its own thread, and its
// event list only under the scheduler's mutex. Returns 0, or -1 on bad input.
int hkv_sched_sim_threads(int n_threads, int ops_per_thread, const int* groups,
                          const double* dur, int rw_lock, int launch_us, double* start,
                          double* end) {
  if (n_threads <= 0 || ops_per_thread < 0) return -1;
  for (int i = 0; i < n_threads * ops_per_thread; ++i)
    if (groups[i] < 0 || groups[i] > 2) return -1;
  SimEvents be;
  be.ready.assign(n_threads, 0.0);
  be.ev_time.reserve((size_t)n_threads * ops_per_thread + 1);
  hkv::TripleGroup<SimEvents> tg(be);
  tg.set_rw_lock(rw_lock != 0);
  std::vector<std::thread> th;
  for (int k = 0; k < n_threads; ++k)
    th.emplace_back([&, k]() {
      for (int j = 0; j < ops_per_thread; ++j) {
        const int i = k * ops_per_thread + j;
        tg.acquire(static_cast<hkv::Group>(groups[i]), k);
        auto& b = tg.backend();
        start[i] = b.ready[k];
        end[i] = start[i] + dur[i];
        if (launch_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(launch_us));
        b.ready[k] = end[i];
        tg.release(k);
      }
    });
  for (auto& t : th) t.join();
  return 0;
}

}  // extern "C"
