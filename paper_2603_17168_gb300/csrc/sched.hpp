// Triple-group concurrency control as a host-side scheduler over streams
// (Sec. 3.5, Table 4; Sec. 4.4).
//
// The paper enforces "readers with readers, updaters with updaters, every
// other pair exclusive" with host atomics mirrored to the device by a
// one-thread propagation kernel. Here the same compatibility matrix becomes
// stream-ordering: before an operation of group g is launched on stream s,
// s waits on the completion events of every in-flight operation of a group
// incompatible with g. No device-side spin is involved.
//
// State: the table is in an "epoch" of one group. While operations of that
// group keep arriving (readers or updaters) they join the epoch: each waits
// only for the frontier, the events of the previous epoch. An operation of a
// different group, or any inserter (never compatible, not even with itself),
// opens a new epoch whose frontier is every event of the current one.
// Because each member of an epoch waited for the whole previous frontier,
// waiting on the current epoch's events orders a newcomer after all earlier
// incompatible work, transitively.
//
// The table's mutex is held only while an operation takes its waits
// (acquire) and while it records its completion event (release), not while
// it launches its kernels in between: compatible operations from several
// host threads launch concurrently. An operation that opens a new epoch
// first waits, on the host, until every launch of the current epoch has
// recorded its event (otherwise it would wait on events not yet recorded),
// and while it waits, newcomers queue behind it, so a stream of compatible
// operations cannot starve it. Callers that take several tables' roles take
// them in one global (address) order and release after launching, so the
// waits cannot form a cycle.
//
// Backend supplies: Stream, Event, Event record(Stream), void wait(Stream,
// Event), bool same(Stream, Stream), void recycle(Event).
#pragma once

#include <condition_variable>
#include <mutex>
#include <utility>
#include <vector>

namespace hkv {

enum Group : int { kReader = 0, kUpdater = 1, kInserter = 2 };

// Table 4: readers with readers, updaters with updaters, all else exclusive.
// rw_lock: the conventional reader/writer lock the paper compares against
// (Exp 3e), where updaters are writers and exclude each other too.
inline bool compatible(Group a, Group b, bool rw_lock = false) {
  return a == b && a != kInserter && !(rw_lock && a == kUpdater);
}

template <class Backend>
class TripleGroup {
 public:
  using Stream = typename Backend::Stream;
  using Event = typename Backend::Event;

  explicit TripleGroup(Backend be = Backend()) : be_(std::move(be)) {}
  ~TripleGroup() { clear(); }

  // Order stream s after all in-flight work incompatible with group g. The
  // caller then launches its work on s and calls release(s).
  void acquire(Group g, Stream s) {
    std::unique_lock<std::mutex> lk(mu_);
    cv_.wait(lk, [&] { return !switching_; });
    if (!(have_epoch_ && compatible(group_, g, rw_lock_))) {
      switching_ = true;
      cv_.wait(lk, [&] { return launching_ == 0; });
      for (auto& fe : frontier_) be_.recycle(fe.second);
      frontier_ = std::move(current_);
      current_.clear();
      group_ = g;
      have_epoch_ = true;
      switching_ = false;
      cv_.notify_all();
    }
    for (auto& fe : frontier_)
      if (!be_.same(fe.first, s)) be_.wait(s, fe.second);
    ++launching_;
  }

  // Record the completion point of the operation just launched on s.
  void release(Stream s) {
    std::lock_guard<std::mutex> lk(mu_);
    Event e = be_.record(s);
    --launching_;
    if (launching_ == 0) cv_.notify_all();
    for (auto& ce : current_)
      if (be_.same(ce.first, s)) {
        be_.recycle(ce.second);
        ce.second = e;
        return;
      }
    current_.emplace_back(s, e);
  }

  // Drop every tracked event (the caller has synchronised the device).
  void clear() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& fe : frontier_) be_.recycle(fe.second);
    for (auto& ce : current_) be_.recycle(ce.second);
    frontier_.clear();
    current_.clear();
    have_epoch_ = false;
  }

  Backend& backend() { return be_; }

  // Switch between the triple-group rule and a reader/writer lock; takes
  // effect for operations acquired afterwards.
  void set_rw_lock(bool on) {
    std::lock_guard<std::mutex> lk(mu_);
    rw_lock_ = on;
  }

 private:
  Backend be_;
  std::mutex mu_;
  std::condition_variable cv_;
  int launching_ = 0;        // acquired operations not yet released
  bool switching_ = false;   // an operation waits to open a new epoch
  bool have_epoch_ = false;
  bool rw_lock_ = false;
  Group group_ = kReader;
  std::vector<std::pair<Stream, Event>> frontier_;
  std::vector<std::pair<Stream, Event>> current_;
};

}  // namespace hkv
