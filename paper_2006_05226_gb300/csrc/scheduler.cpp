// Request scheduler of the serving loop (see scheduler.h).
//
// Admission rule, checked by an idle worker under the lock: the oldest waiting request
// starts when a slot is free and the bytes of the running requests plus its footprint fit
// in the budget. Requests start in submission order: a request never overtakes an older
// one, so a large request waits for memory instead of being starved by small ones.
#include "scheduler.h"

#include <algorithm>
#include <chrono>

namespace mlcc {
namespace serve {

static double steady_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Scheduler::Scheduler(int n_slots, int64_t budget_bytes, RunFn run, DropFn drop, int max_attempts)
    : budget_(budget_bytes), max_attempts_(std::max(1, max_attempts)), run_(std::move(run)),
      drop_(std::move(drop)), t0_(steady_seconds()) {
  const int n = std::max(1, n_slots);
  workers_.reserve(n);
  for (int k = 0; k < n; ++k) workers_.emplace_back([this, k] { worker(k); });
}

Scheduler::~Scheduler() {
  {
    std::lock_guard<std::mutex> lk(mu_);
    stop_ = true;
    for (uint64_t t : queue_) {
      Rec& r = recs_[t];
      r.waiting = false;
      r.done = true;
      r.out.status = kCancelled;
      r.out.t_finish = now();
      ++st_.cancelled;
    }
    queue_.clear();
    st_.waiting = 0;
  }
  work_cv_.notify_all();
  done_cv_.notify_all();
  for (auto& w : workers_) w.join();
  if (drop_)
    for (auto& kv : recs_) drop_(kv.second.payload);
}

double Scheduler::now() const { return steady_seconds() - t0_; }

bool Scheduler::admissible_locked(const Rec& r) const {
  if (r.hold_until >= 0 && completions_ <= r.hold_until) return false;
  return st_.in_use_bytes + r.footprint <= budget_;
}

int32_t Scheduler::submit(int64_t footprint, void* payload, uint64_t* ticket) {
  if (!ticket) return kArg;
  *ticket = 0;
  if (footprint <= 0) return kArg;
  if (footprint > budget_) return kRejected;
  {
    std::lock_guard<std::mutex> lk(mu_);
    if (stop_) return kState;
    const uint64_t t = next_ticket_++;
    Rec& r = recs_[t];
    r.payload = payload;
    r.footprint = footprint;
    r.waiting = true;
    r.out.footprint = footprint;
    r.out.t_submit = now();
    queue_.push_back(t);
    ++st_.submitted;
    st_.waiting = int32_t(queue_.size());
    *ticket = t;
  }
  work_cv_.notify_all();
  return kOk;
}

void Scheduler::worker(int slot) {
  std::unique_lock<std::mutex> lk(mu_);
  for (;;) {
    work_cv_.wait(lk, [&] {
      return stop_ || (!queue_.empty() && admissible_locked(recs_[queue_.front()]));
    });
    if (stop_) return;
    const uint64_t t = queue_.front();
    queue_.pop_front();
    Rec& r = recs_[t];
    r.waiting = false;
    r.running = true;
    r.hold_until = -1;
    r.out.slot = slot;
    r.out.attempts += 1;
    r.out.t_start = now();
    st_.waiting = int32_t(queue_.size());
    st_.running += 1;
    st_.peak_running = std::max(st_.peak_running, st_.running);
    st_.in_use_bytes += r.footprint;
    st_.peak_bytes = std::max(st_.peak_bytes, st_.in_use_bytes);
    void* payload = r.payload;
    lk.unlock();
    // another slot may admit the next request while this one runs
    work_cv_.notify_all();
    int32_t status = kArg;
    try {
      status = run_(slot, payload);
    } catch (...) {
      status = kArg;
    }
    lk.lock();
    Rec& q = recs_[t];
    q.running = false;
    st_.running -= 1;
    st_.in_use_bytes -= q.footprint;
    const bool retry = status == kOom && st_.running > 0 && q.out.attempts < max_attempts_ && !stop_;
    if (retry) {
      // out of memory next to other requests: back to the head of the queue, admissible
      // again after one of those finishes
      q.waiting = true;
      q.hold_until = completions_;
      queue_.push_front(t);
      st_.waiting = int32_t(queue_.size());
      ++st_.retried;
    } else {
      q.done = true;
      q.out.status = status;
      q.out.t_finish = now();
      ++completions_;
      ++st_.finished;
    }
    lk.unlock();
    work_cv_.notify_all();
    done_cv_.notify_all();
    lk.lock();
  }
}

int32_t Scheduler::poll(uint64_t ticket, int64_t wait_ms, Outcome* out, void** payload) {
  std::unique_lock<std::mutex> lk(mu_);
  if (recs_.find(ticket) == recs_.end()) return kArg;
  // looked up afresh after every wake-up: another poller of the same ticket may have
  // taken the result meanwhile
  auto finished = [&] {
    auto f = recs_.find(ticket);
    return f == recs_.end() || f->second.done;
  };
  if (!finished()) {
    if (wait_ms == 0) return kPending;
    if (wait_ms < 0) {
      done_cv_.wait(lk, finished);
    } else if (!done_cv_.wait_for(lk, std::chrono::milliseconds(wait_ms), finished)) {
      return kPending;
    }
  }
  auto it = recs_.find(ticket);
  if (it == recs_.end()) return kArg;
  if (out) *out = it->second.out;
  if (payload) *payload = it->second.payload;
  recs_.erase(it);
  return kOk;
}

int32_t Scheduler::cancel(uint64_t ticket) {
  {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = recs_.find(ticket);
    if (it == recs_.end()) return kArg;
    Rec& r = it->second;
    if (!r.waiting) return kState;
    queue_.erase(std::find(queue_.begin(), queue_.end(), ticket));
    r.waiting = false;
    r.done = true;
    r.out.status = kCancelled;
    r.out.t_finish = now();
    st_.waiting = int32_t(queue_.size());
    ++st_.cancelled;
  }
  // the new head of the queue may fit where the cancelled one did not
  work_cv_.notify_all();
  done_cv_.notify_all();
  return kOk;
}

Stats Scheduler::stats() const {
  std::lock_guard<std::mutex> lk(mu_);
  return st_;
}

}  // namespace serve
}  // namespace mlcc
