// Request scheduler of the serving loop: admission by device-memory footprint into a fixed
// number of slots, one worker thread per slot, first-come first-served. Plain C++17 with
// no CUDA: the work of a request is a callback, so the same code runs excitation solves in
// the library and fake work in host-only tests.
#pragma once
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace mlcc {
namespace serve {

// Scheduler status codes; the values are those of mlcc_status in the C ABI.
enum : int32_t {
  kOk = 0,
  kPending = 1,      // poll: the request has not finished
  kArg = -1,         // unknown ticket, bad size
  kOom = -2,         // the work ran out of device memory
  kState = -9,       // cancel of a request that is running or finished
  kRejected = -10,   // footprint above the whole budget
  kCancelled = -11,  // the request was cancelled before it started
};

struct Outcome {
  int32_t status = kPending;   // the work's status, or kCancelled
  int32_t slot = -1;           // slot that ran it last (-1: never ran)
  int32_t attempts = 0;        // admissions (more than 1 after out-of-memory retries)
  int64_t footprint = 0;       // bytes it was admitted with
  double t_submit = 0.0;       // seconds since the scheduler was created
  double t_start = 0.0;        // last admission
  double t_finish = 0.0;
};

struct Stats {
  int64_t submitted = 0, finished = 0, cancelled = 0, retried = 0;
  int32_t running = 0, waiting = 0;
  int32_t peak_running = 0;
  int64_t in_use_bytes = 0, peak_bytes = 0;
};

class Scheduler {
 public:
  // run(slot, payload) executes one request on the worker thread of `slot` and returns its
  // status. It may return kOom: while other requests run, the request goes back to the
  // head of the queue until one of them finishes (at most max_attempts admissions).
  using RunFn = std::function<int32_t(int slot, void* payload)>;
  // drop(payload) releases the payload of a request the caller never polled (destruction).
  using DropFn = std::function<void(void* payload)>;

  Scheduler(int n_slots, int64_t budget_bytes, RunFn run, DropFn drop = {}, int max_attempts = 3);
  ~Scheduler();   // cancels waiting requests, lets running ones finish, joins the workers
  Scheduler(const Scheduler&) = delete;
  Scheduler& operator=(const Scheduler&) = delete;

  // Queues a request of `footprint` bytes (1 <= footprint <= budget, else kRejected or
  // kArg) and returns its ticket (> 0).
  int32_t submit(int64_t footprint, void* payload, uint64_t* ticket);
  // Waits up to wait_ms (0: no wait, < 0: until it finishes) for the request. On kOk fills
  // out and *payload and forgets the ticket; kPending if it has not finished; kArg for an
  // unknown ticket.
  int32_t poll(uint64_t ticket, int64_t wait_ms, Outcome* out, void** payload);
  // Removes a waiting request: kOk (poll then reports kCancelled), kState if it is running
  // or finished, kArg for an unknown ticket.
  int32_t cancel(uint64_t ticket);
  Stats stats() const;
  int n_slots() const { return int(workers_.size()); }
  int64_t budget() const { return budget_; }

 private:
  struct Rec {
    void* payload = nullptr;
    int64_t footprint = 0;
    bool waiting = false, running = false, done = false;
    int64_t hold_until = -1;   // admissible once completions_ exceeds this (OOM retry)
    Outcome out;
  };
  void worker(int slot);
  bool admissible_locked(const Rec& r) const;
  double now() const;

  const int64_t budget_;
  const int max_attempts_;
  RunFn run_;
  DropFn drop_;
  mutable std::mutex mu_;
  std::condition_variable work_cv_;   // workers: a request may be admissible
  std::condition_variable done_cv_;   // pollers: a request finished
  std::deque<uint64_t> queue_;        // waiting tickets, oldest first
  std::map<uint64_t, Rec> recs_;
  uint64_t next_ticket_ = 1;
  int64_t completions_ = 0;
  bool stop_ = false;
  Stats st_;
  std::vector<std::thread> workers_;
  const double t0_;
};

}  // namespace serve
}  // namespace mlcc
