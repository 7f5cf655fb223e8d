"""The request scheduler of the serving loop (csrc/scheduler.cpp), compiled on its own with
g++ and driven by fake work on the host (no GPU). A fake request sleeps for a set time,
returns a set status and can report out-of-memory on its first admission; the fake
records how many requests and bytes run at once. Checked:
  * every request finishes with its own status; slots and the memory budget are never
    exceeded, and the slots are used;
  * admission is first-come first-served: start times follow submission order, and a
    small request that would fit does not overtake a large one waiting for memory;
  * requests submitted while others run are admitted as slots free up;
  * out of memory next to running requests: the request is re-admitted after one of them
    finishes; alone, its status is final;
  * rejection above the budget, cancellation, pending polls, unknown tickets, and
    destruction with requests still queued (no hang, their payloads released).
"""
import ctypes
import os
import shutil
import subprocess
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_05226_gb300", "csrc")

OK, PENDING, ARG, OOM, STATE, REJECTED, CANCELLED = 0, 1, -1, -2, -9, -10, -11

SHIM = r"""
#include "scheduler.h"
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <thread>
using namespace mlcc::serve;

struct Fake {
  int64_t fp = 0;
  int sleep_ms = 0, status = 0, oom_first = 0;
  int attempts_seen = 0, slot_seen = -1;
};

struct Harness {
  std::atomic<int> running{0}, peak{0};
  std::atomic<int64_t> bytes{0}, peak_bytes{0};
  std::atomic<int> dropped{0};
  std::mutex mu;
  std::map<uint64_t, Fake*> fakes;
  Scheduler* s = nullptr;
};

static int32_t fake_run(Harness* h, void* p) {
  Fake* f = static_cast<Fake*>(p);
  const int r = ++h->running;
  int pk = h->peak.load();
  while (r > pk && !h->peak.compare_exchange_weak(pk, r)) {}
  const int64_t b = (h->bytes += f->fp);
  int64_t pb = h->peak_bytes.load();
  while (b > pb && !h->peak_bytes.compare_exchange_weak(pb, b)) {}
  f->attempts_seen += 1;
  int32_t st = f->status;
  if (f->oom_first && f->attempts_seen == 1) st = kOom;
  std::this_thread::sleep_for(std::chrono::milliseconds(f->sleep_ms));
  h->bytes -= f->fp;
  --h->running;
  return st;
}

extern "C" void* t_create(int slots, int64_t budget, int max_attempts) {
  Harness* h = new Harness();
  h->s = new Scheduler(slots, budget, [h](int slot, void* p) {
    static_cast<Fake*>(p)->slot_seen = slot;
    return fake_run(h, p);
  }, [h](void* p) { ++h->dropped; delete static_cast<Fake*>(p); }, max_attempts);
  return h;
}
extern "C" int t_submit(void* hv, int64_t fp, int sleep_ms, int status, int oom_first, uint64_t* ticket) {
  Harness* h = static_cast<Harness*>(hv);
  Fake* f = new Fake();
  f->fp = fp; f->sleep_ms = sleep_ms; f->status = status; f->oom_first = oom_first;
  const int st = h->s->submit(fp, f, ticket);
  if (st != kOk) { delete f; return st; }
  return st;
}
// out: status, slot, attempts, t_submit_us, t_start_us, t_finish_us, attempts_seen, slot_seen
extern "C" int t_poll(void* hv, uint64_t ticket, int64_t wait_ms, double* out) {
  Harness* h = static_cast<Harness*>(hv);
  Outcome o;
  void* p = nullptr;
  const int st = h->s->poll(ticket, wait_ms, &o, &p);
  if (st != kOk) return st;
  Fake* f = static_cast<Fake*>(p);
  out[0] = o.status; out[1] = o.slot; out[2] = o.attempts;
  out[3] = o.t_submit; out[4] = o.t_start; out[5] = o.t_finish;
  out[6] = f->attempts_seen; out[7] = f->slot_seen;
  delete f;
  return st;
}
extern "C" int t_cancel(void* hv, uint64_t ticket) { return static_cast<Harness*>(hv)->s->cancel(ticket); }
// out: submitted, finished, cancelled, retried, running, waiting, peak_running, in_use, peak_bytes,
//      harness peak running, harness peak bytes
extern "C" void t_stats(void* hv, int64_t* out) {
  Harness* h = static_cast<Harness*>(hv);
  const Stats s = h->s->stats();
  out[0] = s.submitted; out[1] = s.finished; out[2] = s.cancelled; out[3] = s.retried;
  out[4] = s.running; out[5] = s.waiting; out[6] = s.peak_running; out[7] = s.in_use_bytes;
  out[8] = s.peak_bytes; out[9] = h->peak.load(); out[10] = h->peak_bytes.load();
}
extern "C" int t_destroy(void* hv) {
  Harness* h = static_cast<Harness*>(hv);
  delete h->s;
  const int d = h->dropped.load();
  delete h;
  return d;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("scheduler")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libscheduler_test.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared", f"-I{CSRC}", str(shim),
                    os.path.join(CSRC, "scheduler.cpp"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.t_create.restype = ctypes.c_void_p
    L.t_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    L.t_submit.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_uint64)]
    L.t_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    L.t_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.t_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    L.t_destroy.argtypes = [ctypes.c_void_p]
    return L


class Sched:
    def __init__(self, lib, slots, budget, max_attempts=3):
        self.L = lib
        self.h = lib.t_create(slots, budget, max_attempts)

    def submit(self, fp, sleep_ms=0, status=OK, oom_first=0):
        t = ctypes.c_uint64(0)
        st = self.L.t_submit(self.h, fp, sleep_ms, status, oom_first, ctypes.byref(t))
        return st, t.value

    def poll(self, ticket, wait_ms=-1):
        out = (ctypes.c_double * 8)()
        st = self.L.t_poll(self.h, ticket, wait_ms, out)
        if st != OK:
            return st, None
        keys = ["status", "slot", "attempts", "t_submit", "t_start", "t_finish", "attempts_seen", "slot_seen"]
        return st, dict(zip(keys, list(out)))

    def cancel(self, ticket):
        return self.L.t_cancel(self.h, ticket)

    def stats(self):
        out = (ctypes.c_int64 * 11)()
        self.L.t_stats(self.h, out)
        keys = ["submitted", "finished", "cancelled", "retried", "running", "waiting", "peak_running",
                "in_use", "peak_bytes", "fake_peak_running", "fake_peak_bytes"]
        return dict(zip(keys, list(out)))

    def destroy(self):
        return self.L.t_destroy(self.h)


def test_every_request_finishes_with_its_status_within_slots_and_budget(lib):
    s = Sched(lib, 3, 1000)
    sizes = [100, 400, 250, 600, 50, 300, 700, 150, 200, 350, 500, 90]
    statuses = [OK, -3, OK, OK, -4, OK, OK, -6, OK, OK, OK, -5]
    tickets = []
    for fp, st in zip(sizes, statuses):
        r, t = s.submit(fp, sleep_ms=15, status=st)
        assert r == OK and t > 0
        tickets.append(t)
    assert len(set(tickets)) == len(tickets)
    outs = [s.poll(t)[1] for t in tickets]
    for o, st in zip(outs, statuses):
        assert o["status"] == st and o["attempts"] == 1 and o["attempts_seen"] == 1
        assert 0 <= o["slot"] < 3 and o["slot"] == o["slot_seen"]
        assert o["t_submit"] <= o["t_start"] <= o["t_finish"]
    st = s.stats()
    assert st["submitted"] == st["finished"] == len(sizes)
    assert st["running"] == 0 and st["waiting"] == 0 and st["in_use"] == 0
    assert 2 <= st["fake_peak_running"] <= 3 and st["peak_running"] <= 3
    assert st["fake_peak_bytes"] <= 1000 and st["peak_bytes"] <= 1000
    assert s.destroy() == 0


def test_all_slots_run_at_once_when_memory_allows(lib):
    s = Sched(lib, 4, 10**12)
    tickets = [s.submit(10, sleep_ms=60)[1] for _ in range(8)]
    for t in tickets:
        assert s.poll(t)[1]["status"] == OK
    assert s.stats()["fake_peak_running"] == 4
    s.destroy()


def test_admission_is_first_come_first_served(lib):
    s = Sched(lib, 2, 10**9)
    tickets = [s.submit(5, sleep_ms=5)[1] for _ in range(20)]
    starts = [s.poll(t)[1]["t_start"] for t in tickets]
    assert all(b >= a for a, b in zip(starts, starts[1:]))
    s.destroy()


def test_small_request_does_not_overtake_one_waiting_for_memory(lib):
    s = Sched(lib, 3, 100)
    a = s.submit(60, sleep_ms=120)[1]     # runs
    b = s.submit(60, sleep_ms=10)[1]      # does not fit next to a: waits
    c = s.submit(10, sleep_ms=10)[1]      # would fit next to a, but b is older
    oa, ob, oc = s.poll(a)[1], s.poll(b)[1], s.poll(c)[1]
    assert ob["t_start"] >= oa["t_finish"] - 1e-3
    assert oc["t_start"] >= ob["t_start"]
    assert s.stats()["fake_peak_bytes"] <= 100
    s.destroy()


def test_requests_arriving_later_are_admitted_as_slots_free(lib):
    s = Sched(lib, 2, 10**9)
    first = [s.submit(1, sleep_ms=150)[1] for _ in range(2)]
    time.sleep(0.03)
    late = s.submit(1, sleep_ms=10)[1]    # arrives while both slots are busy
    o_first = [s.poll(t)[1] for t in first]
    o_late = s.poll(late)[1]
    assert o_late["t_start"] >= min(o["t_finish"] for o in o_first) - 1e-3
    assert o_late["t_start"] < max(o["t_finish"] for o in o_first) + 0.1
    s.destroy()


def test_rejection_and_bad_sizes(lib):
    s = Sched(lib, 1, 100)
    assert s.submit(101)[0] == REJECTED
    assert s.submit(0)[0] == ARG
    assert s.submit(-5)[0] == ARG
    r, t = s.submit(100)
    assert r == OK
    assert s.poll(t)[1]["status"] == OK
    assert s.stats()["submitted"] == 1
    s.destroy()


def test_out_of_memory_next_to_running_request_is_retried_after_it_finishes(lib):
    s = Sched(lib, 2, 10**9)
    a = s.submit(10, sleep_ms=150)[1]
    time.sleep(0.02)
    b = s.submit(10, sleep_ms=5, oom_first=1)[1]
    oa, ob = s.poll(a)[1], s.poll(b)[1]
    assert oa["status"] == OK
    assert ob["status"] == OK and ob["attempts"] == 2 and ob["attempts_seen"] == 2
    assert ob["t_start"] >= oa["t_finish"] - 1e-3
    assert s.stats()["retried"] == 1
    s.destroy()


def test_out_of_memory_alone_is_final(lib):
    s = Sched(lib, 2, 10**9)
    t = s.submit(10, sleep_ms=1, oom_first=1)[1]
    o = s.poll(t)[1]
    assert o["status"] == OOM and o["attempts"] == 1
    s.destroy()


def test_retries_are_bounded(lib):
    s = Sched(lib, 2, 10**9, max_attempts=2)
    a = s.submit(10, sleep_ms=200)[1]
    b = s.submit(10, sleep_ms=120, status=OOM)[1]   # out of memory on every admission
    time.sleep(0.01)
    c = s.submit(10, sleep_ms=400)[1]
    ob = s.poll(b)[1]
    assert ob["status"] == OOM and ob["attempts"] <= 2
    s.poll(a), s.poll(c)
    s.destroy()


def test_cancel_poll_and_unknown_tickets(lib):
    s = Sched(lib, 1, 10**9)
    a = s.submit(10, sleep_ms=150)[1]
    b = s.submit(10, sleep_ms=150)[1]
    time.sleep(0.03)
    assert s.poll(a, wait_ms=0)[0] == PENDING
    assert s.poll(a, wait_ms=10)[0] == PENDING
    assert s.cancel(a) == STATE            # running
    assert s.cancel(b) == OK               # waiting
    assert s.cancel(b) == STATE            # already finished (cancelled)
    ob = s.poll(b, wait_ms=0)[1]
    assert ob["status"] == CANCELLED and ob["slot"] == -1 and ob["attempts"] == 0
    assert s.poll(a)[1]["status"] == OK
    assert s.poll(a)[0] == ARG             # already polled
    assert s.poll(12345)[0] == ARG and s.cancel(12345) == ARG
    assert s.stats()["cancelled"] == 1
    s.destroy()


def test_destroy_with_queued_requests_returns_and_releases_them(lib):
    s = Sched(lib, 1, 10**9)
    for _ in range(5):
        s.submit(10, sleep_ms=50)
    time.sleep(0.01)
    t0 = time.time()
    dropped = s.destroy()
    assert time.time() - t0 < 1.0          # only the running request is waited for
    assert dropped == 5                    # nobody polled them


def test_many_random_requests(lib):
    import random
    rng = random.Random(7)
    budget = 1000
    s = Sched(lib, 4, budget)
    tickets = []
    for _ in range(200):
        fp = rng.randint(1, budget)
        tickets.append((s.submit(fp, sleep_ms=rng.randint(0, 2), status=rng.choice([OK, -3]))[1], fp))
    starts = []
    for t, fp in tickets:
        o = s.poll(t)[1]
        assert o["status"] in (OK, -3)
        starts.append(o["t_start"])
    assert all(b >= a for a, b in zip(starts, starts[1:]))
    st = s.stats()
    assert st["finished"] == 200 and st["fake_peak_bytes"] <= budget and st["fake_peak_running"] <= 4
    s.destroy()
