// Serving loop of the C ABI: independent excitation solves submitted by tickets, admitted by
// device-memory footprint into slots, each slot a worker thread with its own context and
// stream, so that the work of admitted requests overlaps on the device.
#include "internal.cuh"
#include "scheduler.h"
#include "sizes.h"

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

using namespace mlcc;

static_assert(int(serve::kOk) == int(MLCC_OK) && int(serve::kPending) == int(MLCC_PENDING) &&
                  int(serve::kArg) == int(MLCC_E_ARG) && int(serve::kOom) == int(MLCC_E_OOM) &&
                  int(serve::kState) == int(MLCC_E_STATE) && int(serve::kRejected) == int(MLCC_E_REJECTED) &&
                  int(serve::kCancelled) == int(MLCC_E_CANCELLED),
              "scheduler status codes are the C ABI's");

struct mlcc_server {
  int device = 0;
  std::vector<mlcc_ctx*> ctx;                  // one per slot
  std::unique_ptr<serve::Scheduler> sched;
};

namespace {

// one request: a copy of the problem and options, the borrowed host inputs, the outputs
struct Job {
  mlcc_problem prob{};
  std::vector<int8_t> level;
  const double* chol = nullptr;
  const double* fock = nullptr;
  mlcc_options opt{};
  std::vector<double> omega;
  mlcc_gs_info gs{};
  mlcc_es_info es{};
  std::string error;
};

bool split(int p) { return p == MLCC_BF16 || p == MLCC_BF16X3 || p == MLCC_BF16X6; }
int pieces(int p) { return p == MLCC_BF16X6 ? 6 : p == MLCC_BF16X3 ? 3 : p == MLCC_BF16 ? 1 : 0; }

// bytes per element of the cached operand copies of one sigma precision: bfloat16 pieces of
// the split products, or the 8 integer digits (2 bytes each) and a row exponent share of
// the binary64 emulation
int cache_bytes_per_element(int p) {
  if (split(p)) return 2 * pieces(p);
  if (p == MLCC_FP64E) return 17;
  return 0;
}

int64_t footprint(const sizes::Dims& d, const mlcc_options& o) {
  using sizes::round_alloc;
  const size_t system = round_alloc(sizes::persist_bytes(d)) + round_alloc(sizes::ws_bytes(d));
  // while the system is created: the caller's inputs copied to the device
  const size_t inputs = round_alloc(size_t(d.nn()) * d.nj * 8) + round_alloc(size_t(d.nn()) * 8);
  // afterwards: amplitudes, CCSD value tensors, bfloat16 operands, Davidson subspace and the
  // cached operand copies of the sigma precisions
  const size_t amps = round_alloc(size_t(d.nv) * d.no * 8 + 8) + round_alloc(size_t(d.nd) * 8 + 8);
  const int seg = std::max(pieces(o.precision), pieces(o.gs_precision));
  const size_t lowp = seg > 0 ? round_alloc(sizes::lowp_bytes(d, seg)) : 0;
  const int nr = std::max(1, o.n_roots);
  const size_t dav = round_alloc(sizes::davidson_bytes(d.vector_len(), sizes::davidson_max_subspace(o.max_subspace, nr), nr));
  int bpe = cache_bytes_per_element(o.precision);
  if (split(o.precision) && o.refine_fp64 > 0) bpe += cache_bytes_per_element(o.refine_precision);
  const size_t cache = round_alloc(sizes::operand_cache_allowance(d, bpe));
  // the ground state's ladder operand (with its largest converted copy) is gone before the
  // Jacobian's buffers are made
  const int gs_bpe = std::max(cache_bytes_per_element(o.gs_precision),
                              o.refine_fp64 > 0 ? cache_bytes_per_element(o.refine_precision) : 0);
  const size_t gsl = round_alloc(sizes::gs_ladder_bytes(d, gs_bpe));
  const size_t after = amps + std::max(gsl, round_alloc(sizes::ccsd_cache_bytes(d)) + lowp + dav + cache);
  return int64_t(system + std::max(inputs, after));
}

}  // namespace

extern "C" {

mlcc_status mlcc_solve_footprint(const mlcc_problem* prob, const mlcc_options* opt, int64_t* bytes) {
  return guard([&] {
    MLCC_REQUIRE(prob && opt && bytes, "mlcc_solve_footprint: NULL argument");
    sizes::Dims d;
    MLCC_REQUIRE(sizes::dims_from_levels(prob->n_mo, prob->n_occ, prob->n_chol, prob->level, &d),
                 "mlcc_solve_footprint: need 0 < n_occ < n_mo, n_chol > 0 and levels 0, 1 or 2");
    *bytes = footprint(d, *opt);
    return MLCC_OK;
  });
}

mlcc_status mlcc_server_create(int device, int32_t n_slots, int64_t hbm_budget_bytes, mlcc_server** out) {
  return guard([&] {
    MLCC_REQUIRE(out != nullptr, "mlcc_server_create: out is NULL");
    *out = nullptr;
    MLCC_REQUIRE(n_slots >= 1 && n_slots <= 64, "mlcc_server_create: n_slots must be in [1, 64]");
    auto srv = std::make_unique<mlcc_server>();
    srv->device = device;
    struct Undo {
      mlcc_server* s;
      ~Undo() {
        if (s)
          for (mlcc_ctx* c : s->ctx) mlcc_ctx_destroy(c);
      }
    } undo{srv.get()};
    for (int k = 0; k < n_slots; ++k) {
      mlcc_ctx* c = nullptr;
      const mlcc_status st = mlcc_ctx_create(device, &c);
      if (st != MLCC_OK) return st;
      srv->ctx.push_back(c);
    }
    int64_t budget = hbm_budget_bytes;
    if (budget <= 0) {
      size_t free_b = 0, total_b = 0;
      MLCC_CUDA(cudaSetDevice(device));
      MLCC_CUDA(cudaMemGetInfo(&free_b, &total_b));
      budget = int64_t(double(free_b) * 0.9);
    }
    mlcc_server* raw = srv.get();
    auto run = [raw](int slot, void* payload) -> int32_t {
      auto* j = static_cast<Job*>(payload);
      mlcc_result r{};
      r.omega = j->omega.data();
      const mlcc_status st = mlcc_solve(raw->ctx[slot], &j->prob, j->chol, j->fock, &j->opt, &r);
      j->gs = r.gs;
      j->es = r.es;
      if (st != MLCC_OK) j->error = mlcc_last_error();
      return st;
    };
    auto drop = [](void* payload) { delete static_cast<Job*>(payload); };
    srv->sched = std::make_unique<serve::Scheduler>(n_slots, budget, run, drop);
    undo.s = nullptr;
    *out = srv.release();
    return MLCC_OK;
  });
}

void mlcc_server_destroy(mlcc_server* srv) {
  if (!srv) return;
  srv->sched.reset();   // cancels waiting requests, waits for running ones
  for (mlcc_ctx* c : srv->ctx) mlcc_ctx_destroy(c);
  delete srv;
}

mlcc_status mlcc_submit(mlcc_server* srv, const mlcc_problem* prob, const double* chol_host,
                        const double* fock_host, const mlcc_options* opt, uint64_t* ticket) {
  return guard([&] {
    MLCC_REQUIRE(srv && prob && chol_host && fock_host && opt && ticket, "mlcc_submit: NULL argument");
    *ticket = 0;
    sizes::Dims d;
    MLCC_REQUIRE(sizes::dims_from_levels(prob->n_mo, prob->n_occ, prob->n_chol, prob->level, &d),
                 "mlcc_submit: need 0 < n_occ < n_mo, n_chol > 0 and levels 0, 1 or 2");
    MLCC_REQUIRE(opt->n_roots >= 1 && opt->n_roots <= d.nv * d.no, "mlcc_submit: n_roots out of range");
    auto job = std::make_unique<Job>();
    job->level.assign(prob->level, prob->level + prob->n_mo);
    job->prob = *prob;
    job->prob.level = job->level.data();
    job->chol = chol_host;
    job->fock = fock_host;
    job->opt = *opt;
    job->omega.assign(size_t(opt->n_roots), 0.0);
    const int32_t st = srv->sched->submit(footprint(d, *opt), job.get(), ticket);
    if (st == serve::kRejected)
      throw Error(MLCC_E_REJECTED, "mlcc_submit: the request's footprint exceeds the server's memory budget");
    if (st != serve::kOk) throw Error(MLCC_E_STATE, "mlcc_submit: the server is shutting down");
    job.release();
    return MLCC_OK;
  });
}

mlcc_status mlcc_poll(mlcc_server* srv, uint64_t ticket, int64_t wait_ms, mlcc_request_result* res,
                      double* omega_host) {
  return guard([&] {
    MLCC_REQUIRE(srv && res, "mlcc_poll: NULL argument");
    serve::Outcome o;
    void* payload = nullptr;
    const int32_t st = srv->sched->poll(ticket, wait_ms, &o, &payload);
    if (st == serve::kPending) return MLCC_PENDING;
    MLCC_REQUIRE(st == serve::kOk, "mlcc_poll: unknown ticket");
    std::unique_ptr<Job> job(static_cast<Job*>(payload));
    *res = mlcc_request_result{};
    res->status = o.status;
    res->slot = o.slot;
    res->attempts = o.attempts;
    res->n_roots = int32_t(job->omega.size());
    res->footprint_bytes = o.footprint;
    res->t_submit = o.t_submit;
    res->t_start = o.t_start;
    res->t_finish = o.t_finish;
    res->gs = job->gs;
    res->es = job->es;
    if (omega_host && o.status != MLCC_E_CANCELLED)
      std::copy(job->omega.begin(), job->omega.end(), omega_host);
    if (o.status != MLCC_OK && o.status != MLCC_E_CANCELLED) set_last_error(job->error);
    return MLCC_OK;
  });
}

mlcc_status mlcc_cancel(mlcc_server* srv, uint64_t ticket) {
  return guard([&] {
    MLCC_REQUIRE(srv != nullptr, "mlcc_cancel: NULL server");
    const int32_t st = srv->sched->cancel(ticket);
    MLCC_REQUIRE(st != serve::kArg, "mlcc_cancel: unknown ticket");
    if (st == serve::kState) throw Error(MLCC_E_STATE, "mlcc_cancel: the request has started");
    return MLCC_OK;
  });
}

mlcc_status mlcc_server_stats(mlcc_server* srv, mlcc_server_info* info) {
  return guard([&] {
    MLCC_REQUIRE(srv && info, "mlcc_server_stats: NULL argument");
    const serve::Stats s = srv->sched->stats();
    *info = mlcc_server_info{};
    info->n_slots = srv->sched->n_slots();
    info->budget_bytes = srv->sched->budget();
    info->submitted = s.submitted;
    info->finished = s.finished;
    info->cancelled = s.cancelled;
    info->retried = s.retried;
    info->running = s.running;
    info->waiting = s.waiting;
    info->peak_running = s.peak_running;
    info->in_use_bytes = s.in_use_bytes;
    info->peak_bytes = s.peak_bytes;
    return MLCC_OK;
  });
}

}  // extern "C"
