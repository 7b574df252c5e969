// Serving form: a request loop over independent space-time solves.
//
// Requests queue in arrival order.  A scheduler thread admits the request at the
// head of the queue as soon as an in-flight slot is free and its device memory
// (wr_estimate_bytes plus its solution vector) fits in the remaining budget;
// a request larger than the whole budget is refused.
//
// Per-request mode (wr_server_create): every admitted request runs on a worker
// thread with its own CUDA stream and context, so its level hierarchy, factors and
// Krylov state stay on the device for the whole solve, and the kernels of all
// in-flight solves overlap on the GPU.  When a solve completes its memory and slot
// are released and the scheduler admits the next requests at once.  Each solve runs
// the same deterministic kernels on its own stream, so its result does not depend on
// what else is in flight.
//
// Batched mode (wr_server_create_batched): a slot holds a cohort.  When a slot is
// free, the scheduler takes the head request and every queued request with the same
// (k, q) behind it, in arrival order, up to max_members and the remaining budget, and
// solves them as one lock-step batch (wr_batch: one launch per stage of every V-cycle,
// Newton step and FGMRES iteration for all members, V-cycles replayed as CUDA
// graphs) on the slot's stream.  Cohorts in different slots overlap on the device;
// requests arriving while cohorts run form the next cohort as soon as a slot and
// memory free up.  A member is handed back the moment it leaves its cohort
// (converged, given up, failed or cancelled), so its latency is its own; the
// cohort's memory is released when its last member leaves.  A member's result is its
// solve alone up to rounding (the apply tiles are tuned per cohort).  Requests the
// batch engine does not take (the heat equation, DG(2) and DG(3)) run in the
// per-request way in a slot of their own.
#include <chrono>
#include <condition_variable>
#include <atomic>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "wrmg_internal.h"

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  wr_problem p;
  std::vector<int> mx, my;
  std::vector<double> amp;
  std::vector<double> U0;  // optional initial iterate (host)
  std::vector<double> U;   // result (host)
  wr_stats st;
  int status = WR_ERR_STATE;  // WR_ERR_STATE while queued or running
  bool done = false;
  std::atomic<int> cancel{0};
  int64_t bytes = 0, ndofs = 0;
  double t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct wr_server {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<std::thread> workers;
  std::thread scheduler;
  wr_options opt;
  int64_t budget = 0, used = 0, peak_used = 0;
  int max_inflight = 1, inflight = 0, peak_inflight = 0, device = 0;
  int max_members = 1;  // > 1: batched mode, cohorts of up to max_members requests per slot
  int peak_cohort = 0;
  uint64_t next_id = 1;
  bool stopping = false;
  std::string err;

  // Smaller solves get higher stream priority (the block scheduler then starts their
  // CTAs first whenever SMs free up), so short requests are not stuck behind the
  // persistent kernels of long ones: one priority level per factor 4 in DoFs above
  // 16 Ki DoFs, clamped to the device's range.
  int prio_least = 0, prio_greatest = 0;
  int priority_of(int64_t ndofs) const {
    int lvl = 0;
    for (int64_t d = ndofs >> 14; d > 1 && lvl < 32; d >>= 2) ++lvl;
    const int p = prio_greatest + lvl;  // greatest priority is numerically smallest
    return p < prio_least ? p : prio_least;
  }

  void run_one(std::shared_ptr<Request> r) {
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    wr_ctx* c = nullptr;
    double* dU = nullptr;
    int rc = WR_OK;
    std::memset(&r->st, 0, sizeof(r->st));
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority_of(r->ndofs)) != cudaSuccess)
      rc = WR_ERR_CUDA;
    if (rc == WR_OK && r->cancel.load()) rc = WR_ERR_CANCELLED;
    if (rc == WR_OK) rc = create_context(&c, &r->p, &opt, s, true);
    if (c) set_cancel_flag(c, &r->cancel);
    if (rc == WR_OK && cudaMallocAsync(&dU, sizeof(double) * r->ndofs, s) != cudaSuccess) rc = WR_ERR_NOMEM;
    if (rc == WR_OK) {
      if (!r->U0.empty()) {
        if (cudaMemcpyAsync(dU, r->U0.data(), sizeof(double) * r->ndofs, cudaMemcpyHostToDevice, s) != cudaSuccess)
          rc = WR_ERR_CUDA;
      } else {
        rc = wr_initial_guess(c, dU);
      }
    }
    if (rc == WR_OK) rc = wr_solve(c, dU, &r->st);
    if (rc == WR_OK || rc == WR_ERR_NOT_CONVERGED) {
      r->U.resize(r->ndofs);
      if (cudaMemcpyAsync(r->U.data(), dU, sizeof(double) * r->ndofs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        rc = WR_ERR_CUDA;
    }
    if (dU) cudaFreeAsync(dU, s);
    if (c) wr_destroy(c);
    if (s) cudaStreamDestroy(s);
    std::lock_guard<std::mutex> lock(mu);
    r->status = rc;
    r->t_end = now_ms();
    r->done = true;
    used -= r->bytes;
    --inflight;
    cv.notify_all();
  }

  static bool batchable(const wr_problem& p) {
    return p.kind != WR_HEAT && p.kind != WR_HEAT_EIGEN && (p.q == 0 || p.q == 1);
  }

  // One cohort solved as a lock-step batch on its own stream; each member completes
  // as soon as it leaves the batch.
  void run_cohort(std::vector<std::shared_ptr<Request>> rs) {
    cudaSetDevice(device);
    const int n = (int)rs.size();
    int64_t maxd = 0, bytes = 0;
    for (auto& r : rs) {
      maxd = std::max(maxd, r->ndofs);
      bytes += r->bytes;
      std::memset(&r->st, 0, sizeof(r->st));
    }
    cudaStream_t s = nullptr;
    wr_batch* b = nullptr;
    std::vector<double*> dU(n, nullptr);
    std::vector<wr_stats> st(n);
    std::vector<const std::atomic<int>*> cancel(n);
    std::vector<wr_problem> ps(n);
    for (int m = 0; m < n; ++m) {
      ps[m] = rs[m]->p;
      cancel[m] = &rs[m]->cancel;
    }
    std::vector<char> handed(n, 0);
    auto complete = [&](int m, int rc) {
      auto& r = rs[m];
      if (rc == WR_OK || rc == WR_ERR_NOT_CONVERGED) {
        r->U.resize(r->ndofs);
        if (cudaMemcpyAsync(r->U.data(), dU[m], sizeof(double) * r->ndofs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          rc = WR_ERR_CUDA;
      }
      std::lock_guard<std::mutex> lock(mu);
      r->st = st[m];
      r->status = rc;
      r->t_end = now_ms();
      r->done = true;
      handed[m] = 1;
      cv.notify_all();
    };
    int rc = WR_OK;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority_of(maxd)) != cudaSuccess) rc = WR_ERR_CUDA;
    if (rc == WR_OK) rc = wr_batch_create(&b, n, ps.data(), &opt, s);
    for (int m = 0; m < n && rc == WR_OK; ++m)
      if (cudaMallocAsync(&dU[m], sizeof(double) * rs[m]->ndofs, s) != cudaSuccess) rc = WR_ERR_NOMEM;
    if (rc == WR_OK) rc = wr_batch_initial_guess(b, dU.data());
    for (int m = 0; m < n && rc == WR_OK; ++m)
      if (!rs[m]->U0.empty() && cudaMemcpyAsync(dU[m], rs[m]->U0.data(), sizeof(double) * rs[m]->ndofs,
                                                cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = WR_ERR_CUDA;
    if (rc == WR_OK) {
      const int brc = batch_solve_hooked(b, dU.data(), st.data(), cancel.data(), complete);
      if (brc != WR_OK && brc != WR_ERR_NOT_CONVERGED && brc != WR_ERR_NAN) rc = brc;
    }
    for (int m = 0; m < n; ++m)
      if (!handed[m]) complete(m, rc == WR_OK ? WR_ERR_STATE : rc);
    for (double* p : dU)
      if (p) cudaFreeAsync(p, s);
    if (b) wr_batch_destroy(b);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    std::lock_guard<std::mutex> lock(mu);
    used -= bytes;
    --inflight;
    cv.notify_all();
  }

  void schedule() {
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
      cv.wait(lock, [&] {
        if (stopping) return true;
        if (queue.empty()) return false;
        const auto& h = queue.front();
        return h->bytes > budget || (inflight < max_inflight && used + h->bytes <= budget);
      });
      if (stopping && queue.empty()) return;
      if (stopping) {  // refuse what is still queued
        for (auto& r : queue) {
          r->status = WR_ERR_STATE;
          r->done = true;
        }
        queue.clear();
        cv.notify_all();
        return;
      }
      auto r = queue.front();
      queue.pop_front();
      if (r->bytes > budget) {
        r->status = WR_ERR_NOMEM;
        r->t_end = now_ms();
        r->done = true;
        cv.notify_all();
        continue;
      }
      used += r->bytes;
      ++inflight;
      r->t_start = now_ms();
      if (max_members > 1 && batchable(r->p)) {
        // the cohort: r and the queued requests of the same (k, q) behind it that fit
        std::vector<std::shared_ptr<Request>> cohort{r};
        for (auto it = queue.begin(); it != queue.end() && (int)cohort.size() < max_members;) {
          const auto& c = *it;
          if (batchable(c->p) && c->p.k == r->p.k && c->p.q == r->p.q && used + c->bytes <= budget) {
            used += c->bytes;
            c->t_start = r->t_start;
            cohort.push_back(c);
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
        peak_cohort = std::max(peak_cohort, (int)cohort.size());
        workers.emplace_back([this, cohort] { run_cohort(cohort); });
      } else {
        workers.emplace_back([this, r] { run_one(r); });
      }
      peak_used = std::max(peak_used, used);
      peak_inflight = std::max(peak_inflight, inflight);
    }
  }
};

extern "C" {

int wr_server_create(wr_server** out, int64_t mem_budget_bytes, int max_inflight, const wr_options* o) {
  if (!out || mem_budget_bytes <= 0 || max_inflight < 1) return WR_ERR_ARG;
  auto sv = std::make_unique<wr_server>();
  if (o) sv->opt = *o;
  else wr_default_options(&sv->opt);
  sv->budget = mem_budget_bytes;
  sv->max_inflight = max_inflight;
  if (cudaGetDevice(&sv->device) != cudaSuccess) return WR_ERR_CUDA;
  if (cudaDeviceGetStreamPriorityRange(&sv->prio_least, &sv->prio_greatest) != cudaSuccess) return WR_ERR_CUDA;
  // keep freed blocks in this process's default pool up to the budget, so that
  // admissions after completions reuse them instead of mapping memory afresh
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
    uint64_t keep = (uint64_t)mem_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  wr_server* raw = sv.get();
  sv->scheduler = std::thread([raw] { raw->schedule(); });
  *out = sv.release();
  return WR_OK;
}

int wr_server_create_batched(wr_server** out, int64_t mem_budget_bytes, int max_cohorts, int max_members,
                             const wr_options* o) {
  if (!out || max_members < 1) return WR_ERR_ARG;
  const int rc = wr_server_create(out, mem_budget_bytes, max_cohorts, o);
  if (rc == WR_OK) {
    std::lock_guard<std::mutex> lock((*out)->mu);
    (*out)->max_members = max_members;
  }
  return rc;
}

int wr_server_destroy(wr_server* sv) {
  if (!sv) return WR_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stopping = true;
    sv->cv.notify_all();
  }
  if (sv->scheduler.joinable()) sv->scheduler.join();
  for (auto& t : sv->workers)
    if (t.joinable()) t.join();
  delete sv;
  return WR_OK;
}

int wr_server_submit(wr_server* sv, const wr_problem* p, const double* U0_host, uint64_t* ticket) {
  if (!sv || !p || !ticket) return WR_ERR_ARG;
  auto r = std::make_shared<Request>();
  r->p = *p;
  if (p->n_modes > 0) {
    if (!p->mx || !p->my || !p->amp || p->n_modes > 8) return WR_ERR_ARG;
    r->mx.assign(p->mx, p->mx + p->n_modes);
    r->my.assign(p->my, p->my + p->n_modes);
    r->amp.assign(p->amp, p->amp + p->n_modes);
    r->p.mx = r->mx.data();
    r->p.my = r->my.data();
    r->p.amp = r->amp.data();
  }
  int64_t est = 0;
  const int rc = wr_estimate_bytes(&r->p, &sv->opt, &est);
  if (rc != WR_OK) return rc;
  const LevelGeom g = make_geom(p->n_fine, p->k, p->q, p->n_slabs, p->T);
  r->ndofs = g.ndofs;
  r->bytes = est + (int64_t)sizeof(double) * r->ndofs;
  if (U0_host) r->U0.assign(U0_host, U0_host + r->ndofs);
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stopping) return WR_ERR_STATE;
  r->id = sv->next_id++;
  r->t_submit = now_ms();
  sv->reqs[r->id] = r;
  sv->queue.push_back(r);
  *ticket = r->id;
  sv->cv.notify_all();
  return WR_OK;
}

// Returns WR_ERR_STATE while the request is queued or running (wait == 0), else the
// solve's status; on completion copies the solution (U_host may be NULL), the
// statistics and the latency (submit to completion, ms) and forgets the ticket.
int wr_server_poll(wr_server* sv, uint64_t ticket, int wait, double* U_host, wr_stats* st, double* latency_ms) {
  if (!sv) return WR_ERR_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return WR_ERR_ARG;
  auto r = it->second;
  if (wait) sv->cv.wait(lock, [&] { return r->done; });
  if (!r->done) return WR_ERR_STATE;
  if (U_host && !r->U.empty()) std::memcpy(U_host, r->U.data(), sizeof(double) * r->ndofs);
  if (st) *st = r->st;
  if (latency_ms) *latency_ms = r->t_end - r->t_submit;
  sv->reqs.erase(it);
  return r->status;
}

int wr_server_cancel(wr_server* sv, uint64_t ticket) {
  if (!sv) return WR_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return WR_ERR_ARG;
  auto r = it->second;
  if (r->done) return WR_OK;
  r->cancel.store(1);
  for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
    if (*q == r) {  // still queued: complete it now
      sv->queue.erase(q);
      r->status = WR_ERR_CANCELLED;
      r->t_end = now_ms();
      r->done = true;
      sv->cv.notify_all();
      break;
    }
  return WR_OK;
}

// Peak device bytes admitted at once and peak number of solves in flight so far.
int wr_server_stats(wr_server* sv, int64_t* peak_bytes, int* peak_inflight) {
  if (!sv) return WR_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (peak_bytes) *peak_bytes = sv->peak_used;
  if (peak_inflight) *peak_inflight = sv->peak_inflight;
  return WR_OK;
}

// Largest cohort solved as one batch so far (batched mode; 0 in per-request mode).
int wr_server_peak_cohort(wr_server* sv, int* out) {
  if (!sv || !out) return WR_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  *out = sv->peak_cohort;
  return WR_OK;
}

}  // extern "C"
