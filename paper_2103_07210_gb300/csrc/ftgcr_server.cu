// Request scheduler of libftgcr: continuous batching of independent FT-GCR(k)
// solves (Algorithm 1) over resumable persistent launches.
//
// One scheduler thread per server owns a CUDA stream, two slot tables (FP64
// and mixed precision: a launch runs one precision) and a pool of solver
// handles.  It repeats an epoch:
//   1. admit queued requests, first come first served, while a slot of their
//      precision is free and their handle fits the device-memory budget
//      (an idle pooled handle of the same shape is reused: its coefficients
//      are rebuilt from the request's D; otherwise idle handles are evicted,
//      least recently used first, until a new one fits);
//   2. stage host inputs and begin each admitted solve in its slot;
//   3. run each occupied table for at most `epoch_rounds` rounds;
//   4. hand finished solves back (host solutions copied out, statistics
//      filled) and free their slots and handles.
// A request admitted in epoch e joins the solves already running at the start
// of epoch e + 1's launch, so arrival-to-start latency is bounded by one
// epoch.  Each solve's arithmetic depends only on its own handle, so a served
// result is bitwise the result of the same solve run alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ftgcr.h"
#include "ftgcr_serve.h"

namespace {

using namespace ftgcr::serve;

struct HandleKey {
  ftgcr_grid grid;
  int32_t k;
  double tol;
  bool operator==(const HandleKey& o) const {
    return grid.nlon == o.grid.nlon && grid.nlat == o.grid.nlat && grid.mu == o.grid.mu &&
           grid.precision == o.grid.precision && grid.precond == o.grid.precond && grid.max_steps == o.grid.max_steps &&
           grid.tiles == o.grid.tiles && grid.inner_tol == o.grid.inner_tol && grid.max_outer == o.grid.max_outer &&
           grid.flags == o.grid.flags && k == o.k && tol == o.tol;
  }
};

struct PoolEntry {
  HandleKey key;
  ftgcr_handle* h = nullptr;  // created by the scheduler thread on first use
  const double* setup_D = nullptr;  // coefficients the handle was last set up from
  uint64_t setup_key = 0;           // with their caller-given identity (0: none)
  int64_t bytes = 0;
  bool busy = false;
  uint64_t last_used = 0;
};

struct Request {
  int64_t ticket = 0;
  HandleKey key;
  const double* D = nullptr;
  uint64_t ckey = 0;
  const double* rhs = nullptr;
  double* x = nullptr;
  std::vector<ftgcr_fault> faults;
  std::vector<ftgcr_loss> losses;
  int64_t footprint = 0;
  // placement
  PoolEntry* entry = nullptr;
  int table = -1, slot = -1;
  bool x_host = false;
  // result
  bool done = false;
  int status = FTGCR_PENDING;
  ftgcr_stats_t stats{};
};

int table_of(int precision) { return precision == FTGCR_MIXED ? 1 : 0; }

}  // namespace

struct ftgcr_server {
  int dev = 0;
  cudaStream_t st = nullptr;
  int64_t budget = 0, in_use = 0;
  int max_slots = 0, epoch_rounds = 0;
  SlotTable* tables[2] = {nullptr, nullptr};
  std::vector<Request*> slot_req[2];
  std::list<PoolEntry> pool;
  std::deque<Request*> queue;
  std::deque<int64_t> finished;  // tickets in order of completion, not yet collected
  std::unordered_map<int64_t, Request*> reqs;
  int64_t next_ticket = 1;
  uint64_t tick = 0;
  int64_t submitted = 0, completed = 0, running = 0, epochs = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;

  // ---- under mu
  int free_slot(int t) const {
    for (int s = 0; s < max_slots; ++s)
      if (!slot_req[t][s]) return s;
    return -1;
  }
  // An idle handle of the request's shape, preferably one already set up
  // from the same coefficients.
  PoolEntry* idle_entry(const Request* r) {
    PoolEntry* any = nullptr;
    for (PoolEntry& e : pool) {
      if (e.busy || !e.h || !(e.key == r->key)) continue;
      if (r->ckey && e.setup_key == r->ckey && e.setup_D == r->D) return &e;
      if (!any) any = &e;
    }
    return any;
  }
  // Evict idle handles (least recently used first) until `need` more bytes
  // fit; the evicted handles are destroyed by the caller, outside the lock.
  bool make_room(int64_t need, std::vector<ftgcr_handle*>& victims) {
    while (in_use + need > budget) {
      auto best = pool.end();
      for (auto it = pool.begin(); it != pool.end(); ++it)
        if (!it->busy && (best == pool.end() || it->last_used < best->last_used)) best = it;
      if (best == pool.end()) return false;
      in_use -= best->bytes;
      if (best->h) victims.push_back(best->h);
      pool.erase(best);
    }
    return true;
  }
  void admit(std::vector<Request*>& adm, std::vector<ftgcr_handle*>& victims) {
    while (!queue.empty() && !stop) {
      Request* r = queue.front();
      const int t = table_of(r->key.grid.precision);
      const int slot = free_slot(t);
      if (slot < 0) break;
      PoolEntry* e = idle_entry(r);
      if (!e) {
        if (!make_room(r->footprint, victims)) break;  // wait for running solves to free memory
        pool.emplace_back();
        e = &pool.back();
        e->key = r->key;
        e->bytes = r->footprint;
        in_use += r->footprint;
      }
      e->busy = true;
      r->entry = e;
      r->table = t;
      r->slot = slot;
      slot_req[t][slot] = r;
      queue.pop_front();
      ++running;
      adm.push_back(r);
    }
  }
  void finish_locked(Request* r, int status) {
    if (r->slot >= 0) slot_req[r->table][r->slot] = nullptr;
    if (r->entry) {
      r->entry->busy = false;
      r->entry->last_used = ++tick;
      if (!r->entry->h) {  // creation failed: drop the reservation
        in_use -= r->entry->bytes;
        for (auto it = pool.begin(); it != pool.end(); ++it)
          if (&*it == r->entry) {
            pool.erase(it);
            break;
          }
      }
      r->entry = nullptr;
    }
    r->status = status;
    r->done = true;
    finished.push_back(r->ticket);
    --running;
    ++completed;
  }

  // ---- scheduler thread, outside the lock
  int start(Request* r) {
    PoolEntry* e = r->entry;
    ftgcr_coeffs co{r->D, r->ckey};
    int rc;
    if (!e->h) {
      ftgcr_handle* h = nullptr;
      rc = ftgcr_create(&r->key.grid, &co, r->key.k, r->key.tol, &h);
      if (rc) return rc;
      std::lock_guard<std::mutex> lk(mu);
      e->h = h;
    } else if (!(r->ckey && e->setup_key == r->ckey && e->setup_D == r->D)) {
      e->setup_key = 0;  // invalid until the rebuild is enqueued
      rc = ftgcr_set_coeffs(e->h, &co, st);
      if (rc) return rc;
    }
    e->setup_D = r->D;
    e->setup_key = r->ckey;
    ftgcr_handle* h = e->h;
    const long long N = handle_points(h);
    const double* R = r->rhs;
    double* X = r->x;
    cudaPointerAttributes at;
    const bool rdev = cudaPointerGetAttributes(&at, R) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    const bool xdev = cudaPointerGetAttributes(&at, X) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    // host arrays are staged and checked for finite values on the device
    if (!rdev) {
      if (cudaMemcpyAsync(handle_stage_rhs(h), R, sizeof(double) * N, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FTGCR_ERR_CUDA;
      R = handle_stage_rhs(h);
    }
    if (!xdev) {
      if (cudaMemcpyAsync(handle_stage_x(h), X, sizeof(double) * N, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FTGCR_ERR_CUDA;
      X = handle_stage_x(h);
    }
    r->x_host = !xdev;
    ftgcr_fault_plan plan{r->faults.data(), (int32_t)r->faults.size(), r->losses.data(), (int32_t)r->losses.size()};
    const bool any = !r->faults.empty() || !r->losses.empty();
    return table_begin(tables[r->table], r->slot, h, R, X, any ? &plan : nullptr, st, (rdev ? 0 : 1) | (xdev ? 0 : 2));
  }
  void complete(Request* r) {
    ftgcr_handle* h = r->entry->h;
    int status = FTGCR_OK;
    if (r->x_host &&
        cudaMemcpy(r->x, handle_stage_x(h), sizeof(double) * handle_points(h), cudaMemcpyDeviceToHost) != cudaSuccess)
      status = FTGCR_ERR_CUDA;
    ftgcr_stats_t s{};
    const int rc = ftgcr_stats(h, &s);
    if (!status) status = rc ? rc : s.status;
    std::lock_guard<std::mutex> lk(mu);
    r->stats = s;
    finish_locked(r, status);
  }
  void fail_table(int t, int status) {
    std::vector<Request*> lost;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : slot_req[t])
        if (r) lost.push_back(r);
    }
    table_abandon(tables[t], st);
    std::lock_guard<std::mutex> lk(mu);
    for (Request* r : lost) finish_locked(r, status);
  }

  // Collect the launches in flight: hand back their finished solves.
  void collect(bool* inflight, std::vector<int>& fin) {
    for (int t = 0; t < 2; ++t) {
      if (!inflight[t]) continue;
      inflight[t] = false;
      const int rc = table_collect(tables[t], st, fin.data());
      if (rc && rc != FTGCR_ERR_TIMEOUT) {
        fail_table(t, rc);
        cv_done.notify_all();
        continue;
      }
      std::vector<Request*> done;
      {
        std::lock_guard<std::mutex> lk(mu);
        for (int s = 0; s < max_slots; ++s)
          if (fin[s] && slot_req[t][s]) done.push_back(slot_req[t][s]);
      }
      for (Request* r : done) complete(r);
      if (!done.empty()) cv_done.notify_all();
    }
  }

  // One epoch per iteration, pipelined: while launch e runs on the GPU the
  // thread admits and prepares new requests (host checks, copies and begin
  // kernels queued behind launch e), then collects launch e and enqueues
  // launch e + 1, which the prepared requests join.
  void loop() {
    cudaSetDevice(dev);
    std::vector<int> fin(max_slots);
    bool inflight[2] = {false, false};
    for (;;) {
      std::vector<Request*> adm;
      std::vector<ftgcr_handle*> victims;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (!inflight[0] && !inflight[1]) cv_work.wait(lk, [&] { return stop || running > 0 || !queue.empty(); });
        if (stop && running == 0) break;
        admit(adm, victims);
      }
      for (ftgcr_handle* h : victims) ftgcr_destroy(h);
      for (Request* r : adm) {
        const int rc = start(r);
        if (rc) {  // table_begin failed or never ran: the slot is still free
          std::lock_guard<std::mutex> lk(mu);
          finish_locked(r, rc);
          cv_done.notify_all();
        }
      }
      collect(inflight, fin);
      for (int t = 0; t < 2; ++t) {
        if (table_occupied(tables[t]) == 0) continue;
        const int rc = table_run(tables[t], epoch_rounds, st);
        if (rc) {
          fail_table(t, rc);
          cv_done.notify_all();
          continue;
        }
        inflight[t] = true;
        std::lock_guard<std::mutex> lk(mu);
        ++epochs;
      }
    }
  }

};

extern "C" {

int ftgcr_server_create(int64_t budget_bytes, int32_t max_slots, int32_t epoch_rounds, ftgcr_server** out) {
  if (!out) return FTGCR_ERR_ARG;
  *out = nullptr;
  if (budget_bytes < 0 || max_slots < 1 || max_slots > 1024 || epoch_rounds < 1) return FTGCR_ERR_ARG;
  ftgcr_server* s = new ftgcr_server();
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return FTGCR_ERR_CUDA;
  }
  if (budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return FTGCR_ERR_CUDA;
    }
    budget_bytes = (int64_t)(fr / 2);
  }
  s->budget = budget_bytes;
  s->max_slots = max_slots;
  s->epoch_rounds = epoch_rounds;
  int rc = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) == cudaSuccess ? FTGCR_OK : FTGCR_ERR_CUDA;
  for (int t = 0; t < 2 && !rc; ++t) {
    rc = table_create(t == 1 ? FTGCR_MIXED : FTGCR_FP64, max_slots, &s->tables[t]);
    s->slot_req[t].assign(max_slots, nullptr);
  }
  if (rc) {
    for (SlotTable* t : s->tables) table_destroy(t);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
    return rc;
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return FTGCR_OK;
}

int ftgcr_server_submit(ftgcr_server* srv, const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol,
                        const double* rhs, double* x, const ftgcr_fault_plan* plan, int64_t* ticket) {
  if (!srv || !grid || !coeffs || !coeffs->D || !rhs || !x || !ticket) return FTGCR_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol)) return FTGCR_ERR_ARG;
  const int64_t fp = ftgcr_footprint(grid, k);
  if (fp < 0) return FTGCR_ERR_ARG;
  const long long N = (long long)grid->nlon * grid->nlat;
  Request* r = new Request();
  if (plan && plan->nlosses) {
    if (plan->nlosses < 0 || plan->nlosses > FTGCR_MAX_LOSSES || !plan->losses) {
      delete r;
      return FTGCR_ERR_ARG;
    }
    for (int q = 0; q < plan->nlosses; ++q) {
      const ftgcr_loss& l = plan->losses[q];
      if (l.step < 1 || l.nranks < 1 || l.rank < 0 || l.rank >= l.nranks || l.count < 0) {
        delete r;
        return FTGCR_ERR_ARG;
      }
    }
    r->losses.assign(plan->losses, plan->losses + plan->nlosses);
  }
  if (plan && plan->n) {
    if (plan->n < 0 || plan->n > FTGCR_MAX_FAULTS || !plan->faults) {
      delete r;
      return FTGCR_ERR_ARG;
    }
    const int maxbit = grid->precision == FTGCR_MIXED ? 31 : 63;
    for (int q = 0; q < plan->n; ++q) {
      const ftgcr_fault& f = plan->faults[q];
      if (f.vec < 0 || f.vec > FTGCR_VEC_E || f.index < 0 || f.index >= N || f.bit < 0 || f.bit > maxbit ||
          f.step < 1) {
        delete r;
        return FTGCR_ERR_ARG;
      }
    }
    r->faults.assign(plan->faults, plan->faults + plan->n);
  }
  r->key.grid = *grid;
  r->key.k = k;
  r->key.tol = tol;
  r->D = coeffs->D;
  r->ckey = coeffs->key;
  r->rhs = rhs;
  r->x = x;
  r->footprint = fp;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (fp > srv->budget) {
    delete r;
    return FTGCR_ERR_BUDGET;
  }
  if (srv->stop) {
    delete r;
    return FTGCR_ERR_STATE;
  }
  r->ticket = srv->next_ticket++;
  srv->reqs[r->ticket] = r;
  srv->queue.push_back(r);
  ++srv->submitted;
  *ticket = r->ticket;
  srv->cv_work.notify_one();
  return FTGCR_OK;
}

static int take_result(ftgcr_server* srv, std::unordered_map<int64_t, Request*>::iterator it, ftgcr_stats_t* stats) {
  Request* r = it->second;
  if (stats) *stats = r->stats;
  const int status = r->status;
  auto f = std::find(srv->finished.begin(), srv->finished.end(), r->ticket);
  if (f != srv->finished.end()) srv->finished.erase(f);
  srv->reqs.erase(it);
  delete r;
  return status;
}

int ftgcr_server_poll(ftgcr_server* srv, int64_t ticket, ftgcr_stats_t* stats) {
  if (!srv) return FTGCR_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return FTGCR_ERR_ARG;
  if (!it->second->done) return FTGCR_PENDING;
  return take_result(srv, it, stats);
}

int ftgcr_server_wait(ftgcr_server* srv, int64_t ticket, double timeout_s, ftgcr_stats_t* stats) {
  if (!srv) return FTGCR_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return FTGCR_ERR_ARG;
  Request* r = it->second;
  if (timeout_s < 0) {
    srv->cv_done.wait(lk, [&] { return r->done; });
  } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; })) {
    return FTGCR_PENDING;
  }
  return take_result(srv, srv->reqs.find(ticket), stats);
}

int ftgcr_server_next(ftgcr_server* srv, double timeout_s, int64_t* ticket, ftgcr_stats_t* stats) {
  if (!srv || !ticket) return FTGCR_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto ready = [&] { return !srv->finished.empty(); };
  if (timeout_s < 0) {
    if (srv->reqs.empty()) return FTGCR_ERR_STATE;  // nothing would ever finish
    srv->cv_done.wait(lk, [&] { return ready() || srv->reqs.empty(); });
    if (!ready()) return FTGCR_ERR_STATE;
  } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return FTGCR_PENDING;
  }
  *ticket = srv->finished.front();
  return take_result(srv, srv->reqs.find(*ticket), stats);
}

int ftgcr_server_info(ftgcr_server* srv, ftgcr_server_info_t* out) {
  if (!srv || !out) return FTGCR_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->queued = (int64_t)srv->queue.size();
  out->running = srv->running;
  out->epochs = srv->epochs;
  out->handles = (int64_t)srv->pool.size();
  out->bytes_in_use = srv->in_use;
  out->budget_bytes = srv->budget;
  return FTGCR_OK;
}

int ftgcr_server_destroy(ftgcr_server* srv) {
  if (!srv) return FTGCR_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (Request* r : srv->queue) {  // never started
      r->status = FTGCR_ERR_STATE;
      r->done = true;
    }
    srv->queue.clear();
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();  // running solves finish first
  for (PoolEntry& e : srv->pool)
    if (e.h) ftgcr_destroy(e.h);
  for (SlotTable* t : srv->tables) table_destroy(t);
  if (srv->st) cudaStreamDestroy(srv->st);
  for (auto& kv : srv->reqs) delete kv.second;
  delete srv;
  return FTGCR_OK;
}

}  // extern "C"
