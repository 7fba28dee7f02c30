// Request scheduler of libftgcr: continuous batching of independent FT-GCR(k)
// solves (Algorithm 1) over resumable persistent launches.
//
// One scheduler thread per server owns the launch stream, two slot tables
// (FP64 and mixed precision: a launch runs one precision) and a pool of solver
// handles.  A request passes through three queues:
//   queued  -> a handle is bound to it, first come first served, within the
//              device-memory budget: an idle handle already set up from the
//              request's coefficients (same D and key) is ready at once;
//              otherwise a new handle is made while the budget allows, else
//              an idle handle of the shape is rebuilt, else idle handles are
//              evicted, least recently used first;
//   prep    -> a second thread creates or rebuilds the handle on its own
//              stream (and destroys evicted ones), so set-up never stalls the
//              launches of the solves already running;
//   ready   -> in ticket order into free slots of its precision.
// The scheduler repeats an epoch: admit ready requests, stage their host
// inputs on a copy stream and begin them behind the running launch, collect
// that launch, start the next one for at most `epoch_rounds` rounds, and hand
// back the finished solves (host solutions copied out on the copy stream
// while the next launch runs).  A request made ready in epoch e joins epoch
// e + 1's launch.  Each solve's arithmetic depends only on its own handle, so
// a served result is bitwise the result of the same solve run alone.
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
  ftgcr_handle* h = nullptr;  // created by the preparation thread on first use
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

bool same_coeffs(const PoolEntry& e, const Request* r) { return r->ckey && e.setup_key == r->ckey && e.setup_D == r->D; }

int64_t points(const Request* r) { return (int64_t)r->key.grid.nlon * r->key.grid.nlat; }

}  // namespace

struct ftgcr_server {
  int dev = 0;
  cudaStream_t st = nullptr;   // persistent launches, begin kernels
  cudaStream_t cst = nullptr;  // staging copies of host arrays, both ways
  cudaStream_t pst = nullptr;  // coefficient rebuilds (preparation thread)
  cudaEvent_t staged = nullptr;
  int64_t budget = 0, in_use = 0;
  int max_slots = 0, epoch_rounds = 0;
  int64_t max_points = 0;            // grid points running at once per table (0: no limit)
  int64_t run_points[2] = {0, 0};
  SlotTable* tables[2] = {nullptr, nullptr};
  std::vector<Request*> slot_req[2];
  std::list<PoolEntry> pool;
  std::deque<Request*> queue;     // submitted, no handle yet (arrival order)
  std::deque<Request*> prep;      // handle being created or rebuilt
  std::deque<Request*> ready;     // handle set up, waiting for a slot (ticket order)
  std::vector<ftgcr_handle*> doomed;  // evicted handles, destroyed by the preparation thread
  std::deque<int64_t> finished;  // tickets in order of completion, not yet collected
  std::unordered_map<int64_t, Request*> reqs;
  int64_t next_ticket = 1;
  uint64_t tick = 0;
  int64_t submitted = 0, completed = 0, running = 0, epochs = 0;
  int preparing = 0;  // requests taken by the preparation thread, not yet ready
  bool blocked = false;  // the queue's head waits for memory held by running or preparing solves
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_prep;
  std::thread worker, preparer;

  // ---- under mu
  int free_slot(int t) const {
    for (int s = 0; s < max_slots; ++s)
      if (!slot_req[t][s]) return s;
    return -1;
  }
  // An idle handle of the request's shape: with `same`, only one already set
  // up from the request's coefficients.
  PoolEntry* idle_entry(const Request* r, bool same) {
    for (PoolEntry& e : pool) {
      if (e.busy || !e.h || !(e.key == r->key)) continue;
      if (!same || same_coeffs(e, r)) return &e;
    }
    return nullptr;
  }
  // Evict idle handles (least recently used first) until `need` more bytes
  // fit; the preparation thread destroys the evicted handles.
  bool make_room(int64_t need) {
    while (in_use + need > budget) {
      auto best = pool.end();
      for (auto it = pool.begin(); it != pool.end(); ++it)
        if (!it->busy && (best == pool.end() || it->last_used < best->last_used)) best = it;
      if (best == pool.end()) return false;
      in_use -= best->bytes;
      if (best->h) doomed.push_back(best->h);
      pool.erase(best);
    }
    return true;
  }
  PoolEntry* new_entry(const Request* r) {
    pool.emplace_back();
    PoolEntry* e = &pool.back();
    e->key = r->key;
    e->bytes = r->footprint;
    in_use += r->footprint;
    return e;
  }
  void to_ready(Request* r) {
    auto it = ready.begin();
    while (it != ready.end() && (*it)->ticket < r->ticket) ++it;
    ready.insert(it, r);
  }
  // Give queued requests handles, first come first served, at most
  // max_slots of them waiting for a slot or in preparation.  A request whose
  // coefficients an idle handle already holds is ready at once.  Otherwise a
  // new handle is made while the budget allows (so the pool grows towards a
  // handle per coefficient set in use), else an idle handle of the shape is
  // rebuilt, else idle handles are evicted; preparation runs on its own
  // thread and stream, so it never holds up a launch.
  void bind() {
    while (!queue.empty() && !stop && (int)(ready.size() + preparing) < max_slots) {
      Request* r = queue.front();
      PoolEntry* e = idle_entry(r, true);
      bool setup = false;
      if (!e) {
        setup = true;
        PoolEntry* any = idle_entry(r, false);
        if (any && (!r->ckey || in_use + r->footprint > budget)) {
          e = any;  // rebuilt from the request's coefficients
        } else {
          if (!make_room(r->footprint)) {  // wait for running solves to free memory
            blocked = true;
            break;
          }
          e = new_entry(r);
        }
      }
      e->busy = true;
      r->entry = e;
      queue.pop_front();
      if (setup) {
        prep.push_back(r);
        ++preparing;
      } else {
        to_ready(r);
      }
    }
    if (!prep.empty() || !doomed.empty()) cv_prep.notify_one();
  }
  // Ready requests into free slots, in ticket order.  With max_points, a
  // table takes no request past the first that would push its running grid
  // points over the limit (a request alone in its table always runs).
  void admit(std::vector<Request*>& adm) {
    bool held[2] = {false, false};
    for (auto it = ready.begin(); it != ready.end() && !stop;) {
      Request* r = *it;
      const int t = table_of(r->key.grid.precision);
      const int slot = held[t] ? -1 : free_slot(t);
      if (slot >= 0 && max_points > 0 && run_points[t] > 0 && run_points[t] + points(r) > max_points) {
        held[t] = true;
        ++it;
        continue;
      }
      if (slot < 0) {
        ++it;
        continue;
      }
      run_points[t] += points(r);
      r->table = t;
      r->slot = slot;
      slot_req[t][slot] = r;
      it = ready.erase(it);
      ++running;
      adm.push_back(r);
    }
  }
  void release_entry(Request* r) {
    if (!r->entry) return;
    blocked = false;
    r->entry->busy = false;
    r->entry->last_used = ++tick;
    if (!r->entry->h) {  // creation failed or never ran: drop the reservation
      in_use -= r->entry->bytes;
      for (auto it = pool.begin(); it != pool.end(); ++it)
        if (&*it == r->entry) {
          pool.erase(it);
          break;
        }
    }
    r->entry = nullptr;
  }
  void free_slot_of(Request* r) {
    slot_req[r->table][r->slot] = nullptr;
    run_points[r->table] -= points(r);
    r->slot = -1;
    --running;
  }
  void finish_locked(Request* r, int status) {
    const bool was_running = r->slot >= 0;
    if (was_running) free_slot_of(r);
    release_entry(r);
    r->status = status;
    r->done = true;
    finished.push_back(r->ticket);
    ++completed;
  }

  // ---- preparation thread: handle creation, coefficient rebuilds, eviction
  void prepare_loop() {
    cudaSetDevice(dev);
    for (;;) {
      Request* r = nullptr;
      std::vector<ftgcr_handle*> kill;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_prep.wait(lk, [&] { return stop || !prep.empty() || !doomed.empty(); });
        kill.swap(doomed);
        if (!prep.empty() && !stop) {
          r = prep.front();
          prep.pop_front();
        }
        if (!r && kill.empty()) {
          if (stop) break;
          continue;
        }
      }
      for (ftgcr_handle* h : kill) ftgcr_destroy(h);
      if (!r) continue;
      PoolEntry* e = r->entry;
      ftgcr_coeffs co{r->D, r->ckey};
      int rc = FTGCR_OK;
      if (!e->h) {
        ftgcr_handle* h = nullptr;
        rc = ftgcr_create(&r->key.grid, &co, r->key.k, r->key.tol, &h);
        if (!rc) {
          std::lock_guard<std::mutex> lk(mu);
          e->h = h;
        }
      } else {
        rc = ftgcr_set_coeffs(e->h, &co, pst);
        if (!rc && cudaStreamSynchronize(pst) != cudaSuccess) rc = FTGCR_ERR_CUDA;
      }
      std::lock_guard<std::mutex> lk(mu);
      --preparing;
      if (rc) {
        e->setup_key = 0;
        e->setup_D = nullptr;
        finish_locked(r, rc);
        cv_done.notify_all();
      } else {
        e->setup_D = r->D;
        e->setup_key = r->ckey;
        to_ready(r);
      }
      cv_work.notify_one();
    }
  }

  // ---- scheduler thread, outside the lock
  // Stage host arrays (copy stream) for a request whose handle is set up.
  int stage(Request* r, const double** R, double** X, int* check) {
    ftgcr_handle* h = r->entry->h;
    const long long N = handle_points(h);
    *R = r->rhs;
    *X = r->x;
    cudaPointerAttributes at;
    const bool rdev = cudaPointerGetAttributes(&at, *R) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    const bool xdev = cudaPointerGetAttributes(&at, *X) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    // host arrays are staged and checked for finite values on the device
    if (!rdev) {
      if (cudaMemcpyAsync(handle_stage_rhs(h), *R, sizeof(double) * N, cudaMemcpyHostToDevice, cst) != cudaSuccess)
        return FTGCR_ERR_CUDA;
      *R = handle_stage_rhs(h);
    }
    // FTGCR_FLAG_ZERO_GUESS: x is output only (its staging buffer zeroed, not
    // copied in nor checked)
    const bool zg = (r->key.grid.flags & FTGCR_FLAG_ZERO_GUESS) != 0;
    if (!xdev) {
      const cudaError_t e = zg ? cudaMemsetAsync(handle_stage_x(h), 0, sizeof(double) * N, cst)
                               : cudaMemcpyAsync(handle_stage_x(h), *X, sizeof(double) * N, cudaMemcpyHostToDevice, cst);
      if (e != cudaSuccess) return FTGCR_ERR_CUDA;
      *X = handle_stage_x(h);
    }
    r->x_host = !xdev;
    *check = (rdev ? 0 : 1) | (xdev || zg ? 0 : 2);
    return FTGCR_OK;
  }
  // Stage every admitted request on the copy stream, make the launch stream
  // wait for the copies, then begin each solve in its slot.
  void start_all(const std::vector<Request*>& adm) {
    std::vector<int> rc(adm.size()), check(adm.size());
    std::vector<const double*> R(adm.size());
    std::vector<double*> X(adm.size());
    for (size_t i = 0; i < adm.size(); ++i) rc[i] = stage(adm[i], &R[i], &X[i], &check[i]);
    if (!adm.empty() && (cudaEventRecord(staged, cst) != cudaSuccess || cudaStreamWaitEvent(st, staged, 0) != cudaSuccess))
      for (int& c : rc)
        if (!c) c = FTGCR_ERR_CUDA;
    for (size_t i = 0; i < adm.size(); ++i) {
      Request* r = adm[i];
      if (!rc[i]) {
        ftgcr_fault_plan plan{r->faults.data(), (int32_t)r->faults.size(), r->losses.data(),
                              (int32_t)r->losses.size()};
        const bool any = !r->faults.empty() || !r->losses.empty();
        rc[i] = table_begin(tables[r->table], r->slot, r->entry->h, R[i], X[i], any ? &plan : nullptr, st, check[i]);
      }
      if (rc[i]) {  // table_begin failed or never ran: the slot is still free
        std::lock_guard<std::mutex> lk(mu);
        finish_locked(r, rc[i]);
        cv_done.notify_all();
      }
    }
  }
  // Statistics of a finished solve (its launch has completed); a host
  // solution is copied out on the copy stream, overlapping the next launch.
  bool take_stats(Request* r, int* status) {
    ftgcr_handle* h = r->entry->h;
    ftgcr_stats_t s{};
    const int rc = ftgcr_stats(h, &s);
    r->stats = s;
    *status = rc ? rc : s.status;
    if (!r->x_host) return false;
    if (cudaMemcpyAsync(r->x, handle_stage_x(h), sizeof(double) * handle_points(h), cudaMemcpyDeviceToHost, cst) !=
        cudaSuccess && !*status)
      *status = FTGCR_ERR_CUDA;
    return true;
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

  // Collect the launches in flight.  Solves whose solution stays on the
  // device are handed back at once; the others go to `out` with their
  // status, to be handed back once their copy has landed.
  void collect(bool* inflight, std::vector<int>& fin, std::vector<std::pair<Request*, int>>& out) {
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
      bool any = false;
      for (Request* r : done) {
        int status = FTGCR_OK;
        if (take_stats(r, &status)) {
          std::lock_guard<std::mutex> lk(mu);  // the slot is free; the handle stays busy until the copy lands
          free_slot_of(r);
          out.emplace_back(r, status);
        } else {
          std::lock_guard<std::mutex> lk(mu);
          finish_locked(r, status);
          any = true;
        }
      }
      if (any) cv_done.notify_all();
    }
  }
  void hand_back(std::vector<std::pair<Request*, int>>& out) {
    if (out.empty()) return;
    const bool ok = cudaStreamSynchronize(cst) == cudaSuccess;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& ro : out) finish_locked(ro.first, ok ? ro.second : (ro.second ? ro.second : FTGCR_ERR_CUDA));
    out.clear();
    cv_done.notify_all();
  }

  // One epoch per iteration, pipelined: while launch e runs on the GPU the
  // thread binds handles, admits ready requests and stages them (copies on
  // the copy stream, begin kernels queued behind launch e), then collects
  // launch e, enqueues launch e + 1, which the staged requests join, and
  // hands back launch e's host solutions while e + 1 runs.
  void loop() {
    cudaSetDevice(dev);
    std::vector<int> fin(max_slots);
    std::vector<std::pair<Request*, int>> out;
    bool inflight[2] = {false, false};
    for (;;) {
      std::vector<Request*> adm;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (!inflight[0] && !inflight[1])
          cv_work.wait(lk, [&] {
            return stop || running > 0 || !ready.empty() ||
                   (!queue.empty() && !blocked && (int)(ready.size() + preparing) < max_slots);
          });
        if (stop && running == 0) break;
        bind();
        admit(adm);
      }
      start_all(adm);
      collect(inflight, fin, out);
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
      hand_back(out);
    }
    hand_back(out);
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
  int rc = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaStreamCreateWithFlags(&s->pst, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&s->staged, cudaEventDisableTiming) == cudaSuccess
               ? FTGCR_OK
               : FTGCR_ERR_CUDA;
  for (int t = 0; t < 2 && !rc; ++t) {
    rc = table_create(t == 1 ? FTGCR_MIXED : FTGCR_FP64, max_slots, &s->tables[t]);
    s->slot_req[t].assign(max_slots, nullptr);
  }
  if (rc) {
    for (SlotTable* t : s->tables) table_destroy(t);
    for (cudaStream_t q : {s->st, s->cst, s->pst})
      if (q) cudaStreamDestroy(q);
    if (s->staged) cudaEventDestroy(s->staged);
    delete s;
    return rc;
  }
  s->worker = std::thread([s] { s->loop(); });
  s->preparer = std::thread([s] { s->prepare_loop(); });
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

int ftgcr_server_set_max_points(ftgcr_server* srv, int64_t max_points) {
  if (!srv || max_points < 0) return FTGCR_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->max_points = max_points;
  srv->cv_work.notify_one();
  return FTGCR_OK;
}

int ftgcr_server_info(ftgcr_server* srv, ftgcr_server_info_t* out) {
  if (!srv || !out) return FTGCR_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->queued = (int64_t)(srv->queue.size() + srv->ready.size()) + srv->preparing;
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
    srv->cv_prep.notify_all();
    srv->cv_done.notify_all();
  }
  if (srv->preparer.joinable()) srv->preparer.join();  // ends after the preparation in progress
  if (srv->worker.joinable()) srv->worker.join();      // running solves finish first
  for (Request* r : srv->prep) r->done = true, r->status = FTGCR_ERR_STATE;  // never started
  for (Request* r : srv->ready) r->done = true, r->status = FTGCR_ERR_STATE;
  for (ftgcr_handle* h : srv->doomed) ftgcr_destroy(h);
  for (PoolEntry& e : srv->pool)
    if (e.h) ftgcr_destroy(e.h);
  for (SlotTable* t : srv->tables) table_destroy(t);
  for (cudaStream_t q : {srv->st, srv->cst, srv->pst})
    if (q) cudaStreamDestroy(q);
  if (srv->staged) cudaEventDestroy(srv->staged);
  for (auto& kv : srv->reqs) delete kv.second;
  delete srv;
  return FTGCR_OK;
}

}  // extern "C"
