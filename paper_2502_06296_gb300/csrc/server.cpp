// server.cpp -- a serving loop for Poisson and Helmholtz solve requests from
// many concurrently running channel simulations ("runs").
//
// Each run is one grid with up to `slots` plans (tables, factors, Algorithm 2
// sets, FP32 work fields), so that as many requests of one run can be solved
// at once.  A plan stays resident in HBM while memory allows: it is created
// when a request first needs the slot, and idle plans are destroyed, least
// recently used first, when a new plan would exceed the memory budget.
// Worker threads, each with its own CUDA stream and one reusable group,
// practise continuous batching: a free worker takes the oldest pending
// request whose run has a free slot, adds every other pending request of the
// same kind for which a slot is free (up to the batch limit), and solves the
// batch as one grouped refined solve.  Requests that arrive while batches run
// wait in the queue and join the next batch a worker forms; batches of
// different workers overlap on the device.  A request's result is
// bit-identical to the refined solve of its run's plan alone (the grouped
// solve guarantees it, and every slot of a run computes the same).
//
// Failures are per request: a plan that cannot be created (the device
// allocation refused) fails the requests that needed it with that status and
// leaves the rest of the batch to be solved; a worker that cannot start
// (stream or group) leaves; a server with no worker fails at creation.  For
// tests, plan creations and worker start-ups can be made to fail on the host.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "chanfs_internal.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  unsigned long long id;
  int run, kind, loc, slot = -1;
  double c;
  const double* rhs;
  double* out;
  double t_submit = 0, t_done = 0;
  int status = 0;
  bool done = false;
};

struct Slot {
  cfs_plan_t plan = nullptr;
  size_t bytes = 0;  // device bytes of the plan (the estimate until created)
  bool busy = false;
  unsigned long long last_used = 0;
};

struct Run {
  int nx, ny, nz, bc;
  double lx, ly;
  std::vector<double> dz;
  std::vector<Slot> slots;
};

// Device bytes of a refined plan of this size: FP64 and FP32 factors of
// every (kx, ky) system, the two FP32 and the FP64 work fields, and a margin
// for the tables.
size_t plan_estimate(int nx, int ny, int nz) {
  const size_t cols = (size_t)(nx / 2 + 1) * (ny / 2 + 1);
  return cols * nz * (24 + 12) + (size_t)nx * ny * nz * (4 + 4 + 8) + (size_t)(1u << 20);
}

// Worker start-ups to refuse in the next servers created (test hook).
std::atomic<int> g_fail_worker_starts{0};

}  // namespace

struct cfs_server {
  std::mutex mu;
  std::condition_variable work_cv, done_cv, start_cv;
  std::deque<Request*> pending;
  std::unordered_map<unsigned long long, Request*> requests;
  std::deque<Run> runs;  // a deque: references stay valid as runs are added
  size_t budget = 0, used = 0;
  int max_batch = 1, slots = 1, device = 0, autotune = 0;
  int started = 0, alive = 0;
  int fail_plan_creates = 0;  // test hook: plan creations to refuse
  bool stop = false, paused = false;
  unsigned long long next_id = 1, clock = 0;
  std::vector<std::thread> workers;
  cfs_server_stats_t stats{};
};

// Slot of `run` a request can take now: an idle one with a plan (not in the
// batch), else an empty one.  -1 if none.
static int free_slot(const Run& run, const char* taken) {
  int empty = -1;
  for (size_t q = 0; q < run.slots.size(); ++q) {
    if (run.slots[q].busy || taken[q]) continue;
    if (run.slots[q].plan) return (int)q;
    if (empty < 0) empty = (int)q;
  }
  return empty;
}

// Picks a batch under the lock: the oldest pending request whose run has a
// free slot, then every later one of the same kind that finds a free slot.
// Memory for plans that must be created is reserved (evicting idle plans,
// least recently used first); requests whose plan does not fit stay pending.
static void take_batch(cfs_server* S, std::vector<Request*>* batch,
                       std::vector<cfs_plan_t>* evict) {
  batch->clear();
  if (S->paused) return;
  const size_t nslot = (size_t)S->slots;
  std::vector<char> taken(S->runs.size() * nslot, 0);  // slots already in the batch
  auto taken_of = [&](int run) { return taken.data() + (size_t)run * nslot; };
  int kind = -1;
  for (const Request* r : S->pending)
    if (free_slot(S->runs[r->run], taken_of(r->run)) >= 0) {
      kind = r->kind;
      break;
    }
  if (kind < 0) return;
  for (auto it = S->pending.begin();
       it != S->pending.end() && (int)batch->size() < S->max_batch;) {
    Request* r = *it;
    Run& run = S->runs[r->run];
    const int q = (r->kind == kind) ? free_slot(run, taken_of(r->run)) : -1;
    if (q < 0) {
      ++it;
      continue;
    }
    Slot& slot = run.slots[q];
    if (!slot.plan) {
      const size_t need = plan_estimate(run.nx, run.ny, run.nz);
      while (S->used + need > S->budget) {  // evict the least recently used idle plan
        Slot* victim = nullptr;
        for (size_t v = 0; v < S->runs.size(); ++v)
          for (size_t w = 0; w < nslot; ++w) {
            Slot& o = S->runs[v].slots[w];
            if (o.plan && !o.busy && !taken[v * nslot + w] &&
                (!victim || o.last_used < victim->last_used))
              victim = &o;
          }
        if (!victim) break;
        evict->push_back(victim->plan);
        S->used -= victim->bytes;
        victim->plan = nullptr;
        victim->bytes = 0;
        S->stats.plans_evicted++;
      }
      if (S->used + need > S->budget) {
        ++it;
        continue;
      }
      S->used += need;
      slot.bytes = need;
    }
    taken[r->run * nslot + q] = 1;
    slot.busy = true;
    r->slot = q;
    batch->push_back(r);
    it = S->pending.erase(it);
  }
}

// Every pending request fails with `status` (no worker is left to take it).
static void fail_pending(cfs_server* S, int status) {
  const double t = now_s();
  for (Request* r : S->pending) {
    r->status = status;
    r->t_done = t;
    r->done = true;
    S->stats.completed++;
    S->stats.failed++;
  }
  S->pending.clear();
}

static void worker_main(cfs_server* S) {
  cudaStream_t st = nullptr;
  cfs_group_t group = nullptr;
  bool ok = cudaSetDevice(S->device) == cudaSuccess;
  if (ok) {
    int left = g_fail_worker_starts.load();
    while (left > 0 && !g_fail_worker_starts.compare_exchange_weak(left, left - 1)) {
    }
    ok = left <= 0;  // a start-up refused by the test hook
  }
  ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
       cfs_group_reserve(&group, S->max_batch) == CFS_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->started++;
    if (ok) S->alive++;
  }
  S->start_cv.notify_all();
  if (!ok) {
    if (group) cfs_group_destroy(group);
    if (st) cudaStreamDestroy(st);
    return;
  }
  std::vector<Request*> batch, solve;
  std::vector<cfs_plan_t> evict, plans;
  std::vector<const double*> in;
  std::vector<double*> out;
  std::vector<double> cs;
  std::vector<int> locs;
  for (;;) {
    // nothing carried over from the last batch (a stopping server with an
    // empty queue leaves the loop below without taking a new one)
    batch.clear();
    evict.clear();
    {
      std::unique_lock<std::mutex> lock(S->mu);
      for (;;) {
        if (S->stop && S->pending.empty()) break;
        evict.clear();
        take_batch(S, &batch, &evict);
        if (!batch.empty() || !evict.empty()) break;
        S->work_cv.wait(lock);
      }
      if (batch.empty() && evict.empty()) break;  // stopping, nothing left
    }
    for (cfs_plan_t p : evict) cfs_plan_destroy(p);
    if (batch.empty()) continue;
    // plans of slots that have none yet (memory already reserved); a
    // request whose plan cannot be made fails alone
    solve.clear();
    plans.clear();
    for (Request* r : batch) {
      Run& run = S->runs[r->run];
      Slot& slot = run.slots[r->slot];  // busy: only this worker touches it
      if (!slot.plan) {
        int prc = CFS_OK;
        {
          std::lock_guard<std::mutex> lock(S->mu);
          if (S->fail_plan_creates > 0) {
            S->fail_plan_creates--;
            prc = CFS_ENOMEM;  // as if the device allocation was refused
          }
        }
        if (!prc)
          prc = cfs_plan_create(&slot.plan, run.nx, run.ny, run.nz, run.lx, run.ly,
                                run.dz.data(), run.bc, CFS_F32_REFINED);
        if (!prc && S->autotune) prc = cfs_plan_autotune(slot.plan, st);
        size_t bytes = 0;
        if (!prc) cfs_plan_device_bytes(slot.plan, &bytes);
        if (prc && slot.plan) {
          cfs_plan_destroy(slot.plan);
          slot.plan = nullptr;
        }
        std::lock_guard<std::mutex> lock(S->mu);
        S->used = S->used - slot.bytes + (prc ? 0 : bytes);
        slot.bytes = prc ? 0 : bytes;
        if (prc) r->status = prc;
        else S->stats.plans_created++;
      }
      if (slot.plan) {
        solve.push_back(r);
        plans.push_back(slot.plan);
      }
    }
    int rc = CFS_OK;
    if (!solve.empty()) {
      in.clear();
      out.clear();
      cs.clear();
      locs.clear();
      for (Request* r : solve) {
        in.push_back(r->rhs);
        out.push_back(r->out);
        cs.push_back(r->c);
        locs.push_back(r->loc);
      }
      rc = cfs_group_rebind(group, (int)solve.size(), plans.data(), st);
      if (!rc) {
        if (solve[0]->kind == CFS_REQ_POISSON)
          rc = cfs_group_poisson_solve(group, in.data(), out.data(), st);
        else
          rc = cfs_group_helmholtz_solve(group, cs.data(), locs.data(), in.data(), out.data(), st);
      }
      for (Request* r : solve) r->status = rc;
    }
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (Request* r : batch) {
        r->t_done = t;
        r->done = true;
        Slot& slot = S->runs[r->run].slots[r->slot];
        slot.busy = false;
        slot.last_used = ++S->clock;
        if (r->status) S->stats.failed++;
      }
      S->stats.completed += batch.size();
      S->stats.batches += 1;
      if (batch.size() > (size_t)S->stats.max_batch_seen) S->stats.max_batch_seen = (int)batch.size();
    }
    S->done_cv.notify_all();
    S->work_cv.notify_all();  // freed slots may complete other workers' batches
  }
  cfs_group_destroy(group);
  cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lock(S->mu);
  S->alive--;
}

extern "C" int cfs_server_create(cfs_server_t* out, size_t hbm_budget_bytes, int workers,
                                 int max_batch, int slots_per_run, int autotune) {
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (workers < 1 || workers > 64 || max_batch < 1 || max_batch > chanfs::kMaxGroup ||
      slots_per_run < 1 || slots_per_run > 16 || hbm_budget_bytes == 0)
    return CFS_EINVAL;
  cfs_server* S = new (std::nothrow) cfs_server();
  if (!S) return CFS_ENOMEM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return CFS_ECUDA;
  }
  S->budget = hbm_budget_bytes;
  S->max_batch = max_batch;
  S->slots = slots_per_run;
  S->autotune = autotune;
  for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_main, S);
  int alive = 0;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    S->start_cv.wait(lock, [&] { return S->started == workers; });
    alive = S->alive;
  }
  if (alive == 0) {  // no worker could start: nothing would ever be solved
    for (auto& t : S->workers) t.join();
    delete S;
    return CFS_ECUDA;
  }
  *out = S;
  return CFS_OK;
}

extern "C" int cfs_server_add_run(cfs_server_t S, int nx, int ny, int nz, double lx, double ly,
                                  const double* dz, int poisson_bc, int* run) {
  if (!S || !dz || !run || nx < 2 || ny < 1 || nz < 3) return CFS_EINVAL;
  if (nx % 4 || plan_estimate(nx, ny, nz) > S->budget) return CFS_EUNSUPPORTED;
  Run r;
  r.nx = nx;
  r.ny = ny;
  r.nz = nz;
  r.lx = lx;
  r.ly = ly;
  r.bc = poisson_bc;
  r.dz.assign(dz, dz + nz);
  std::lock_guard<std::mutex> lock(S->mu);
  r.slots.resize((size_t)S->slots);
  *run = (int)S->runs.size();
  S->runs.push_back(std::move(r));
  return CFS_OK;
}

extern "C" int cfs_server_submit(cfs_server_t S, int run, int kind, double c, int loc,
                                 const double* rhs, double* out, unsigned long long* ticket) {
  if (!S || !rhs || !out || !ticket || static_cast<const void*>(rhs) == out) return CFS_EINVAL;
  if (kind != CFS_REQ_POISSON && kind != CFS_REQ_HELMHOLTZ) return CFS_EINVAL;
  if (kind == CFS_REQ_HELMHOLTZ &&
      (!(c >= 0) || !std::isfinite(c) || (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE)))
    return CFS_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return CFS_ENOMEM;
  r->kind = kind;
  r->c = c;
  r->loc = loc;
  r->rhs = rhs;
  r->out = out;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (run < 0 || run >= (int)S->runs.size() || S->stop) {
      delete r;
      return CFS_EINVAL;
    }
    r->run = run;
    r->id = S->next_id++;
    r->t_submit = now_s();
    S->requests[r->id] = r;
    S->stats.submitted++;
    *ticket = r->id;
    if (S->alive == 0) {  // every worker has left: fail at once
      r->status = CFS_ECUDA;
      r->t_done = r->t_submit;
      r->done = true;
      S->stats.completed++;
      S->stats.failed++;
      return CFS_OK;
    }
    S->pending.push_back(r);
  }
  S->work_cv.notify_one();
  return CFS_OK;
}

extern "C" int cfs_server_wait(cfs_server_t S, unsigned long long ticket, double timeout_s,
                               int* status, double* latency_s) {
  if (!S) return CFS_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->requests.find(ticket);
  if (it == S->requests.end()) return CFS_EINVAL;
  Request* r = it->second;
  const auto deadline =
      std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s);
  while (!r->done) {
    if (S->done_cv.wait_until(lock, deadline) == std::cv_status::timeout && !r->done)
      return CFS_ETIMEOUT;
  }
  if (status) *status = r->status;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  S->requests.erase(it);
  delete r;
  return CFS_OK;
}

extern "C" int cfs_server_cancel(cfs_server_t S, unsigned long long ticket) {
  if (!S) return CFS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return CFS_EINVAL;
    Request* r = it->second;
    bool found = false;
    for (auto p = S->pending.begin(); p != S->pending.end(); ++p)
      if (*p == r) {
        S->pending.erase(p);
        found = true;
        break;
      }
    if (!found) return CFS_EINVAL;  // already taken by a worker, or done
    r->status = CFS_ECANCELED;
    r->t_done = now_s();
    r->done = true;
    S->stats.completed++;
    S->stats.cancelled++;
  }
  S->done_cv.notify_all();
  return CFS_OK;
}

extern "C" int cfs_server_pause(cfs_server_t S, int paused) {
  if (!S) return CFS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->paused = paused != 0;
  }
  S->work_cv.notify_all();
  return CFS_OK;
}

extern "C" int cfs_server_inject_fault(cfs_server_t S, int fault, int count) {
  if (count < 0) return CFS_EINVAL;
  if (fault == CFS_FAULT_WORKER_START) {
    if (S) return CFS_EINVAL;
    g_fail_worker_starts.store(count);
    return CFS_OK;
  }
  if (fault != CFS_FAULT_PLAN_ALLOC || !S) return CFS_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  S->fail_plan_creates = count;
  return CFS_OK;
}

extern "C" int cfs_server_stats(cfs_server_t S, cfs_server_stats_t* out) {
  if (!S || !out) return CFS_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  out->bytes_in_use = S->used;
  int resident = 0;
  for (const Run& r : S->runs)
    for (const Slot& s : r.slots) resident += (s.plan != nullptr);
  out->plans_resident = resident;
  out->workers_alive = S->alive;
  out->pending = (int)S->pending.size();
  return CFS_OK;
}

extern "C" int cfs_server_destroy(cfs_server_t S) {
  if (!S) return CFS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
    S->paused = false;  // the pending requests are finished first
    if (S->alive == 0) fail_pending(S, CFS_ECUDA);
  }
  S->work_cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (Run& r : S->runs)
    for (Slot& s : r.slots)
      if (s.plan) cfs_plan_destroy(s.plan);
  for (auto& kv : S->requests) delete kv.second;
  delete S;
  return CFS_OK;
}
