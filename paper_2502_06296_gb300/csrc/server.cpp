// server.cpp -- a serving loop for Poisson and Helmholtz solve requests from
// many concurrently running channel simulations ("runs").
//
// Each run is one grid.  Its plan (tables, factors, Algorithm 2 sets, FP32
// work field) stays resident in HBM while memory allows: a plan is created
// when a request first needs it and the plans of idle runs are destroyed,
// least recently used first, when a new plan would exceed the memory budget.
// Worker threads, each with its own CUDA stream and one reusable group,
// practise continuous batching: a free worker takes the oldest pending
// request, adds every other pending request of the same kind whose run is
// idle (at most one per run, up to the batch limit), and solves the batch as
// one grouped refined solve.  Requests that arrive while batches run wait in
// the queue and join the next batch a worker forms; batches of different
// workers overlap on the device.  A request's result is bit-identical to the
// refined solve of its run's plan alone (the grouped solve guarantees it).
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
  int run, kind, loc;
  double c;
  const double* rhs;
  double* out;
  double t_submit = 0, t_done = 0;
  int status = 0;
  bool done = false;
};

struct Run {
  int nx, ny, nz, bc;
  double lx, ly;
  std::vector<double> dz;
  cfs_plan_t plan = nullptr;
  size_t bytes = 0;  // device bytes of the plan (estimate until created)
  bool busy = false;
  unsigned long long last_used = 0;
};

// Device bytes of a refined plan of this size: FP64 and FP32 factors of
// every (kx, ky) system, the two FP32 and the FP64 work fields, and a margin
// for the tables.
size_t plan_estimate(int nx, int ny, int nz) {
  const size_t cols = (size_t)(nx / 2 + 1) * (ny / 2 + 1);
  return cols * nz * (24 + 12) + (size_t)nx * ny * nz * (4 + 4 + 8) + (size_t)(1u << 20);
}

}  // namespace

struct cfs_server {
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<Request*> pending;
  std::unordered_map<unsigned long long, Request*> requests;
  std::deque<Run> runs;  // a deque: references stay valid as runs are added
  size_t budget = 0, used = 0;
  int max_batch = 1, device = 0, autotune = 0;
  bool stop = false;
  unsigned long long next_id = 1, clock = 0;
  std::vector<std::thread> workers;
  cfs_server_stats_t stats{};
};

// Picks a batch under the lock: the oldest pending request, then every later
// one of the same kind whose run is idle and not yet in the batch.  Memory for
// plans that must be created is reserved (evicting idle plans, least recently
// used first); requests whose plan does not fit stay pending.
static void take_batch(cfs_server* S, std::vector<Request*>* batch,
                       std::vector<cfs_plan_t>* evict) {
  batch->clear();
  // the kind of the oldest request whose run is idle
  int kind = -1;
  for (const Request* r : S->pending)
    if (!S->runs[r->run].busy) {
      kind = r->kind;
      break;
    }
  if (kind < 0) return;
  std::vector<char> in_batch(S->runs.size(), 0);
  for (auto it = S->pending.begin();
       it != S->pending.end() && (int)batch->size() < S->max_batch;) {
    Request* r = *it;
    Run& run = S->runs[r->run];
    if (r->kind != kind || run.busy || in_batch[r->run]) {
      ++it;
      continue;
    }
    if (!run.plan) {
      const size_t need = plan_estimate(run.nx, run.ny, run.nz);
      while (S->used + need > S->budget) {  // evict the least recently used idle plan
        int victim = -1;
        for (size_t q = 0; q < S->runs.size(); ++q) {
          const Run& o = S->runs[q];
          if (o.plan && !o.busy && !in_batch[q] &&
              (victim < 0 || o.last_used < S->runs[victim].last_used))
            victim = (int)q;
        }
        if (victim < 0) break;
        evict->push_back(S->runs[victim].plan);
        S->used -= S->runs[victim].bytes;
        S->runs[victim].plan = nullptr;
        S->runs[victim].bytes = 0;
        S->stats.plans_evicted++;
      }
      if (S->used + need > S->budget) {
        ++it;
        continue;
      }
      S->used += need;
      run.bytes = need;
    }
    in_batch[r->run] = 1;
    run.busy = true;
    batch->push_back(r);
    it = S->pending.erase(it);
  }
}

static void worker_main(cfs_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cfs_group_t group = nullptr;
  bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cfs_group_reserve(&group, S->max_batch) == CFS_OK;
  std::vector<Request*> batch;
  std::vector<cfs_plan_t> evict, plans;
  std::vector<const double*> in;
  std::vector<double*> out;
  std::vector<double> cs;
  std::vector<int> locs;
  for (;;) {
    {
      std::unique_lock<std::mutex> lock(S->mu);
      for (;;) {
        if (S->stop && S->pending.empty()) break;
        evict.clear();
        if (ok) take_batch(S, &batch, &evict);
        if (!batch.empty() || !evict.empty()) break;
        S->work_cv.wait(lock);
      }
      if (batch.empty() && evict.empty()) break;  // stopping, nothing left
    }
    for (cfs_plan_t p : evict) cfs_plan_destroy(p);
    if (batch.empty()) continue;
    // plans of runs that have none yet (memory already reserved)
    int rc = CFS_OK;
    plans.clear();
    for (Request* r : batch) {
      Run& run = S->runs[r->run];  // busy: only this worker touches it
      if (!run.plan) {
        int prc = cfs_plan_create(&run.plan, run.nx, run.ny, run.nz, run.lx, run.ly,
                                  run.dz.data(), run.bc, CFS_F32_REFINED);
        if (!prc && S->autotune) prc = cfs_plan_autotune(run.plan, st);
        size_t bytes = 0;
        if (!prc) cfs_plan_device_bytes(run.plan, &bytes);
        if (prc && run.plan) {
          cfs_plan_destroy(run.plan);
          run.plan = nullptr;
        }
        std::lock_guard<std::mutex> lock(S->mu);
        S->used = S->used - run.bytes + (prc ? 0 : bytes);
        run.bytes = prc ? 0 : bytes;
        if (prc) rc = prc;
        else S->stats.plans_created++;
      }
      plans.push_back(run.plan);
    }
    if (!rc) {
      in.clear();
      out.clear();
      cs.clear();
      locs.clear();
      for (Request* r : batch) {
        in.push_back(r->rhs);
        out.push_back(r->out);
        cs.push_back(r->c);
        locs.push_back(r->loc);
      }
      rc = cfs_group_rebind(group, (int)batch.size(), plans.data(), st);
      if (!rc) {
        if (batch[0]->kind == CFS_REQ_POISSON)
          rc = cfs_group_poisson_solve(group, in.data(), out.data(), st);
        else
          rc = cfs_group_helmholtz_solve(group, cs.data(), locs.data(), in.data(), out.data(), st);
      }
    }
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (Request* r : batch) {
        r->status = rc;
        r->t_done = t;
        r->done = true;
        Run& run = S->runs[r->run];
        run.busy = false;
        run.last_used = ++S->clock;
      }
      S->stats.completed += batch.size();
      S->stats.batches += 1;
      if (batch.size() > (size_t)S->stats.max_batch_seen) S->stats.max_batch_seen = (int)batch.size();
      if (rc) S->stats.failed += batch.size();
    }
    S->done_cv.notify_all();
    S->work_cv.notify_all();  // freed runs may complete other workers' batches
  }
  if (group) cfs_group_destroy(group);
  if (st) cudaStreamDestroy(st);
}

extern "C" int cfs_server_create(cfs_server_t* out, size_t hbm_budget_bytes, int workers,
                                 int max_batch, int autotune) {
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (workers < 1 || workers > 64 || max_batch < 1 || max_batch > chanfs::kMaxGroup ||
      hbm_budget_bytes == 0)
    return CFS_EINVAL;
  cfs_server* S = new (std::nothrow) cfs_server();
  if (!S) return CFS_ENOMEM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return CFS_ECUDA;
  }
  S->budget = hbm_budget_bytes;
  S->max_batch = max_batch;
  S->autotune = autotune;
  for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_main, S);
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
    S->pending.push_back(r);
    S->stats.submitted++;
    *ticket = r->id;
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

extern "C" int cfs_server_stats(cfs_server_t S, cfs_server_stats_t* out) {
  if (!S || !out) return CFS_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  out->bytes_in_use = S->used;
  int resident = 0;
  for (const Run& r : S->runs) resident += (r.plan != nullptr);
  out->plans_resident = resident;
  return CFS_OK;
}

extern "C" int cfs_server_destroy(cfs_server_t S) {
  if (!S) return CFS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->work_cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (Run& r : S->runs)
    if (r.plan) cfs_plan_destroy(r.plan);
  for (auto& kv : S->requests) delete kv.second;
  delete S;
  return CFS_OK;
}
