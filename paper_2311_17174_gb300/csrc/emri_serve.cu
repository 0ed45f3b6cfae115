// emri_serve.cu -- continuous-batching request loop, multi-chain launches
// and the autotuner of libemri.
//
// Serving: a scheduler thread owns S stream slots and one device pool, the
// serving budget allocated once at start.  Requests (a dataset and W
// walkers) wait in arrival order; a request is admitted when a slot is free
// and a contiguous range of the pool holds everything it needs on the device
// (parameters, results, and the likelihood path's workspace), so admission
// and allocation are one decision and no request admitted can run out of
// memory.  A request that does not fit yet keeps its place while later ones
// that fit pass it, at most kMaxBypass times; then admission waits for it
// (the ranges of running requests return to the pool as they complete, so it
// is admitted at the latest when the device drains).  On admission its
// parameters go host->device from the slot's pinned staging buffer, the
// likelihood path is enqueued on the slot's stream and the results come back
// device->host into pinned memory, all asynchronously.  Requests in different
// slots overlap on the device; completion is detected by polling an event per
// slot.  The scheduler never allocates or frees device memory.  The kernels
// reduce in a fixed order per walker, so a request's results are bitwise the
// same alone or in a mix.
#include <math.h>
#include <time.h>

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/emri.h"
#include "emri_api_internal.h"
#include "emri_common.cuh"

using namespace emri;

namespace emri {

static int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

// Admission may pass a request that does not fit yet at most this many times.
constexpr int kMaxBypass = 32;
// Pinned staging per slot at start (walkers); grows when a request is larger.
constexpr int kStageWalkers = 1024;

struct Request {
  uint64_t ticket = 0;
  const emri_dataset* ds = nullptr;
  std::vector<double> theta;   // [16][w]
  int w = 0;
  OptsN o{};
  bool fd = false;             // frequency-dependent propagation (paper Sec. 2)
  int qm = 0, qt = 0;
  double fstar = 1.0;
  std::vector<double> coef;    // [qm + qt][w]
  size_t need = 0;             // pool bytes: parameters and results, then the workspace
  size_t off = 0;              // its range of the pool while it runs
  int bypassed = 0;            // later requests admitted while this one waited
  int wave = 0;
  std::vector<double> lnl;
  std::vector<uint32_t> st;
  emri_req_stats stats{};
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double* h_theta = nullptr;   // pinned staging
  double* h_lnl = nullptr;
  uint32_t* h_st = nullptr;
  size_t h_cap = 0;            // walkers
  std::vector<void*> retired;  // outgrown staging, freed at stop
  std::shared_ptr<Request> req;
};

struct Server {
  emri_ctx* ctx = nullptr;
  emri_serve_cfg cfg{};
  size_t budget = 0;           // pool bytes
  char* pool = nullptr;
  std::map<size_t, size_t> free_ranges;   // offset -> bytes, coalesced
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<Slot> slots;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  int64_t launches = 0;
};

// ------------------------------------------------------------ the pool
// First fit over the free ranges (every size is a multiple of 256 bytes).
static bool pool_take(Server* sv, size_t bytes, size_t* off) {
  for (auto it = sv->free_ranges.begin(); it != sv->free_ranges.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const size_t rest = it->second - bytes, next = it->first + bytes;
    sv->free_ranges.erase(it);
    if (rest) sv->free_ranges[next] = rest;
    return true;
  }
  return false;
}

// Return a range, merged with its free neighbours.
static void pool_give(Server* sv, size_t off, size_t bytes) {
  auto it = sv->free_ranges.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != sv->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    sv->free_ranges.erase(nx);
  }
  if (it != sv->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      sv->free_ranges.erase(it);
    }
  }
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Most frequency-dependent coefficients per walker (q_m + q_t <= 6).
constexpr int kMaxCoef = 6;

// Pool bytes of a request: parameters, lnL and status (and the propagation
// coefficients and records when fd), then the workspace of the likelihood
// path.
static size_t request_bytes(const emri_dataset* ds, const OptsN& o, int w, int wave, bool fd, int ncoef) {
  return round256(sizeof(double) * (kNParam + 2 + (size_t)ncoef) * (size_t)w) +
         (fd ? round256(sizeof(FdW) * (size_t)w) : 0) + round256(loglike_layout(ds->plan, o, w, wave, nullptr, nullptr));
}

// Pinned staging for w walkers (host memory only; outgrown buffers are kept
// until stop, so nothing here waits for the device).
static int slot_staging(Slot& sl, int w) {
  if ((size_t)w <= sl.h_cap) return EMRI_OK;
  const size_t cap = std::max<size_t>((size_t)w, 2 * sl.h_cap);
  double *t = nullptr, *l = nullptr;
  uint32_t* st = nullptr;
  if (cudaHostAlloc(&t, sizeof(double) * (kNParam + kMaxCoef) * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&l, sizeof(double) * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&st, sizeof(uint32_t) * cap, cudaHostAllocDefault) != cudaSuccess) {
    if (t) sl.retired.push_back(t);
    if (l) sl.retired.push_back(l);
    return set_err(EMRI_ENOMEM, "serve: pinned staging for %d walkers", w);
  }
  for (void* p : {(void*)sl.h_theta, (void*)sl.h_lnl, (void*)sl.h_st})
    if (p) sl.retired.push_back(p);
  sl.h_theta = t;
  sl.h_lnl = l;
  sl.h_st = st;
  sl.h_cap = cap;
  return EMRI_OK;
}

// Enqueue an admitted request (its pool range at r->off) on a slot
// (scheduler thread, lock held by the caller).
static void launch_request(Server* sv, Slot& sl, const std::shared_ptr<Request>& r) {
  emri_ctx* ctx = sv->ctx;
  r->stats.start_ns = now_ns();
  r->stats.slot = (int32_t)(&sl - sv->slots.data());
  int rc = slot_staging(sl, r->w);
  if (rc != EMRI_OK) {
    pool_give(sv, r->off, r->need);
    r->stats.status = rc;
    r->stats.done_ns = now_ns();
    r->done = true;
    sv->cv_done.notify_all();
    return;
  }
  const size_t nc = r->coef.size();
  memcpy(sl.h_theta, r->theta.data(), sizeof(double) * kNParam * r->w);
  if (nc) memcpy(sl.h_theta + (size_t)kNParam * r->w, r->coef.data(), sizeof(double) * nc);
  char* base = sv->pool + r->off;
  double* d_theta = (double*)base;
  double* d_lnl = d_theta + (size_t)kNParam * r->w;
  uint32_t* d_st = (uint32_t*)(d_lnl + r->w);
  double* d_coef = d_lnl + 2 * (size_t)r->w;   // [qm + qt][w], after lnL and status
  cudaMemcpyAsync(d_theta, sl.h_theta, sizeof(double) * kNParam * r->w, cudaMemcpyHostToDevice, sl.stream);
  if (nc) cudaMemcpyAsync(d_coef, sl.h_theta + (size_t)kNParam * r->w, sizeof(double) * nc, cudaMemcpyHostToDevice,
                          sl.stream);
  Carve cv(base + round256(sizeof(double) * (kNParam + 2 + nc / (size_t)r->w) * (size_t)r->w));
  FdW* fdw = nullptr;
  int64_t nl = 0;
  if (r->fd) {
    fdw = cv.take<FdW>(r->w);
    cv.off = round256(cv.off);
    launch_fdprop(d_theta, r->w, r->w, r->ds->n, r->ds->dt, r->o, r->qm, r->qt, r->fstar, d_coef, r->w, fdw,
                  sl.stream);
    nl += 1;
  }
  LoglikeBufs b;
  loglike_layout(r->ds->plan, r->o, r->w, r->wave, &cv, &b);
  int64_t nr = 0;
  rc = run_loglike(ctx, r->ds, d_theta, r->w, r->w, r->o, r->wave, b, d_lnl, nullptr, nullptr, d_st, sl.stream, &nr,
                   fdw);
  nl += nr;
  cudaMemcpyAsync(sl.h_lnl, d_lnl, sizeof(double) * r->w, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_st, d_st, sizeof(uint32_t) * r->w, cudaMemcpyDeviceToHost, sl.stream);
  cudaEventRecord(sl.done, sl.stream);
  ctx->launches += nl;
  r->stats.status = rc;
  sl.req = r;
}

static void scheduler(Server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (Slot& sl : sv->slots) {
      if (!sl.req) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      auto r = sl.req;
      if (q != cudaSuccess) {
        r->stats.status = EMRI_ECUDA;
      } else {
        memcpy(r->lnl.data(), sl.h_lnl, sizeof(double) * r->w);
        memcpy(r->st.data(), sl.h_st, sizeof(uint32_t) * r->w);
      }
      r->stats.done_ns = now_ns();
      r->done = true;
      pool_give(sv, r->off, r->need);
      sl.req.reset();
      progressed = true;
      sv->cv_done.notify_all();
    }
    // admissions in arrival order: a request that does not fit the pool yet
    // keeps its place, later ones that fit may pass the first such request
    // up to kMaxBypass times, then admission waits for it
    {
      Request* waiting = nullptr;
      for (auto it = sv->queue.begin(); it != sv->queue.end();) {
        Slot* free_slot = nullptr;
        for (Slot& sl : sv->slots)
          if (!sl.req) {
            free_slot = &sl;
            break;
          }
        if (!free_slot) break;
        if (waiting && waiting->bypassed >= kMaxBypass) break;
        auto r = *it;
        size_t off = 0;
        if (!pool_take(sv, r->need, &off)) {
          if (!waiting) waiting = r.get();
          ++it;
          continue;
        }
        r->off = off;
        it = sv->queue.erase(it);
        if (waiting) ++waiting->bypassed;
        launch_request(sv, *free_slot, r);
        progressed = true;
      }
    }
    if (sv->stop) {
      bool busy = false;
      for (Slot& sl : sv->slots) busy |= (bool)sl.req;
      if (!busy && sv->queue.empty()) break;
    }
    if (!progressed) {
      bool busy = false;
      for (Slot& sl : sv->slots) busy |= (bool)sl.req;
      // poll running work at 20 us, otherwise sleep until a submit
      if (busy)
        sv->cv_sched.wait_for(lk, std::chrono::microseconds(20));
      else
        sv->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

void serve_shutdown(emri_ctx* ctx) {
  std::shared_ptr<Server> sp;
  {
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    sp.swap(ctx->server);
  }
  Server* sv = sp.get();
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // requests never admitted are failed
    for (auto& r : sv->queue) {
      r->stats.status = EMRI_ENOTFOUND;
      r->done = true;
    }
    sv->queue.clear();
  }
  sv->cv_sched.notify_all();
  if (sv->th.joinable()) sv->th.join();
  cudaSetDevice(ctx->device);
  for (Slot& sl : sv->slots) {
    cudaStreamSynchronize(sl.stream);
    if (sl.h_theta) cudaFreeHost(sl.h_theta);
    if (sl.h_lnl) cudaFreeHost(sl.h_lnl);
    if (sl.h_st) cudaFreeHost(sl.h_st);
    for (void* p : sl.retired) cudaFreeHost(p);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
  }
  if (sv->pool) {
    cudaFree(sv->pool);
    std::lock_guard<std::mutex> blk(ctx->budget_mu);
    ctx->used -= sv->budget;
  }
  {
    // pollers still waiting wake up to completed or failed requests; the
    // Server object itself lives until the last of them lets go of it
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->cv_done.notify_all();
  }
}

// The tuned plan for (n, n_max, precision); without one for this n_max, the
// plan tuned for the same length and precision at the nearest n_max (the
// choices depend on the length far more than on the harmonic count).
static const Plan* find_plan(emri_ctx* ctx, int64_t n, const OptsN& o) {
  auto it = ctx->plans.find(std::make_tuple(n, o.n_max, o.precision));
  if (it != ctx->plans.end()) return &it->second;
  const Plan* best = nullptr;
  int dist = 1 << 30;
  for (auto lo = ctx->plans.lower_bound(std::make_tuple(n, 0, 0)); lo != ctx->plans.end(); ++lo) {
    if (std::get<0>(lo->first) != n) break;
    if (std::get<2>(lo->first) != o.precision) continue;
    const int d = std::abs(std::get<1>(lo->first) - o.n_max);
    if (d < dist) {
      dist = d;
      best = &lo->second;
    }
  }
  return best;
}

int ctx_plan_ks(emri_ctx* ctx, int64_t n, const OptsN& o) {
  const Plan* p = find_plan(ctx, n, o);
  return p ? p->ks : 0;
}

int ctx_plan_wave(emri_ctx* ctx, int64_t n, const OptsN& o) {
  const Plan* p = find_plan(ctx, n, o);
  return p ? p->wave : 0;
}

}  // namespace emri

// ================================================================ serving
extern "C" int emri_serve_start(emri_ctx* ctx, const emri_serve_cfg* cfg) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  std::lock_guard<std::mutex> slk(ctx->server_mu);
  if (ctx->server) return set_err(EMRI_EINVAL, "serving already started");
  emri_serve_cfg c = cfg ? *cfg : emri_serve_cfg{4, 1024, 0};
  if (c.slots < 1 || c.slots > 64) return set_err(EMRI_EINVAL, "slots must be in [1, 64]");
  if (c.queue_capacity < 1) return set_err(EMRI_EINVAL, "queue_capacity must be >= 1");
  cudaSetDevice(ctx->device);
  auto sp = std::make_shared<Server>();
  Server* sv = sp.get();
  sv->ctx = ctx;
  sv->cfg = c;
  // the pool: the requested budget (at most what the context has left), or
  // half the context's remaining budget (the other half stays for direct
  // calls on the same context); charged to the context while serving runs
  size_t want;
  {
    std::lock_guard<std::mutex> blk(ctx->budget_mu);
    const size_t room = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
    want = (c.budget_bytes ? std::min(c.budget_bytes, room) : room / 2) & ~(size_t)255;
    if (want < 256) return set_err(EMRI_EBUDGET, "no room left in the context's budget for serving");
    ctx->used += want;
  }
  sv->budget = want;
  auto fail = [&](int code, const char* what) {
    for (Slot& q : sv->slots) {
      if (q.done) cudaEventDestroy(q.done);
      if (q.stream) cudaStreamDestroy(q.stream);
      for (void* hp : {(void*)q.h_theta, (void*)q.h_lnl, (void*)q.h_st})
        if (hp) cudaFreeHost(hp);
    }
    if (sv->pool) cudaFree(sv->pool);
    std::lock_guard<std::mutex> blk(ctx->budget_mu);
    ctx->used -= want;
    return set_err(code, "serve: %s", what);
  };
  if (cudaMalloc(&sv->pool, want) != cudaSuccess) {
    sv->pool = nullptr;
    return fail(EMRI_ENOMEM, "pool allocation failed");
  }
  sv->free_ranges[0] = want;
  sv->slots.resize(c.slots);
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      return fail(EMRI_ECUDA, "stream/event creation failed");
    if (slot_staging(sl, kStageWalkers) != EMRI_OK) return fail(EMRI_ENOMEM, "pinned staging");
  }
  ctx->server = sp;
  sv->th = std::thread(scheduler, sv);
  return EMRI_OK;
}

static std::shared_ptr<Server> server_of(emri_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->server_mu);
  return ctx->server;
}

extern "C" int emri_serve_stop(emri_ctx* ctx) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  if (!server_of(ctx)) return set_err(EMRI_ENOTFOUND, "serving not started");
  serve_shutdown(ctx);
  return EMRI_OK;
}

static int serve_submit(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                        const emri_opts* opts, bool fd, int qm, int qt, double fstar, const double* coef_host,
                        uint64_t* ticket) {
  if (!ctx || !ds || !ticket) return set_err(EMRI_EINVAL, "NULL argument");
  const std::shared_ptr<Server> sp = server_of(ctx);
  Server* sv = sp.get();
  if (!sv) return set_err(EMRI_ENOTFOUND, "serving not started");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 1) return set_err(EMRI_EINVAL, "w must be >= 1");
  if (!theta_host) return set_err(EMRI_EINVAL, "NULL theta");
  if (fd) {
    if (qm < 0 || qm > 3 || qt < 0 || qt > 3) return set_err(EMRI_EINVAL, "q_m and q_t must be in [0, 3]");
    if (!(fstar > 0) || !isfinite(fstar)) return set_err(EMRI_EINVAL, "f_star must be positive and finite");
    if (qm + qt > 0 && !coef_host) return set_err(EMRI_EINVAL, "NULL propagation coefficients");
  }
  auto r = std::make_shared<Request>();
  int rc = normalize_opts(opts, ds->n, &r->o);
  if (rc) return rc;
  r->ds = ds;
  r->w = w;
  r->theta.assign(theta_host, theta_host + (size_t)kNParam * w);
  r->fd = fd;
  if (fd) {
    r->qm = qm;
    r->qt = qt;
    r->fstar = fstar;
    if (qm + qt > 0) r->coef.assign(coef_host, coef_host + (size_t)(qm + qt) * w);
  }
  {
    std::lock_guard<std::mutex> clk(ctx->mu);   // the tuned plans
    r->wave = pick_wave(ctx, ds->plan, r->o, w);
  }
  r->need = request_bytes(ds, r->o, w, r->wave, fd, fd ? qm + qt : 0);
  r->lnl.assign(w, 0.0);
  r->st.assign(w, 0u);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return set_err(EMRI_ENOTFOUND, "serving is stopping");
  if (r->need > sv->budget)
    return set_err(EMRI_EBUDGET, "request needs %zu bytes, serving budget is %zu", r->need, sv->budget);
  if ((int)sv->queue.size() >= sv->cfg.queue_capacity) return set_err(EMRI_EAGAIN, "serving queue full");
  r->ticket = sv->next_ticket++;
  r->stats.arrival_ns = now_ns();
  r->stats.slot = -1;
  sv->queue.push_back(r);
  sv->reqs[r->ticket] = r;
  *ticket = r->ticket;
  sv->cv_sched.notify_all();
  return EMRI_OK;
}

extern "C" int emri_serve_submit(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                                 const emri_opts* opts, uint64_t* ticket) {
  return serve_submit(ctx, ds, theta_host, w, opts, false, 0, 0, 1.0, nullptr, ticket);
}

extern "C" int emri_serve_submit_fd(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                                    const emri_opts* opts, int q_m, int q_t, double f_star, const double* coef_host,
                                    uint64_t* ticket) {
  return serve_submit(ctx, ds, theta_host, w, opts, true, q_m, q_t, f_star, coef_host, ticket);
}

extern "C" int emri_serve_request_bytes(emri_ctx* ctx, const emri_dataset* ds, int w, const emri_opts* opts,
                                        size_t* bytes) {
  if (!ctx || !ds || !bytes) return set_err(EMRI_EINVAL, "NULL argument");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 1) return set_err(EMRI_EINVAL, "w must be >= 1");
  OptsN o;
  int rc = normalize_opts(opts, ds->n, &o);
  if (rc) return rc;
  std::lock_guard<std::mutex> clk(ctx->mu);   // the tuned plans
  *bytes = request_bytes(ds, o, w, pick_wave(ctx, ds->plan, o, w), false, 0);
  return EMRI_OK;
}

extern "C" int emri_serve_poll(emri_ctx* ctx, uint64_t ticket, double* lnl_host, uint32_t* status_host,
                               emri_req_stats* stats, int64_t timeout_us) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  const std::shared_ptr<Server> sp = server_of(ctx);
  Server* sv = sp.get();
  if (!sv) return set_err(EMRI_ENOTFOUND, "serving not started");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_err(EMRI_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_us < 0) {
    sv->cv_done.wait(lk, pred);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    return set_err(EMRI_ETIMEDOUT, "request %llu not done", (unsigned long long)ticket);
  }
  if (lnl_host) memcpy(lnl_host, r->lnl.data(), sizeof(double) * r->w);
  if (status_host) memcpy(status_host, r->st.data(), sizeof(uint32_t) * r->w);
  if (stats) *stats = r->stats;
  sv->reqs.erase(it);
  if (r->stats.status != EMRI_OK) return set_err(r->stats.status, "request %llu failed", (unsigned long long)ticket);
  return EMRI_OK;
}

// ========================================================= uneven batching
namespace emri {

// A captured multi-chain launch: one branch per chain inside one CUDA graph.
struct MultiGraph {
  std::vector<uint64_t> key;
  std::vector<Workspace> ws;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
};

void multi_destroy(emri_ctx* ctx) {
  MultiGraph* m = ctx->multi;
  if (!m) return;
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  for (Workspace& w : m->ws) w.destroy(ctx);
  for (cudaStream_t b : m->branches) cudaStreamDestroy(b);
  for (cudaEvent_t e : m->joins) cudaEventDestroy(e);
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
  ctx->multi = nullptr;
}

static void key_push(std::vector<uint64_t>& k, const void* p) { k.push_back((uint64_t)(uintptr_t)p); }

}  // namespace emri

extern "C" int emri_loglike_multi(emri_ctx* ctx, const emri_work* items, int n_items, void* stream) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  if (n_items < 0 || (n_items > 0 && !items)) return set_err(EMRI_EINVAL, "bad item list");
  if (n_items == 0) return EMRI_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::vector<OptsN> on(n_items);
  std::vector<uint64_t> key;
  for (int i = 0; i < n_items; ++i) {
    const emri_work& it = items[i];
    if (!it.ds || it.ds->ctx != ctx) return set_err(EMRI_EINVAL, "item %d: missing or foreign dataset", i);
    if (it.w < 0) return set_err(EMRI_EINVAL, "item %d: w must be >= 0", i);
    if (it.w > 0 && (!it.theta_dev || !it.lnl_dev)) return set_err(EMRI_EINVAL, "item %d: NULL pointer", i);
    int rc = normalize_opts(&it.opts, it.ds->n, &on[i]);
    if (rc) return rc;
    if (it.fd) {
      if (it.fd->q_m < 0 || it.fd->q_m > 3 || it.fd->q_t < 0 || it.fd->q_t > 3)
        return set_err(EMRI_EINVAL, "item %d: q_m and q_t must be in [0, 3]", i);
      if (!(it.fd->f_star > 0) || !isfinite(it.fd->f_star))
        return set_err(EMRI_EINVAL, "item %d: f_star must be positive and finite", i);
      if (it.w > 0 && it.fd->q_m + it.fd->q_t > 0 && !it.fd->coef_dev)
        return set_err(EMRI_EINVAL, "item %d: NULL propagation coefficients", i);
    }
    if (!it.opts.knot_spacing) {   // the autotuner's choice for this shape, if any
      const int pk = ctx_plan_ks(ctx, it.ds->n, on[i]);
      if (pk) on[i].ks = pk;
    }
    key_push(key, it.ds);
    key_push(key, it.theta_dev);
    key.push_back((uint64_t)it.w);
    key_push(key, it.lnl_dev);
    key_push(key, it.dh_dev);
    key_push(key, it.hh_dev);
    key_push(key, it.status_dev);
    key.push_back(((uint64_t)on[i].precision << 48) | ((uint64_t)on[i].n_max << 32) | ((uint64_t)on[i].ks << 8) |
                  ((uint64_t)on[i].pn_terms << 1) | (uint64_t)on[i].doppler);
    uint64_t f[3];
    memcpy(&f[0], &on[i].n_xi, 8);
    memcpy(&f[1], &on[i].omega_m, 8);
    memcpy(&f[2], &on[i].h0, 8);
    key.insert(key.end(), f, f + 3);
    if (it.fd) {
      uint64_t fs;
      memcpy(&fs, &it.fd->f_star, 8);
      key.push_back(1 + ((uint64_t)it.fd->q_m << 8) + ((uint64_t)it.fd->q_t << 16));
      key.push_back(fs);
      key_push(key, it.fd->coef_dev);
    } else {
      key.push_back(0);
    }
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(EMRI_ECUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  MultiGraph* m = ctx->multi;
  if (!m || m->key != key) {
    multi_destroy(ctx);
    m = new MultiGraph();
    ctx->multi = m;
    m->key = key;
    m->ws.resize(n_items);
    const int nb = std::min(n_items, 64);
    m->branches.resize(nb);
    m->joins.resize(n_items);
    cudaError_t e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&m->branches[b], cudaStreamNonBlocking);
    for (int i = 0; i < n_items && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&m->joins[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      multi_destroy(ctx);
      return cuda_err(e, "multi: streams/events");
    }
    // per-chain workspaces; the time series of a chain is bounded to ~512 MiB per wave
    std::vector<int> wave(n_items, 0);
    for (int i = 0; i < n_items; ++i) {
      if (items[i].w == 0) continue;
      const size_t cs = on[i].precision ? sizeof(float2) : sizeof(double2);
      const size_t per = (size_t)items[i].ds->n * cs;
      wave[i] = (int)std::max<size_t>(1, std::min<size_t>((size_t)items[i].w, ((size_t)512 << 20) / per));
      const int pw = ctx_plan_wave(ctx, items[i].ds->n, on[i]);
      if (pw > 0 && pw < wave[i]) wave[i] = pw;
      const size_t fdb = items[i].fd ? ((sizeof(FdW) * (size_t)items[i].w + 255) & ~(size_t)255) : 0;
      int rc = m->ws[i].reserve(
          ctx, fdb + loglike_layout(items[i].ds->plan, on[i], items[i].w, wave[i], nullptr, nullptr), m->cap);
      if (rc) {
        multi_destroy(ctx);
        return rc;
      }
    }
    // capture: fork from the capture stream into one branch per chain, join back
    const bool prof_was_on = ctx->prof.on;
    ctx->prof.on = false;   // no timing events inside a capture
    e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
    int rc = EMRI_OK;
    if (e == cudaSuccess) {
      cudaEventRecord(m->fork, m->cap);
      for (int i = 0; i < n_items && rc == EMRI_OK; ++i) {
        cudaStream_t br = m->branches[i % nb];
        cudaStreamWaitEvent(br, m->fork, 0);
        if (items[i].w > 0) {
          Carve cv(m->ws[i].ptr);
          FdW* fdw = nullptr;
          const emri_fdprop* fd = items[i].fd;
          if (fd) {
            fdw = cv.take<FdW>(items[i].w);
            cv.off = (cv.off + 255) & ~(size_t)255;
            launch_fdprop(items[i].theta_dev, items[i].w, items[i].w, items[i].ds->n, items[i].ds->dt, on[i],
                          fd->q_m, fd->q_t, fd->f_star, fd->coef_dev, items[i].w, fdw, br);
            m->launches += 1;
          }
          LoglikeBufs b;
          loglike_layout(items[i].ds->plan, on[i], items[i].w, wave[i], &cv, &b);
          int64_t nl = 0;
          rc = run_loglike(ctx, items[i].ds, items[i].theta_dev, items[i].w, items[i].w, on[i], wave[i], b,
                           items[i].lnl_dev, items[i].dh_dev, items[i].hh_dev, items[i].status_dev, br, &nl, fdw);
          m->launches += nl;
        }
        cudaEventRecord(m->joins[i], br);
        cudaStreamWaitEvent(m->cap, m->joins[i], 0);
      }
      cudaError_t e2 = cudaStreamEndCapture(m->cap, &m->graph);
      if (e == cudaSuccess) e = e2;
    }
    ctx->prof.on = prof_was_on;
    if (rc == EMRI_OK && e == cudaSuccess) e = cudaGraphInstantiate(&m->exec, m->graph, 0);
    if (rc != EMRI_OK || e != cudaSuccess) {
      multi_destroy(ctx);
      return rc != EMRI_OK ? rc : cuda_err(e, "multi: graph capture");
    }
  }
  cudaError_t e = cudaGraphLaunch(m->exec, s);
  if (e != cudaSuccess) return cuda_err(e, "multi: graph launch");
  ctx->launches += m->launches;
  return EMRI_OK;
}

// ============================================================== autotuner
// Candidates, timed on a synthetic batch of the requested shape:
//  * knot spacing: FP64 keeps 128 (its accuracy budget); mixed tries 512, 1024;
//  * walkers per wave (the time-series buffer): all, 64, 16, 4 -- small waves
//    keep a wave's series resident in L2 between the waveform and FFT kernels;
//  * FFT split n = n1 * n2: the default n2 and its neighbours within the
//    shared-memory limits.  The split becomes part of a dataset when it is
//    created, so tune before creating the datasets it should apply to.
namespace emri {

static void synth_walkers(int w, int64_t n, double dt, std::vector<double>& th) {
  // representative sources (M ~ 1e6, mu ~ 10, e0 ~ 0.2) starting ~2 T before the LSO
  th.assign((size_t)kNParam * w, 0.0);
  const double tsun = kGMsun / (kC * kC * kC);
  for (int i = 0; i < w; ++i) {
    const double M = 6e5 + 1e5 * (i % 7), mu = 8.0 + (i % 5), e0 = 0.15 + 0.02 * (i % 6);
    const double ms = M * tsun, mus = mu * tsun;
    const double ul = pow((1 - e0 * e0) / (6 + 2 * e0), 1.5);
    const double u0 = pow(pow(ul, -8.0 / 3.0) + 256.0 / 5.0 * (mus / (ms * ms)) * 2.0 * (double)n * dt, -3.0 / 8.0);
    double v[kNParam] = {M, mu, 0.3 + 0.05 * (i % 9), e0, u0 / (2 * kPi * ms), 0.1 * i, 0.2 * i, 0.3 * i,
                         0.4 + 0.1 * (i % 20), 0.5 * i, 0.9, 0.3 * i, 0.8, 0.4, 1.0, 0.0};
    for (int p = 0; p < kNParam; ++p) th[(size_t)p * w + i] = v[p];
  }
}

static bool read_cache(const char* path, int64_t n, int n_max, int prec, Plan* out, int* n2) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    long long nn = 0, ks = 0, wave = 0, s2 = 0;
    int nm = 0, pr = 0;
    if (sscanf(line.c_str(), "{\"n\": %lld, \"n_max\": %d, \"precision\": %d, \"knot_spacing\": %lld, \"wave\": %lld, \"n2\": %lld",
               &nn, &nm, &pr, &ks, &wave, &s2) == 6 &&
        nn == n && nm == n_max && pr == prec) {
      out->ks = (int)ks;
      out->wave = (int)wave;
      *n2 = (int)s2;
      found = true;   // the last matching line wins
    }
  }
  return found;
}

}  // namespace emri

extern "C" int emri_autotune(emri_ctx* ctx, const emri_grid* grid, int n_max, int precision, const char* cache_path,
                             int64_t* choice_out) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  int rc = check_grid(grid);
  if (rc) return rc;
  emri_opts oo;
  emri_opts_default(&oo);
  oo.precision = precision;
  oo.n_max = n_max;
  OptsN base;
  if ((rc = normalize_opts(&oo, grid->n, &base))) return rc;
  const int64_t n = grid->n;
  Plan best;
  int best_n2 = 0;
  if (read_cache(cache_path, n, n_max, precision, &best, &best_n2)) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->plans[std::make_tuple(n, n_max, precision)] = best;
    if (best_n2) ctx->fft_split[n] = best_n2;
    if (choice_out) {
      choice_out[0] = best.ks;
      choice_out[1] = best.wave;
      choice_out[2] = best_n2 ? n / best_n2 : make_fft_plan(n).n1;
    }
    return EMRI_OK;
  }
  const size_t cs = precision ? sizeof(float2) : sizeof(double2);
  const int w = (int)std::max<int64_t>(4, std::min<int64_t>(64, ((int64_t)4 << 30) / (n * (int64_t)cs)));
  std::vector<double> th;
  synth_walkers(w, n, grid->dt, th);
  // device buffers for the synthetic batch
  double* d = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(EMRI_ECUDA, "cudaSetDevice");
  if (cudaMalloc(&d, sizeof(double) * (kNParam + 3) * w) != cudaSuccess) return set_err(EMRI_ENOMEM, "autotune buffers");
  cudaMemcpy(d, th.data(), sizeof(double) * kNParam * w, cudaMemcpyHostToDevice);
  double* lnl = d + (size_t)kNParam * w;
  std::vector<int> ks_c = precision ? std::vector<int>{512, 1024} : std::vector<int>{128};
  std::vector<int> wave_c = {w, 64, 16, 4};
  const FftPlan def = make_fft_plan(n);
  std::vector<int> n2_c = {def.n2};
  if (def.n2 / 2 >= 32 && n / (def.n2 / 2) <= 4096) n2_c.push_back(def.n2 / 2);
  if (def.n2 * 2 <= 1024 && n / (def.n2 * 2) >= 32) n2_c.push_back(def.n2 * 2);
  float best_ms = 1e30f;
  std::vector<double> zeros((size_t)2 * n, 0.0), psd((size_t)n / 2 + 1);
  for (int64_t k = 0; k <= n / 2; ++k) {
    const double f = (double)(k ? k : 1) / ((double)n * grid->dt);
    psd[k] = 9.18e-52 / (f * f * f * f) + 1.59e-41 + 9.18e-38 * f * f;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int n2 : n2_c) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->fft_split[n] = n2;
    }
    emri_dataset* ds = nullptr;
    rc = emri_dataset_create(ctx, grid, zeros.data(), 0, psd.data(), 1e-4, 0.5 / grid->dt, &ds);
    if (rc) break;
    for (int ks : ks_c) {
      for (int wv : wave_c) {
        if (wv > w) continue;
        emri_opts o = oo;
        o.knot_spacing = ks;
        {
          std::lock_guard<std::mutex> lk(ctx->mu);
          ctx->plans[std::make_tuple(n, n_max, precision)] = Plan{ks, wv};
        }
        float ms = 0.f;
        for (int rep = 0; rep < 3 && rc == EMRI_OK; ++rep) {
          cudaEventRecord(e0, ctx->stream);
          rc = emri_loglike_batch(ctx, ds, d, w, &o, lnl, nullptr, nullptr, nullptr, ctx->stream);
          cudaEventRecord(e1, ctx->stream);
          cudaEventSynchronize(e1);
          float m = 0.f;
          cudaEventElapsedTime(&m, e0, e1);
          if (rep > 0) ms += m;   // first run warms up
        }
        if (rc) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = Plan{ks, wv};
          best_n2 = n2;
        }
      }
      if (rc) break;
    }
    emri_dataset_destroy(ds);
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (rc == EMRI_OK) {
      ctx->plans[std::make_tuple(n, n_max, precision)] = best;
      ctx->fft_split[n] = best_n2;
    } else {
      ctx->plans.erase(std::make_tuple(n, n_max, precision));
      ctx->fft_split.erase(n);
    }
  }
  if (rc) return rc;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "{\"n\": %lld, \"n_max\": %d, \"precision\": %d, \"knot_spacing\": %d, \"wave\": %d, \"n2\": %d, \"ms\": %.4f}\n",
              (long long)n, n_max, precision, best.ks, best.wave, best_n2, best_ms / 2.0f);
      fclose(f);
    }
  }
  if (choice_out) {
    choice_out[0] = best.ks;
    choice_out[1] = best.wave;
    choice_out[2] = n / best_n2;
  }
  return EMRI_OK;
}
