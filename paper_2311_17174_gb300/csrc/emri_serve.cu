// emri_serve.cu -- continuous-batching request loop, multi-chain launches
// and the autotuner of libemri.
//
// Serving: a scheduler thread owns S stream slots.  Requests (a dataset and
// W walkers) wait in a FIFO; whenever a slot is free and the HBM budget has
// room for the request's workspace, the request is admitted: its parameters
// go host->device from a pinned staging buffer, the likelihood path is
// enqueued on the slot's stream, and the results come back device->host into
// pinned memory, all asynchronously.  Requests in different slots overlap on
// the device; completion is detected by polling an event per slot.  The
// kernels reduce in a fixed order per walker, so a request's results are
// bitwise the same alone or in a mix.
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <fstream>
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

struct Request {
  uint64_t ticket = 0;
  const emri_dataset* ds = nullptr;
  std::vector<double> theta;   // [16][w]
  int w = 0;
  OptsN o{};
  size_t need = 0;             // workspace bytes
  int wave = 0;
  std::vector<double> lnl;
  std::vector<uint32_t> st;
  emri_req_stats stats{};
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Workspace ws;
  double* h_theta = nullptr;   // pinned staging
  double* h_lnl = nullptr;
  uint32_t* h_st = nullptr;
  size_t h_cap = 0;            // walkers
  double* d_io = nullptr;      // device theta + lnl + status
  size_t d_cap = 0;
  std::shared_ptr<Request> req;
  size_t reserved = 0;         // budget charged while busy
};

struct Server {
  emri_ctx* ctx = nullptr;
  emri_serve_cfg cfg{};
  size_t budget = 0;
  size_t in_use = 0;
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

static int slot_buffers(Slot& sl, int w) {
  if ((size_t)w > sl.h_cap) {
    if (sl.h_theta) cudaFreeHost(sl.h_theta);
    if (sl.h_lnl) cudaFreeHost(sl.h_lnl);
    if (sl.h_st) cudaFreeHost(sl.h_st);
    sl.h_theta = nullptr;
    sl.h_lnl = nullptr;
    sl.h_st = nullptr;
    if (cudaMallocHost(&sl.h_theta, sizeof(double) * kNParam * w) != cudaSuccess ||
        cudaMallocHost(&sl.h_lnl, sizeof(double) * w) != cudaSuccess ||
        cudaMallocHost(&sl.h_st, sizeof(uint32_t) * w) != cudaSuccess) {
      sl.h_cap = 0;
      return EMRI_ENOMEM;
    }
    sl.h_cap = w;
  }
  if ((size_t)w > sl.d_cap) {
    if (sl.d_io) cudaFree(sl.d_io);
    sl.d_io = nullptr;
    if (cudaMalloc(&sl.d_io, sizeof(double) * (kNParam + 2) * w) != cudaSuccess) {
      sl.d_cap = 0;
      return EMRI_ENOMEM;
    }
    sl.d_cap = w;
  }
  return EMRI_OK;
}

// Enqueue a request on a slot (scheduler thread, lock held by caller).
static void launch_request(Server* sv, Slot& sl, const std::shared_ptr<Request>& r) {
  emri_ctx* ctx = sv->ctx;
  r->stats.start_ns = now_ns();
  int rc = slot_buffers(sl, r->w);
  if (rc == EMRI_OK) rc = sl.ws.reserve(ctx, r->need, sl.stream);
  if (rc != EMRI_OK) {
    r->stats.status = rc;
    r->stats.done_ns = now_ns();
    r->done = true;
    sv->cv_done.notify_all();
    return;
  }
  memcpy(sl.h_theta, r->theta.data(), sizeof(double) * kNParam * r->w);
  double* d_theta = sl.d_io;
  double* d_lnl = sl.d_io + (size_t)kNParam * r->w;
  uint32_t* d_st = (uint32_t*)(d_lnl + r->w);
  cudaMemcpyAsync(d_theta, sl.h_theta, sizeof(double) * kNParam * r->w, cudaMemcpyHostToDevice, sl.stream);
  Carve cv(sl.ws.ptr);
  LoglikeBufs b;
  loglike_layout(r->ds->plan, r->o, r->w, r->wave, &cv, &b);
  int64_t nl = 0;
  rc = run_loglike(ctx, r->ds, d_theta, r->w, r->w, r->o, r->wave, b, d_lnl, nullptr, nullptr, d_st, sl.stream, &nl);
  cudaMemcpyAsync(sl.h_lnl, d_lnl, sizeof(double) * r->w, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_st, d_st, sizeof(uint32_t) * r->w, cudaMemcpyDeviceToHost, sl.stream);
  cudaEventRecord(sl.done, sl.stream);
  ctx->launches += nl;
  r->stats.status = rc;
  r->stats.slot = (int32_t)(&sl - sv->slots.data());
  sl.req = r;
  sl.reserved = r->need;
  sv->in_use += r->need;
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
      sv->in_use -= sl.reserved;
      sl.reserved = 0;
      sl.req.reset();
      progressed = true;
      sv->cv_done.notify_all();
    }
    // admissions, FIFO: the head waits for a slot and for budget room
    while (!sv->queue.empty()) {
      auto r = sv->queue.front();
      Slot* free_slot = nullptr;
      for (Slot& sl : sv->slots)
        if (!sl.req) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      if (sv->in_use + r->need > sv->budget) break;
      sv->queue.pop_front();
      launch_request(sv, *free_slot, r);
      progressed = true;
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
  Server* sv = ctx->server;
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
    sl.ws.destroy(ctx);
    if (sl.h_theta) cudaFreeHost(sl.h_theta);
    if (sl.h_lnl) cudaFreeHost(sl.h_lnl);
    if (sl.h_st) cudaFreeHost(sl.h_st);
    if (sl.d_io) cudaFree(sl.d_io);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
  }
  sv->cv_done.notify_all();
  delete sv;
  ctx->server = nullptr;
}

int ctx_plan_wave(emri_ctx* ctx, int64_t n, const OptsN& o) {
  auto it = ctx->plans.find(std::make_tuple(n, o.n_max, o.precision));
  return it == ctx->plans.end() ? 0 : it->second.wave;
}

}  // namespace emri

// ================================================================ serving
extern "C" int emri_serve_start(emri_ctx* ctx, const emri_serve_cfg* cfg) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  if (ctx->server) return set_err(EMRI_EINVAL, "serving already started");
  emri_serve_cfg c = cfg ? *cfg : emri_serve_cfg{4, 1024, 0};
  if (c.slots < 1 || c.slots > 64) return set_err(EMRI_EINVAL, "slots must be in [1, 64]");
  if (c.queue_capacity < 1) return set_err(EMRI_EINVAL, "queue_capacity must be >= 1");
  cudaSetDevice(ctx->device);
  Server* sv = new Server();
  sv->ctx = ctx;
  sv->cfg = c;
  size_t room = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
  sv->budget = c.budget_bytes ? std::min(c.budget_bytes, room) : room;
  sv->slots.resize(c.slots);
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      delete sv;
      return set_err(EMRI_ECUDA, "serve: stream/event creation failed");
    }
  }
  ctx->server = sv;
  sv->th = std::thread(scheduler, sv);
  return EMRI_OK;
}

extern "C" int emri_serve_stop(emri_ctx* ctx) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  if (!ctx->server) return set_err(EMRI_ENOTFOUND, "serving not started");
  serve_shutdown(ctx);
  return EMRI_OK;
}

extern "C" int emri_serve_submit(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                                 const emri_opts* opts, uint64_t* ticket) {
  if (!ctx || !ds || !ticket) return set_err(EMRI_EINVAL, "NULL argument");
  Server* sv = ctx->server;
  if (!sv) return set_err(EMRI_ENOTFOUND, "serving not started");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 1) return set_err(EMRI_EINVAL, "w must be >= 1");
  if (!theta_host) return set_err(EMRI_EINVAL, "NULL theta");
  auto r = std::make_shared<Request>();
  int rc = normalize_opts(opts, ds->n, &r->o);
  if (rc) return rc;
  r->ds = ds;
  r->w = w;
  r->theta.assign(theta_host, theta_host + (size_t)kNParam * w);
  r->wave = pick_wave(ctx, ds->plan, r->o, w);
  r->need = loglike_layout(ds->plan, r->o, w, r->wave, nullptr, nullptr);
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

extern "C" int emri_serve_poll(emri_ctx* ctx, uint64_t ticket, double* lnl_host, uint32_t* status_host,
                               emri_req_stats* stats, int64_t timeout_us) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  Server* sv = ctx->server;
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
extern "C" int emri_loglike_multi(emri_ctx* ctx, const emri_work* items, int n_items, void* stream) {
  return set_err(EMRI_EINVAL, "multi-chain launches are not available in this build");
}

// ============================================================== autotuner
extern "C" int emri_autotune(emri_ctx* ctx, const emri_grid* grid, int n_max, int precision, const char* cache_path,
                             int64_t* choice_out) {
  return set_err(EMRI_EINVAL, "autotuning is not available in this build");
}
