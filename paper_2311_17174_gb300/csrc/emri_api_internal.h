// emri_api_internal.h -- host-side objects behind the C-ABI handles.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/emri.h"
#include "emri_internal.h"

namespace emri {
struct Server;
struct MultiGraph;
}

struct emri_ctx;

namespace emri {

// A growable device buffer reused across calls; cross-stream use is ordered
// through an event recorded after the last call that used it.
struct Workspace {
  char* ptr = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool has_ev = false;
  cudaStream_t last_stream = nullptr;
  bool poison = false;   // fill with 0xFF bytes (FP NaN) at every acquire
  int reserve(emri_ctx* ctx, size_t bytes, cudaStream_t s);
  void acquire(cudaStream_t s);
  void release(cudaStream_t s);
  void destroy(emri_ctx* ctx);
};

// Carve a workspace into per-call buffers (256-byte aligned); with a NULL
// base it only measures.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* p) : base((char*)p) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* r = (T*)(base ? base + off : nullptr);
    off += count * sizeof(T);
    return r;
  }
};

struct LoglikeBufs {
  WalkerC* wc;
  Knot* knots;
  char* ivs;       // mixed interval records [w][n/ks]
  double* lisa;    // per-tile LISA-phase table [n/256][8]
  char* dtab;
  char* rtab;      // per-walker row delay factors [w][n2]
  double2* partial;
  char* z;
};

// Per-kernel event timing (enabled by emri_ctx_profile).
struct Profiler {
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> pool;
  double ms[EMRI_NKERNEL] = {};
  int64_t count[EMRI_NKERNEL] = {};
  cudaEvent_t get();
  // bracket one launch: begin() before, end() after
  cudaEvent_t begin(cudaStream_t s);
  void end(int kind, cudaEvent_t b, cudaStream_t s);
  void drain();
  void reset();
};

// RAII helper: times one launch when profiling is on
struct KTimer {
  Profiler* p;
  int kind;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  KTimer(Profiler* p_, int k, cudaStream_t s_) : p(p_), kind(k), s(s_) {
    if (p && p->on) b = p->begin(s);
  }
  ~KTimer() {
    if (b) p->end(kind, b, s);
  }
};

// most walker groups of a pipelined likelihood call (emri_ctx_set_pipeline)
constexpr int kMaxPipe = 64;

// autotuned schedule of one (n, n_max, precision) shape
struct Plan {
  int ks = 0;
  int wave = 0;
};

}  // namespace emri

struct emri_ctx {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;            // guarded by budget_mu (the serving thread reserves too)
  std::mutex budget_mu;
  std::mutex mu;
  cudaStream_t stream = nullptr;
  char* tables = nullptr;
  emri::Twiddles tw{};
  emri::BesselTab bt{};
  double* gl = nullptr;
  double* mcpi = nullptr;     // orbit integration tables (qn, qk)
  emri::Workspace ws;
  std::atomic<int64_t> launches{0};
  // the serving loop; submit/poll hold a reference, so a concurrent stop
  // cannot free it under them (swapped under server_mu)
  std::shared_ptr<emri::Server> server;
  std::mutex server_mu;
  emri::MultiGraph* multi = nullptr;
  emri::Profiler prof;
  std::map<std::tuple<int64_t, int, int>, emri::Plan> plans;   // (n, n_max, precision)
  std::map<int64_t, int> fft_split;                             // n -> n2 for new datasets
  // pipelined likelihood schedule (emri_ctx_set_pipeline): walker groups
  // per wave by precision (1 = the steps in sequence on the caller's
  // stream, 0 = by the call's size), the two context streams it adds
  // (orbits; FFT passes and reduction) and its events, created at the first
  // pipelined call
  int pipe[2] = {1, 0};
  cudaStream_t pstream[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> pev;
};

struct emri_dataset {
  emri_ctx* ctx = nullptr;
  int64_t n = 0;
  double dt = 0, t0 = 0, fmin = 0, fmax = 0;
  emri::FftPlan plan{};
  char* mem = nullptr;
  size_t bytes = 0;
  double2* g_perm = nullptr;   // w conj(D) in pass-2 order (FP64), then the FP32 copies
  double* w_perm = nullptr;
  float2* g_perm32 = nullptr;
  float* w_perm32 = nullptr;
  double d_scale = 1.0, w_scale = 1.0;
  double dd = 0.0;
};

namespace emri {
int set_err(int code, const char* fmt, ...);
int cuda_err(cudaError_t e, const char* where);
int normalize_opts(const emri_opts* in, int64_t n, OptsN* o);
int check_grid(const emri_grid* g);
size_t loglike_layout(const FftPlan& p, const OptsN& o, int w, int wave, Carve* c, LoglikeBufs* b);
int pick_wave(emri_ctx* ctx, const FftPlan& p, const OptsN& o, int w);
int run_loglike(emri_ctx* ctx, const emri_dataset* ds, const double* theta, int64_t ld, int w, const OptsN& o,
                int wave, const LoglikeBufs& b, double* lnl, double* dh, double* hh, uint32_t* status,
                cudaStream_t s, int64_t* launches, const FdW* fd = nullptr, int pipe = 1);
// walker groups for a likelihood call on stream s: the context's setting for
// the precision (0: by the call's size), 1 while s is being captured
int pipe_groups(emri_ctx* ctx, const OptsN& o, cudaStream_t s);
int ctx_plan_wave(emri_ctx* ctx, int64_t n, const OptsN& o);
int ctx_plan_ks(emri_ctx* ctx, int64_t n, const OptsN& o);
void serve_shutdown(emri_ctx* ctx);
void multi_destroy(emri_ctx* ctx);
}  // namespace emri
