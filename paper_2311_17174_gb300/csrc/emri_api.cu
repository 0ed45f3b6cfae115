// emri_api.cu -- the C-ABI of libemri (include/emri.h): contexts, datasets,
// workspaces and the launch sequence of the batched AK log-likelihood.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/emri.h"
#include "emri_api_internal.h"
#include "emri_common.cuh"
#include "emri_internal.h"

using namespace emri;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

namespace emri {
int set_err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_err(cudaError_t e, const char* where) {
  return set_err(EMRI_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}
}  // namespace emri

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_err(e_, #call); \
  } while (0)

extern "C" const char* emri_last_error(void) { return g_err.c_str(); }
extern "C" const char* emri_version(void) { return "emri-gb300 0.1 (sm_103a)"; }

extern "C" void emri_opts_default(emri_opts* o) {
  if (!o) return;
  o->precision = EMRI_FP64;
  o->n_max = 10;
  o->doppler = 1;
  o->pn_terms = 1;
  o->mode = EMRI_FORWARD;
  o->knot_spacing = 0;
  o->n_xi = 2.0;
  o->omega_m = 0.315;
  o->h0 = 67.4;
}

namespace emri {

static bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

int normalize_opts(const emri_opts* in, int64_t n, OptsN* o) {
  emri_opts d;
  emri_opts_default(&d);
  const emri_opts& a = in ? *in : d;
  if (a.precision != EMRI_FP64 && a.precision != EMRI_MIXED)
    return set_err(EMRI_EINVAL, "opts.precision must be EMRI_FP64 or EMRI_MIXED");
  if (a.n_max < 1 || a.n_max > 32) return set_err(EMRI_EINVAL, "opts.n_max must be in [1, 32]");
  if (a.mode != EMRI_FORWARD && a.mode != EMRI_BACKWARD_FROM_LSO)
    return set_err(EMRI_EINVAL, "opts.mode must be EMRI_FORWARD or EMRI_BACKWARD_FROM_LSO");
  o->precision = a.precision;
  o->n_max = a.n_max;
  o->doppler = a.doppler ? 1 : 0;
  o->pn_terms = a.pn_terms ? 1 : 0;
  o->mode = a.mode;
  int ks = a.knot_spacing;
  if (ks == 0) ks = a.precision == EMRI_FP64 ? 128 : 1024;
  if (!pow2(ks) || ks < 64 || ks > 1024 || ks > n)
    return set_err(EMRI_EINVAL, "opts.knot_spacing must be a power of two in [64, 1024] and <= n");
  o->ks = ks;
  o->n_xi = a.n_xi > 0 ? a.n_xi : 2.0;
  o->omega_m = a.omega_m > 0 ? a.omega_m : 0.315;
  o->h0 = a.h0 > 0 ? a.h0 : 67.4;
  if (!(o->omega_m > 0 && o->omega_m < 1)) return set_err(EMRI_EINVAL, "opts.omega_m must be in (0, 1)");
  return EMRI_OK;
}

int check_grid(const emri_grid* g) {
  if (!g) return set_err(EMRI_EINVAL, "grid is NULL");
  if (!pow2(g->n) || g->n < (1 << 10) || g->n > (1 << 22))
    return set_err(EMRI_EINVAL, "grid.n must be a power of two in [2^10, 2^22] (got %lld)", (long long)g->n);
  if (!(g->dt > 0) || !isfinite(g->dt)) return set_err(EMRI_EINVAL, "grid.dt must be positive");
  if (!isfinite(g->t0)) return set_err(EMRI_EINVAL, "grid.t0 must be finite");
  return EMRI_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_32 with the
// three-term recurrence; Abramowitz & Stegun 25.4.29).
static void gauss_legendre32(double* x, double* w) {
  const int n = 32;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Chebyshev-Picard integration tables for the orbit kernel: with the 32
// Chebyshev-Gauss-Lobatto nodes x_j = -cos(pi j/31) on [-1, 1] and the
// Lagrange basis l_j(x) = sum_k (2/(31 c_j c_k)) T_k(x_j) T_k(x)
// (c_0 = c_31 = 2, else 1), the weights
//   Q_j(x) = (1/2) int_{-1}^{x} l_j(s) ds   (unit segment, dtau = dx/2)
// at the nodes (qn, stored transposed: qn[j*32 + i]) and at the 129 knot
// positions x = -1 + 2q/128 (qk[q*32 + j]); long double, rounded once.
static void mcpi_tables(double* qn, double* qk) {
  typedef long double LD;
  const int m = 32;
  const LD pi = 3.141592653589793238462643383279502884L;
  LD xn[32], cc[32];
  for (int j = 0; j < m; ++j) {
    xn[j] = -cosl(pi * j / (m - 1));
    cc[j] = (j == 0 || j == m - 1) ? 2.0L : 1.0L;
  }
  auto cheb = [](int k, LD x) {
    LD t0 = 1, t1 = x;
    if (k == 0) return t0;
    for (int i = 2; i <= k; ++i) {
      LD t2 = 2 * x * t1 - t0;
      t0 = t1;
      t1 = t2;
    }
    return t1;
  };
  auto cint = [&](int k, LD x) {   // int_{-1}^{x} T_k
    if (k == 0) return x + 1;
    if (k == 1) return (x * x - 1) / 2;
    auto prim = [&](LD y) { return cheb(k + 1, y) / (2 * (k + 1)) - cheb(k - 1, y) / (2 * (k - 1)); };
    return prim(x) - prim(-1.0L);
  };
  auto weight = [&](int j, LD x) {
    LD acc = 0;
    for (int k = 0; k < m; ++k) acc += 2.0L / ((m - 1) * cc[j] * cc[k]) * cheb(k, xn[j]) * cint(k, x);
    return acc / 2;
  };
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) qn[j * 32 + i] = (double)weight(j, xn[i]);
  for (int q = 0; q <= 128; ++q)
    for (int j = 0; j < m; ++j) qk[q * 32 + j] = (double)weight(j, -1.0L + 2.0L * q / 128);
}

// ----------------------------------------------------------- workspace
int Workspace::reserve(emri_ctx* ctx, size_t bytes, cudaStream_t s) {
  if (bytes <= cap) return EMRI_OK;
  size_t want = std::max(bytes, cap + cap / 4);
  if (ptr) {
    cudaStreamSynchronize(last_stream);
    cudaFree(ptr);
    {
      std::lock_guard<std::mutex> lk(ctx->budget_mu);
      ctx->used -= cap;
    }
    ptr = nullptr;
    cap = 0;
  }
  {
    std::lock_guard<std::mutex> lk(ctx->budget_mu);
    if (ctx->used + want > ctx->budget) {
      want = bytes;
      if (ctx->used + want > ctx->budget)
        return set_err(EMRI_EBUDGET, "workspace of %zu bytes exceeds the HBM budget (%zu of %zu in use)", bytes,
                       ctx->used, ctx->budget);
    }
    ctx->used += want;   // charged before the allocation, returned on failure
  }
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    std::lock_guard<std::mutex> lk(ctx->budget_mu);
    ctx->used -= want;
    return set_err(EMRI_ENOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
  }
  cap = want;
  (void)s;
  return EMRI_OK;
}

void Workspace::acquire(cudaStream_t s) {
  if (!ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (has_ev && s != last_stream) cudaStreamWaitEvent(s, ev, 0);
  // debug aid: a kernel that reads workspace it did not write this call sees NaN
  if (poison && ptr) cudaMemsetAsync(ptr, 0xFF, cap, s);
}

void Workspace::release(cudaStream_t s) {
  cudaEventRecord(ev, s);
  has_ev = true;
  last_stream = s;
}

void Workspace::destroy(emri_ctx* ctx) {
  if (ptr) {
    cudaDeviceSynchronize();
    cudaFree(ptr);
    std::lock_guard<std::mutex> lk(ctx->budget_mu);
    ctx->used -= cap;
  }
  if (ev) cudaEventDestroy(ev);
  ptr = nullptr;
  cap = 0;
  ev = nullptr;
}

size_t loglike_layout(const FftPlan& p, const OptsN& o, int w, int wave, Carve* c, LoglikeBufs* b) {
  const int64_t nk = p.n / o.ks;
  const size_t cs = o.precision ? sizeof(float2) : sizeof(double2);
  Carve dummy(nullptr);
  Carve& cv = c ? *c : dummy;
  LoglikeBufs t;
  t.wc = cv.take<WalkerC>(w);
  t.knots = cv.take<Knot>((size_t)w * (nk + 1));
  t.ivs = cv.take<char>(o.precision ? (size_t)w * nk * kIvMBytes : 0);
  t.lisa = cv.take<double>((size_t)(p.n / 256) * 8);
  t.dtab = cv.take<char>((size_t)w * p.n1 * cs);
  t.rtab = cv.take<char>((size_t)w * p.n2 * cs);
  t.partial = cv.take<double2>((size_t)w * p.n2);
  t.z = cv.take<char>((size_t)wave * p.n * cs);
  if (b) *b = t;
  return cv.off + 256;
}

int pick_wave(emri_ctx* ctx, const FftPlan& p, const OptsN& o, int w) {
  const size_t cs = o.precision ? sizeof(float2) : sizeof(double2);
  const size_t per = (size_t)p.n * cs;
  int plan = ctx_plan_wave(ctx, p.n, o);
  if (plan > 0) return std::min({plan, w, kMaxGridY});
  // default: waves of up to 16 GiB of time series (and at most 65535
  // walkers, the kernels' grid y)
  size_t cap = (size_t)16 << 30;
  int wave = (int)std::max<size_t>(1, cap / per);
  return std::min({wave, w, kMaxGridY});
}

int pipe_groups(emri_ctx* ctx, const OptsN& o, cudaStream_t s) {
  const int g = ctx->pipe[o.precision ? 1 : 0];
  if (g == 1) return 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 1;
  return g;
}

// The context's two pipeline streams, both at the device's highest priority
// (a group's FFT passes are dispatched as soon as its waveform is written,
// ahead of the next group's waveform CTAs; at normal priority the schedule
// measured no faster than the sequential one), and the events of the
// schedule:
// [0] fork, [1] first group's orbits done, [2] waveform done / FFT join,
// [3] every orbit done,
// [4 + (wave & 1) kMaxPipe + q] group q of a wave has left the series buffer.
static int pipe_resources(emri_ctx* ctx) {
  if (ctx->pstream[1]) return EMRI_OK;
  int lo = 0, hi = 0;
  CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (ctx->pev.empty()) ctx->pev.assign(4 + 2 * kMaxPipe, nullptr);
  for (cudaEvent_t& e : ctx->pev)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i)
    if (!ctx->pstream[i]) CK(cudaStreamCreateWithPriority(&ctx->pstream[i], cudaStreamNonBlocking, hi));
  return EMRI_OK;
}

// The launch sequence of steps S0-S7 for W walkers of one dataset.
// pipe = 1: every step on s, in order (pipe = 0: 1 or 2 by the call's size,
// below).  pipe = G > 1: the prologue, delay tables and LISA tiles on s,
// then each wave's walkers in G groups whose orbits run on the context's
// first pipeline stream, waveforms on s, and FFT passes and reduction on the
// second, so group g's waveform can run beside group g-1's passes and the
// orbits of groups 1.. beside group 0's waveform.  Each walker is computed
// by the same kernels on the same data either way, so the results are
// bitwise the same for every G.
int run_loglike(emri_ctx* ctx, const emri_dataset* ds, const double* theta, int64_t ld, int w, const OptsN& o,
                int wave, const LoglikeBufs& b, double* lnl, double* dh, double* hh, uint32_t* status,
                cudaStream_t s, int64_t* launches, const FdW* fd, int pipe) {
  const FftPlan& p = ds->plan;
  const bool f32 = o.precision != 0;
  const size_t cs = f32 ? sizeof(float2) : sizeof(double2);
  int64_t nl = 0;
  Profiler* pf = &ctx->prof;
  const int64_t nk = p.n / o.ks;
  const void* dperm = f32 ? (const void*)ds->g_perm32 : (const void*)ds->g_perm;
  const void* wperm = f32 ? (const void*)ds->w_perm32 : (const void*)ds->w_perm;
  const double dh_scale = f32 ? 1.0 / (ds->d_scale * ds->w_scale) : 1.0;
  const double hh_scale = f32 ? 1.0 / ds->w_scale : 1.0;
  // steps S5-S7 of walkers [j0, j0 + gw), whose series start at zg
  auto passes = [&](int j0, int gw, char* zg, cudaStream_t st) {
    { KTimer t(pf, EMRI_K_FFT1, st); launch_fft_pass1(zg, gw, p, f32, -1, ctx->tw, st); }
    {
      KTimer t(pf, EMRI_K_FFT2_IP, st);
      launch_fft_pass2_ip(zg, gw, p, f32, ctx->tw, b.wc + j0, b.dtab + (size_t)j0 * p.n1 * cs,
                          b.rtab + (size_t)j0 * p.n2 * cs, dperm, wperm, b.partial + (size_t)j0 * p.n2, st,
                          fd ? fd + j0 : nullptr);
    }
    {
      KTimer t(pf, EMRI_K_FINALIZE, st);
      launch_finalize(b.partial + (size_t)j0 * p.n2, p.n2, b.wc + j0, gw, dh_scale, hh_scale, lnl + j0,
                      dh ? dh + j0 : nullptr, hh ? hh + j0 : nullptr, status ? status + j0 : nullptr, st);
    }
  };
  auto wave_of = [&](int j0, int gw, char* zg, cudaStream_t st) {
    KTimer t(pf, EMRI_K_WAVE, st);
    launch_wave(b.knots + (size_t)j0 * (nk + 1), b.wc + j0, gw, p.n, ds->dt, ds->t0, o, zg, false, ctx->bt,
                b.lisa, b.ivs + (size_t)j0 * nk * kIvMBytes, st);
  };
  auto orbit_of = [&](int j0, int gw, cudaStream_t st) {
    Knot* kj = b.knots + (size_t)j0 * (nk + 1);
    { KTimer t(pf, EMRI_K_ORBIT, st); launch_orbit(b.wc + j0, gw, p.n, ds->dt, ds->t0, o, kj, ctx->mcpi, st); }
    if (f32) {
      KTimer t(pf, EMRI_K_ORBIT, st);
      launch_intervals_mixed(kj, gw, p.n, o.ks, ds->dt, b.ivs + (size_t)j0 * nk * kIvMBytes, st);
    }
  };
  if (pipe == 0) {
    // by size: two groups when each holds at least 2^30 samples (walkers x
    // n).  On the 1024-walker 2^21 mixed step two groups take 44.5 against
    // 45.3 ms; smaller groups lose more to the extra orbit launch and the
    // stream hand-offs than the overlap gains (8 walkers: 2.5 -> 4.4 ms).
    const int64_t w1 = std::min(wave, w);
    pipe = w1 * p.n >= ((int64_t)1 << 31) ? 2 : 1;
  }
  { KTimer t(pf, EMRI_K_PROLOGUE, s); launch_prologue(theta, ld, w, p.n, ds->dt, o, ctx->gl, b.wc, s); }
  { KTimer t(pf, EMRI_K_DELAY, s); launch_delay_table(b.wc, w, p.n1, p.n2, f32, b.dtab, b.rtab, s); }
  if (pipe <= 1) {
    orbit_of(0, w, s);
    launch_lisa_tiles(p.n, ds->t0, ds->dt, b.lisa, s);
    nl += f32 ? 6 : 5;
    for (int i0 = 0; i0 < w; i0 += wave) {
      const int ww = std::min(wave, w - i0);
      wave_of(i0, ww, b.z, s);
      passes(i0, ww, b.z, s);
      nl += 4;
    }
  } else {
    int rc = pipe_resources(ctx);
    if (rc) return rc;
    launch_lisa_tiles(p.n, ds->t0, ds->dt, b.lisa, s);
    nl += 4;
    cudaStream_t so = ctx->pstream[0], sf = ctx->pstream[1];
    cudaEvent_t* ev = ctx->pev.data();
    cudaEventRecord(ev[0], s);
    cudaStreamWaitEvent(so, ev[0], 0);
    cudaStreamWaitEvent(sf, ev[0], 0);
    // orbits: the first group's alone, then every other walker's in one
    // launch that runs beside the first group's waveform (an orbit launch
    // takes about as long for a few walkers as for a thousand: each walker's
    // integration is sequential in time, so one launch per group would queue
    // G of those latencies)
    const int w1 = std::min(wave, w);
    const int g0 = (w1 + std::min(pipe, w1) - 1) / std::min(pipe, w1);
    orbit_of(0, g0, so);
    cudaEventRecord(ev[1], so);
    if (g0 < w) orbit_of(g0, w - g0, so);
    cudaEventRecord(ev[3], so);
    nl += f32 ? 2 : 1;
    if (g0 < w) nl += f32 ? 2 : 1;
    int prev_gs = 0, prev_g = 0;   // group size and count of the previous wave
    for (int i0 = 0, wv = 0; i0 < w; i0 += wave, ++wv) {
      const int ww = std::min(wave, w - i0);
      const int G = std::min(pipe, ww);
      const int gs = (ww + G - 1) / G;
      cudaEvent_t* gone = ev + 4 + (wv & 1) * kMaxPipe;        // this wave's groups
      cudaEvent_t* gone_prev = ev + 4 + ((wv + 1) & 1) * kMaxPipe;
      for (int q = 0, j0 = i0; j0 < i0 + ww; ++q, j0 += gs) {
        const int gw = std::min(gs, i0 + ww - j0);
        cudaStreamWaitEvent(s, j0 == 0 ? ev[1] : ev[3], 0);   // the group's orbits
        if (wv > 0) {   // the previous wave's groups that used this part of the series buffer
          const int qa = (j0 - i0) / prev_gs, qb = std::min((j0 - i0 + gw - 1) / prev_gs, prev_g - 1);
          for (int r = qa; r <= qb; ++r) cudaStreamWaitEvent(s, gone_prev[r], 0);
        }
        char* zg = b.z + (size_t)(j0 - i0) * p.n * cs;
        wave_of(j0, gw, zg, s);
        cudaEventRecord(ev[2], s);
        cudaStreamWaitEvent(sf, ev[2], 0);
        passes(j0, gw, zg, sf);
        cudaEventRecord(gone[q], sf);
        nl += 4;
      }
      prev_gs = gs;
      prev_g = (ww + gs - 1) / gs;
    }
    cudaStreamWaitEvent(s, ev[3], 0);
    cudaEventRecord(ev[2], sf);
    cudaStreamWaitEvent(s, ev[2], 0);
  }
  if (launches) *launches = nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "loglike launch");
  return EMRI_OK;
}

}  // namespace emri

// -------------------------------------------------------------- profiler
cudaEvent_t Profiler::get() {
  cudaEvent_t e;
  if (!pool.empty()) {
    e = pool.back();
    pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}

cudaEvent_t Profiler::begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu);
  cudaEvent_t e = get();
  cudaEventRecord(e, s);
  return e;
}

void Profiler::end(int kind, cudaEvent_t b, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu);
  cudaEvent_t e = get();
  cudaEventRecord(e, s);
  pending.emplace_back(kind, b, e);
}

void Profiler::drain() {
  std::lock_guard<std::mutex> lk(mu);
  for (auto& t : pending) {
    cudaEventSynchronize(std::get<2>(t));
    float m = 0.f;
    cudaEventElapsedTime(&m, std::get<1>(t), std::get<2>(t));
    ms[std::get<0>(t)] += m;
    count[std::get<0>(t)] += 1;
    pool.push_back(std::get<1>(t));
    pool.push_back(std::get<2>(t));
  }
  pending.clear();
}

void Profiler::reset() {
  drain();
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < EMRI_NKERNEL; ++i) {
    ms[i] = 0.0;
    count[i] = 0;
  }
}

extern "C" int emri_ctx_profile(emri_ctx* c, int enable) {
  if (!c) return set_err(EMRI_EINVAL, "NULL context");
  cudaSetDevice(c->device);
  c->prof.reset();
  c->prof.on = enable != 0;
  return EMRI_OK;
}

extern "C" int emri_ctx_kernel_times(emri_ctx* c, double* ms, int64_t* launches) {
  if (!c) return set_err(EMRI_EINVAL, "NULL context");
  cudaSetDevice(c->device);
  c->prof.drain();
  for (int i = 0; i < EMRI_NKERNEL; ++i) {
    if (ms) ms[i] = c->prof.ms[i];
    if (launches) launches[i] = c->prof.count[i];
  }
  return EMRI_OK;
}

// ===================================================================== ctx
extern "C" int emri_ctx_create(int device, size_t budget, emri_ctx** out) {
  if (!out) return set_err(EMRI_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return set_err(EMRI_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  if (device < 0 || device >= ndev) return set_err(EMRI_EINVAL, "device %d out of range (%d devices)", device, ndev);
  CK(cudaSetDevice(device));
  emri_ctx* c = new emri_ctx();
  c->device = device;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  c->budget = budget ? budget : (size_t)(0.8 * (double)fr);
  {
    const char* pz = getenv("EMRI_DEBUG_POISON");
    c->ws.poison = pz && pz[0] && pz[0] != '0';
  }
  c->used = 0;
  cudaError_t e2 = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e2 != cudaSuccess) {
    delete c;
    return cuda_err(e2, "cudaStreamCreate");
  }
  // twiddle and quadrature tables
  constexpr size_t kBc = (size_t)emri::kBesselOrders * emri::kBesselTerms;
  size_t tb = 4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8 + 64 * 8 + kBc * 12 + emri::kBesselOrders * 12 + 256 +
              (32 + 129) * 32 * 8 + 4096 * 16 + 16 + 4096 * 8;
  char* p = nullptr;
  e2 = cudaMalloc(&p, tb);
  if (e2 != cudaSuccess) {
    cudaStreamDestroy(c->stream);
    delete c;
    return cuda_err(e2, "cudaMalloc(tables)");
  }
  c->tables = p;
  c->used += tb;
  c->tw.ta64 = (double2*)p;
  c->tw.tb64 = (double2*)(p + 4096 * 16);
  c->tw.ta32 = (float2*)(p + 4096 * 16 + 1024 * 16);
  c->tw.tb32 = (float2*)(p + 4096 * 16 + 1024 * 16 + 4096 * 8);
  c->tw.tc64 = (double2*)(p + 4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8);   // 16-byte aligned offset
  c->gl = (double*)(p + 4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8 + 4096 * 16);
  {
    char* q = (char*)(c->gl + 64);
    constexpr size_t no = emri::kBesselOrders;
    c->bt.c64 = (double*)q;
    c->bt.f64 = (double*)(q + kBc * 8);
    c->bt.c32 = (float*)(q + kBc * 8 + no * 8);
    c->bt.f32 = (float*)(q + kBc * 8 + no * 8 + kBc * 4);
    size_t off = kBc * 12 + no * 12;
    off = (off + 7) & ~(size_t)7;   // 8-byte aligned (q is)
    c->mcpi = (double*)(q + off);
    // the FP32 stage twiddles after the orbit tables, 16-byte aligned
    const uintptr_t tt = ((uintptr_t)(c->mcpi + (32 + 129) * 32) + 15) & ~(uintptr_t)15;
    c->tw.tt32 = (float2*)tt;
  }
  double glh[64];
  gauss_legendre32(glh, glh + 32);
  {
    std::vector<double> mt((32 + 129) * 32);
    mcpi_tables(mt.data(), mt.data() + 32 * 32);
    cudaMemcpy(c->mcpi, mt.data(), mt.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  launch_twiddle_init(c->tw, c->stream);
  cudaMemcpyAsync(c->gl, glh, sizeof glh, cudaMemcpyHostToDevice, c->stream);
  fft_set_smem_limits();
  e2 = cudaStreamSynchronize(c->stream);
  if (e2 == cudaSuccess) e2 = cudaGetLastError();
  if (e2 == cudaSuccess && upload_exp512()) e2 = cudaErrorUnknown;
  if (e2 == cudaSuccess && emri::upload_bessel_tables(c->bt)) e2 = cudaErrorUnknown;
  if (e2 != cudaSuccess) {
    cudaFree(p);
    cudaStreamDestroy(c->stream);
    delete c;
    return cuda_err(e2, "context tables");
  }
  c->launches = 2;
  *out = c;
  return EMRI_OK;
}

extern "C" int emri_ctx_destroy(emri_ctx* c) {
  if (!c) return EMRI_OK;
  cudaSetDevice(c->device);
  serve_shutdown(c);
  multi_destroy(c);
  c->prof.on = false;
  c->prof.drain();
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->ws.destroy(c);
  if (c->tables) cudaFree(c->tables);
  for (cudaStream_t st : c->pstream)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : c->pev)
    if (e) cudaEventDestroy(e);
  cudaStreamDestroy(c->stream);
  delete c;
  return EMRI_OK;
}

extern "C" int emri_ctx_set_pipeline(emri_ctx* c, int precision, int groups) {
  if (!c) return set_err(EMRI_EINVAL, "NULL context");
  if (precision != EMRI_FP64 && precision != EMRI_MIXED) return set_err(EMRI_EINVAL, "unknown precision %d", precision);
  if (groups < 0 || groups > kMaxPipe) return set_err(EMRI_EINVAL, "groups must be in [0, %d]", kMaxPipe);
  std::lock_guard<std::mutex> lk(c->mu);
  c->pipe[precision == EMRI_MIXED ? 1 : 0] = groups;
  return EMRI_OK;
}

extern "C" int emri_ctx_launches(const emri_ctx* c, int64_t* count) {
  if (!c || !count) return set_err(EMRI_EINVAL, "NULL argument");
  *count = c->launches.load();
  return EMRI_OK;
}

extern "C" int emri_ctx_memory(const emri_ctx* c, size_t* used, size_t* budget) {
  if (!c) return set_err(EMRI_EINVAL, "NULL context");
  if (used) {
    std::lock_guard<std::mutex> blk(const_cast<emri_ctx*>(c)->budget_mu);
    *used = c->used;
  }
  if (budget) *budget = c->budget;
  return EMRI_OK;
}

// ================================================================= dataset
__global__ void k_absmax(const double* __restrict__ v, int64_t n, int stride2, unsigned long long* out) {
  // max |v| over n doubles (stride2 = 2: complex magnitudes), positive-double bit order
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = stride2 == 2 ? hypot(v[2 * i], v[2 * i + 1]) : fabs(v[i]);
    m = a > m ? a : m;
  }
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

extern "C" int emri_dataset_create(emri_ctx* ctx, const emri_grid* grid, const void* data, int kind,
                                   const double* psd, double fmin, double fmax, emri_dataset** out) {
  if (!ctx || !out || !data || !psd) return set_err(EMRI_EINVAL, "NULL argument");
  *out = nullptr;
  int rc = check_grid(grid);
  if (rc) return rc;
  if (kind != 0 && kind != 1) return set_err(EMRI_EINVAL, "data_kind must be 0 (spectrum) or 1 (time series)");
  if (!(fmax > fmin) || fmin < 0) return set_err(EMRI_EINVAL, "need 0 <= fmin < fmax");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const int64_t n = grid->n;
  emri_dataset* ds = new emri_dataset();
  ds->ctx = ctx;
  ds->n = n;
  ds->dt = grid->dt;
  ds->t0 = grid->t0;
  ds->fmin = fmin;
  ds->fmax = fmax;
  {
    auto it = ctx->fft_split.find(n);
    ds->plan = make_fft_plan(n, it == ctx->fft_split.end() ? 0 : it->second);
  }
  const size_t keep = (size_t)n * (16 + 8 + 8 + 4) + 1024;
  const size_t tmp = (size_t)n * (16 + 16 + 8) + (size_t)(n / 2 + 1) * 8 + 4096;
  {
    std::lock_guard<std::mutex> blk(ctx->budget_mu);
    if (ctx->used + keep + tmp > ctx->budget) {
      delete ds;
      return set_err(EMRI_EBUDGET, "dataset of %zu bytes exceeds the HBM budget", keep);
    }
  }
  char* kp = nullptr;
  char* tp = nullptr;
  cudaError_t e = cudaMalloc(&kp, keep);
  if (e == cudaSuccess) e = cudaMalloc(&tp, tmp);
  if (e != cudaSuccess) {
    cudaFree(kp);
    delete ds;
    return set_err(EMRI_ENOMEM, "dataset allocation: %s", cudaGetErrorString(e));
  }
  ds->mem = kp;
  ds->bytes = keep;
  {
    std::lock_guard<std::mutex> blk(ctx->budget_mu);
    ctx->used += keep;
  }
  Carve k(kp), t(tp);
  ds->g_perm = k.take<double2>(n);
  ds->w_perm = k.take<double>(n);
  ds->g_perm32 = k.take<float2>(n);
  ds->w_perm32 = k.take<float>(n);
  double2* dnat = t.take<double2>(n);
  double2* scratch = t.take<double2>(n);
  double* wnat = t.take<double>(n);
  double* psd_d = t.take<double>(n / 2 + 1);
  unsigned long long* mx = t.take<unsigned long long>(4);
  double* ddv = (double*)(mx + 2);
  cudaStream_t s = ctx->stream;
  int rc2 = EMRI_OK;
  do {
    if (kind == 0) {
      if ((e = cudaMemcpyAsync(dnat, data, (size_t)n * 16, cudaMemcpyDefault, s)) != cudaSuccess) break;
    } else {
      double* d2 = (double*)scratch;   // [2][n] doubles fit in the n-complex scratch
      if ((e = cudaMemcpyAsync(d2, data, (size_t)n * 16, cudaMemcpyDefault, s)) != cudaSuccess) break;
      launch_pack_time_series(d2, n, dnat, s);
      launch_fft_pass1(dnat, 1, ds->plan, false, -1, ctx->tw, s);
      launch_fft_pass2_store(dnat, scratch, 1, ds->plan, false, -1, ctx->tw, s);
      if ((e = cudaMemcpyAsync(dnat, scratch, (size_t)n * 16, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
    }
    if ((e = cudaMemcpyAsync(psd_d, psd, (size_t)(n / 2 + 1) * 8, cudaMemcpyDefault, s)) != cudaSuccess) break;
    launch_weights(psd_d, n, grid->dt, fmin, fmax, wnat, s);
    cudaMemsetAsync(mx, 0, 16, s);
    k_absmax<<<152, 256, 0, s>>>((const double*)dnat, n, 2, mx);
    k_absmax<<<152, 256, 0, s>>>(wnat, n, 1, mx + 1);
    unsigned long long hm[2];
    if ((e = cudaMemcpyAsync(hm, mx, 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    double dmax, wmax;
    memcpy(&dmax, &hm[0], 8);
    memcpy(&wmax, &hm[1], 8);
    if (!(wmax > 0) || !isfinite(wmax) || !isfinite(dmax)) {
      rc2 = set_err(EMRI_EINVAL, "dataset has no positive finite weight in the band or a non-finite value");
      break;
    }
    ds->d_scale = dmax > 0 ? 1.0 / dmax : 1.0;
    ds->w_scale = 1.0 / wmax;
    launch_dataset_permute(dnat, wnat, ds->plan, ds->g_perm, ds->w_perm, ds->g_perm32, ds->w_perm32, ds->d_scale,
                           ds->w_scale, s);
    launch_inner_dd(dnat, wnat, n, ddv, s);
    if ((e = cudaMemcpyAsync(&ds->dd, ddv, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    e = cudaGetLastError();
  } while (0);
  cudaFree(tp);
  if (e != cudaSuccess || rc2 != EMRI_OK) {
    {
      std::lock_guard<std::mutex> blk(ctx->budget_mu);
      ctx->used -= keep;
    }
    cudaFree(kp);
    delete ds;
    return rc2 != EMRI_OK ? rc2 : cuda_err(e, "dataset preparation");
  }
  ctx->launches += kind == 1 ? 9 : 6;
  *out = ds;
  return EMRI_OK;
}

extern "C" int emri_dataset_destroy(emri_dataset* ds) {
  if (!ds) return EMRI_OK;
  emri_ctx* c = ds->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(ds->mem);
  {
    std::lock_guard<std::mutex> blk(c->budget_mu);
    c->used -= ds->bytes;
  }
  delete ds;
  return EMRI_OK;
}

extern "C" int emri_dataset_dd(const emri_dataset* ds, double* dd_out) {
  if (!ds || !dd_out) return set_err(EMRI_EINVAL, "NULL argument");
  *dd_out = ds->dd;
  return EMRI_OK;
}

// =========================================================== batch calls
extern "C" int emri_prologue(emri_ctx* ctx, const emri_grid* grid, const double* theta, int w,
                             const emri_opts* opts, double* out, void* stream) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  int rc = check_grid(grid);
  if (rc) return rc;
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (!theta || !out) return set_err(EMRI_EINVAL, "NULL pointer");
  OptsN o;
  if ((rc = normalize_opts(opts, grid->n, &o))) return rc;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  size_t need = (size_t)w * sizeof(WalkerC) + 256;
  if ((rc = ctx->ws.reserve(ctx, need, s))) return rc;
  ctx->ws.acquire(s);
  WalkerC* wc = (WalkerC*)ctx->ws.ptr;
  launch_prologue(theta, w, w, grid->n, grid->dt, o, ctx->gl, wc, s);
  launch_prologue_export(wc, w, out, s);
  ctx->ws.release(s);
  ctx->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "prologue launch");
  return EMRI_OK;
}

extern "C" int emri_ak_waveform(emri_ctx* ctx, const emri_grid* grid, const double* theta, int w,
                                const emri_opts* opts, void* z_out, uint32_t* status, void* stream) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  int rc = check_grid(grid);
  if (rc) return rc;
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (!theta || !z_out) return set_err(EMRI_EINVAL, "NULL pointer");
  OptsN o;
  if ((rc = normalize_opts(opts, grid->n, &o))) return rc;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nk = grid->n / o.ks;
  Carve probe(nullptr);
  probe.take<WalkerC>(w);
  probe.take<Knot>((size_t)w * (nk + 1));
  probe.take<char>(o.precision ? (size_t)w * nk * kIvMBytes : 0);
  probe.take<double>((size_t)(grid->n / 256) * 8);
  if ((rc = ctx->ws.reserve(ctx, probe.off + 512, s))) return rc;
  ctx->ws.acquire(s);
  Carve cv(ctx->ws.ptr);
  WalkerC* wc = cv.take<WalkerC>(w);
  Knot* kn = cv.take<Knot>((size_t)w * (nk + 1));
  char* ivs = cv.take<char>(o.precision ? (size_t)w * nk * kIvMBytes : 0);
  double* lisa = cv.take<double>((size_t)(grid->n / 256) * 8);
  Profiler* pf = &ctx->prof;
  { KTimer t(pf, EMRI_K_PROLOGUE, s); launch_prologue(theta, w, w, grid->n, grid->dt, o, ctx->gl, wc, s); }
  { KTimer t(pf, EMRI_K_ORBIT, s); launch_orbit(wc, w, grid->n, grid->dt, grid->t0, o, kn, ctx->mcpi, s); }
  launch_lisa_tiles(grid->n, grid->t0, grid->dt, lisa, s);
  if (o.precision) launch_intervals_mixed(kn, w, grid->n, o.ks, grid->dt, ivs, s);
  { KTimer t(pf, EMRI_K_WAVE, s); launch_wave(kn, wc, w, grid->n, grid->dt, grid->t0, o, z_out, true, ctx->bt, lisa, ivs, s); }
  if (status) cudaMemcpy2DAsync(status, sizeof(uint32_t), &wc[0].status, sizeof(WalkerC), sizeof(uint32_t), w,
                                cudaMemcpyDeviceToDevice, s);
  ctx->ws.release(s);
  ctx->launches += o.precision ? 5 : 4;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "waveform launch");
  return EMRI_OK;
}

extern "C" int emri_fft_batch(emri_ctx* ctx, void* z, int64_t n, int batch, int precision, int direction,
                              void* stream) {
  if (!ctx) return set_err(EMRI_EINVAL, "NULL context");
  emri_grid g{n, 1.0, 0.0};
  int rc = check_grid(&g);
  if (rc) return rc;
  if (batch < 0) return set_err(EMRI_EINVAL, "batch must be >= 0");
  if (precision != EMRI_FP64 && precision != EMRI_MIXED) return set_err(EMRI_EINVAL, "bad precision");
  if (direction != -1 && direction != 1) return set_err(EMRI_EINVAL, "direction must be -1 or +1");
  if (batch == 0) return EMRI_OK;
  if (!z) return set_err(EMRI_EINVAL, "NULL pointer");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool f32 = precision == EMRI_MIXED;
  const size_t cs = f32 ? 8 : 16;
  const FftPlan p = make_fft_plan(n);
  // at most 1 GiB of scratch, and at most 65535 sequences (the passes' grid y)
  const int chunk = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)batch, ((int64_t)1 << 30) / ((int64_t)n * (int64_t)cs), (int64_t)kMaxGridY}));
  if ((rc = ctx->ws.reserve(ctx, (size_t)chunk * n * cs + 256, s))) return rc;
  ctx->ws.acquire(s);
  int64_t nl = 0;
  cudaError_t e = cudaSuccess;
  for (int b0 = 0; b0 < batch && e == cudaSuccess; b0 += chunk) {
    const int bb = std::min(chunk, batch - b0);
    char* zb = (char*)z + (size_t)b0 * n * cs;
    launch_fft_pass1(zb, bb, p, f32, direction, ctx->tw, s);
    launch_fft_pass2_store(zb, ctx->ws.ptr, bb, p, f32, direction, ctx->tw, s);
    e = cudaMemcpyAsync(zb, ctx->ws.ptr, (size_t)bb * n * cs, cudaMemcpyDeviceToDevice, s);
    nl += 2;
  }
  ctx->ws.release(s);
  ctx->launches += nl;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "fft launch");
  return EMRI_OK;
}

extern "C" int emri_loglike_batch(emri_ctx* ctx, const emri_dataset* ds, const double* theta, int w,
                                  const emri_opts* opts, double* lnl, double* dh, double* hh, uint32_t* status,
                                  void* stream) {
  if (!ctx || !ds) return set_err(EMRI_EINVAL, "NULL context or dataset");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (!theta || !lnl) return set_err(EMRI_EINVAL, "NULL pointer");
  OptsN o;
  int rc = normalize_opts(opts, ds->n, &o);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!(opts && opts->knot_spacing)) {
    const int pk = ctx_plan_ks(ctx, ds->n, o);
    if (pk) o.ks = pk;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int wave = pick_wave(ctx, ds->plan, o, w);
  const size_t need = loglike_layout(ds->plan, o, w, wave, nullptr, nullptr);
  if ((rc = ctx->ws.reserve(ctx, need, s))) return rc;
  ctx->ws.acquire(s);
  Carve cv(ctx->ws.ptr);
  LoglikeBufs b;
  loglike_layout(ds->plan, o, w, wave, &cv, &b);
  int64_t nl = 0;
  rc = run_loglike(ctx, ds, theta, w, w, o, wave, b, lnl, dh, hh, status, s, &nl, nullptr, pipe_groups(ctx, o, s));
  ctx->ws.release(s);
  ctx->launches += nl;
  return rc;
}

extern "C" int emri_loglike_batch_fd(emri_ctx* ctx, const emri_dataset* ds, const double* theta, int w,
                                     const emri_opts* opts, const emri_fdprop* fd, double* lnl, double* dh,
                                     double* hh, uint32_t* status, void* stream) {
  if (!ctx || !ds || !fd) return set_err(EMRI_EINVAL, "NULL context, dataset or propagation model");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (fd->q_m < 0 || fd->q_m > 3 || fd->q_t < 0 || fd->q_t > 3)
    return set_err(EMRI_EINVAL, "q_m and q_t must be in [0, 3]");
  if (!(fd->f_star > 0) || !isfinite(fd->f_star)) return set_err(EMRI_EINVAL, "f_star must be positive and finite");
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (!theta || !lnl || (fd->q_m + fd->q_t > 0 && !fd->coef_dev)) return set_err(EMRI_EINVAL, "NULL pointer");
  OptsN o;
  int rc = normalize_opts(opts, ds->n, &o);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!(opts && opts->knot_spacing)) {
    const int pk = ctx_plan_ks(ctx, ds->n, o);
    if (pk) o.ks = pk;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int wave = pick_wave(ctx, ds->plan, o, w);
  Carve probe(nullptr);
  probe.take<FdW>(w);
  probe.off = (probe.off + 255) & ~(size_t)255;
  const size_t need = probe.off + loglike_layout(ds->plan, o, w, wave, nullptr, nullptr);
  if ((rc = ctx->ws.reserve(ctx, need, s))) return rc;
  ctx->ws.acquire(s);
  Carve cv(ctx->ws.ptr);
  FdW* fdw = cv.take<FdW>(w);
  LoglikeBufs b;
  loglike_layout(ds->plan, o, w, wave, &cv, &b);
  launch_fdprop(theta, w, w, ds->n, ds->dt, o, fd->q_m, fd->q_t, fd->f_star, fd->coef_dev, w, fdw, s);
  int64_t nl = 1;
  int64_t nr = 0;
  rc = run_loglike(ctx, ds, theta, w, w, o, wave, b, lnl, dh, hh, status, s, &nr, fdw, pipe_groups(ctx, o, s));
  ctx->ws.release(s);
  ctx->launches += nl + nr;
  return rc;
}
