// k_mcmc.cu -- one affine-invariant ensemble step on the device.
//
// The paper samples the posterior with an affine-invariant ensemble sampler
// (Sec. 3, "Posterior sampling": emcee, after Goodman & Weare 2010); each of
// its steps evaluates the likelihood of every walker's proposal, which is the
// batched likelihood path of this library.  emri_stretch_step keeps the whole
// step on the GPU: for each half of the ensemble a propose kernel forms the
// stretch-move proposals Y = X_j + z (X_k - X_j), the likelihood path
// evaluates them (steps S0-S7), and an accept kernel applies the
// Metropolis-Hastings rule with the z^(d-1) factor of the stretch move.  No
// host synchronisation happens inside a step; the uniforms that drive it are
// inputs, drawn by the caller.
//
// The proposal and the acceptance margin are evaluated with explicitly
// rounded operations (no fused multiply-add), in the same order as the plain
// definition, so that a proposal is bit-identical to the textbook formula.
#include <math.h>

#include <algorithm>

#include "../../include/emri.h"
#include "emri_api_internal.h"
#include "emri_common.cuh"
#include "emri_internal.h"

using namespace emri;

namespace {

constexpr uint32_t kInvalid = ST_BADPARAM | ST_NONFINITE;

struct StretchArgs {
  double a;
  uint32_t free_mask;
  int d;
  double lo[kNParam], hi[kNParam];
};

// Proposals of the active half [a0, a0 + m) against the other half
// [o0, o0 + nc); Y is [P][m].
__global__ void k_stretch_propose(const double* __restrict__ theta, int64_t w, int a0, int m, int o0, int nc,
                                  const double* __restrict__ u, StretchArgs sa, double* __restrict__ y,
                                  double* __restrict__ zs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int k = a0 + i;
  int jj = (int)__dmul_rn(u[k], (double)nc);
  if (jj > nc - 1) jj = nc - 1;
  if (jj < 0) jj = 0;
  const int j = o0 + jj;
  const double t = __dadd_rn(__dmul_rn(sa.a - 1.0, u[w + k]), 1.0);
  const double z = __ddiv_rn(__dmul_rn(t, t), sa.a);
  zs[i] = z;
#pragma unroll
  for (int p = 0; p < kNParam; ++p) {
    const double xk = theta[(int64_t)p * w + k];
    double v = xk;
    if ((sa.free_mask >> p) & 1u) {
      const double xj = theta[(int64_t)p * w + j];
      v = __dadd_rn(xj, __dmul_rn(z, __dsub_rn(xk, xj)));
    }
    y[(int64_t)p * m + i] = v;
  }
}

__global__ void k_stretch_accept(double* __restrict__ theta, double* __restrict__ lnp, int64_t w, int a0, int m,
                                 const double* __restrict__ y, const double* __restrict__ zs,
                                 const double* __restrict__ lly, const uint32_t* __restrict__ sty,
                                 const double* __restrict__ u, StretchArgs sa, int32_t* __restrict__ accepted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int k = a0 + i;
  bool ok = !(sty[i] & kInvalid) && isfinite(lly[i]);
#pragma unroll
  for (int p = 0; p < kNParam; ++p) {
    if ((sa.free_mask >> p) & 1u) {
      const double v = y[(int64_t)p * m + i];
      ok = ok && v >= sa.lo[p] && v <= sa.hi[p];
    }
  }
  int acc = 0;
  if (ok) {
    const double lz = __dmul_rn((double)(sa.d - 1), log(zs[i]));
    const double margin = __dsub_rn(__dsub_rn(__dadd_rn(lz, lly[i]), lnp[k]), log(u[2 * w + k]));
    if (margin > 0.0) {
      acc = 1;
#pragma unroll
      for (int p = 0; p < kNParam; ++p) theta[(int64_t)p * w + k] = y[(int64_t)p * m + i];
      lnp[k] = lly[i];
    }
  }
  if (accepted) accepted[k] = acc;
}

}  // namespace

namespace {

// Validated stretch-move arguments of a configuration.
int stretch_args(const emri_stretch_cfg* cfg, StretchArgs* sa) {
  if (!(cfg->a > 1.0) || !isfinite(cfg->a)) return set_err(EMRI_EINVAL, "stretch scale a must be finite and > 1");
  *sa = StretchArgs{};
  sa->a = cfg->a;
  sa->free_mask = cfg->free_mask & ((1u << kNParam) - 1u);
  if (sa->free_mask != cfg->free_mask)
    return set_err(EMRI_EINVAL, "free_mask has bits above parameter %d", kNParam - 1);
  if (!sa->free_mask) return set_err(EMRI_EINVAL, "free_mask selects no parameter");
  sa->d = __builtin_popcount(sa->free_mask);
  for (int p = 0; p < kNParam; ++p) {
    sa->lo[p] = cfg->lo[p];
    sa->hi[p] = cfg->hi[p];
    if (((sa->free_mask >> p) & 1u) && !(cfg->lo[p] <= cfg->hi[p]))
      return set_err(EMRI_EINVAL, "prior box of parameter %d is empty or NaN", p);
  }
  return EMRI_OK;
}

// The walkers k0 <= k < k1 of halves first..last, each half against the
// whole other half of theta, the halves in order (half 0 = [0, W/2),
// half 1 = [W/2, W)).
int stretch_run(emri_ctx* ctx, const emri_dataset* ds, double* theta, double* lnp, int w, const emri_opts* opts,
                const StretchArgs& sa, const double* u, int32_t* accepted, cudaStream_t s, int first, int last,
                int k0, int k1, const emri_fdprop* fd) {
  OptsN o;
  int rc = normalize_opts(opts, ds->n, &o);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!(opts && opts->knot_spacing)) {
    const int pk = ctx_plan_ks(ctx, ds->n, o);
    if (pk) o.ks = pk;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(EMRI_ECUDA, "cudaSetDevice");
  const int h = w / 2;
  auto block = [&](int half, int* a0, int* m) {
    const int lo = half == 0 ? 0 : h, hi = half == 0 ? h : w;
    *a0 = std::max(lo, k0);
    *m = std::max(0, std::min(hi, k1) - *a0);
  };
  int mmax = 0;
  for (int half = first; half <= last; ++half) {
    int a0, m;
    block(half, &a0, &m);
    mmax = std::max(mmax, m);
  }
  if (mmax == 0) return EMRI_OK;
  const int wave = pick_wave(ctx, ds->plan, o, mmax);
  // workspace: proposals Y[P][m], z[m], lnL(Y)[m], status(Y)[m], then the likelihood buffers
  Carve probe(nullptr);
  probe.take<double>((size_t)kNParam * mmax);
  probe.take<double>(mmax);
  probe.take<double>(mmax);
  probe.take<uint32_t>(mmax);
  if (fd) probe.take<FdW>(mmax);
  probe.off = (probe.off + 255) & ~(size_t)255;
  const size_t need = probe.off + loglike_layout(ds->plan, o, mmax, wave, nullptr, nullptr);
  if ((rc = ctx->ws.reserve(ctx, need, s))) return rc;
  ctx->ws.acquire(s);
  Carve cv(ctx->ws.ptr);
  double* y = cv.take<double>((size_t)kNParam * mmax);
  double* zs = cv.take<double>(mmax);
  double* lly = cv.take<double>(mmax);
  uint32_t* sty = cv.take<uint32_t>(mmax);
  FdW* fdw = fd ? cv.take<FdW>(mmax) : nullptr;
  LoglikeBufs b;
  loglike_layout(ds->plan, o, mmax, wave, &cv, &b);
  int64_t nl = 0;
  for (int half = first; half <= last && rc == EMRI_OK; ++half) {
    int a0, m;
    block(half, &a0, &m);
    const int o0 = half == 0 ? h : 0, nc = half == 0 ? w - h : h;
    if (m == 0 || nc == 0) continue;
    const int tb = 128, gb = (m + tb - 1) / tb;
    k_stretch_propose<<<gb, tb, 0, s>>>(theta, w, a0, m, o0, nc, u, sa, y, zs);
    if (fd) {   // each proposal with its walker's propagation coefficients
      launch_fdprop(y, m, m, ds->n, ds->dt, o, fd->q_m, fd->q_t, fd->f_star, fd->coef_dev + a0, w, fdw, s);
      nl += 1;
    }
    rc = run_loglike(ctx, ds, y, m, m, o, std::min(wave, m), b, lly, nullptr, nullptr, sty, s, &nl, fdw,
                     pipe_groups(ctx, o, s));
    k_stretch_accept<<<gb, tb, 0, s>>>(theta, lnp, w, a0, m, y, zs, lly, sty, u, sa, accepted);
    nl += 2;
  }
  ctx->ws.release(s);
  ctx->launches += nl;
  if (rc) return rc;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "stretch step launch");
  return EMRI_OK;
}

}  // namespace

extern "C" int emri_stretch_step(emri_ctx* ctx, const emri_dataset* ds, double* theta, double* lnp, int w,
                                 const emri_opts* opts, const emri_stretch_cfg* cfg, const double* u,
                                 int32_t* accepted, void* stream) {
  if (!ctx || !ds || !cfg) return set_err(EMRI_EINVAL, "NULL context, dataset or configuration");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (w < 2) return set_err(EMRI_EINVAL, "the stretch move needs at least 2 walkers");
  if (!theta || !lnp || !u) return set_err(EMRI_EINVAL, "NULL pointer");
  StretchArgs sa;
  int rc = stretch_args(cfg, &sa);
  if (rc) return rc;
  return stretch_run(ctx, ds, theta, lnp, w, opts, sa, u, accepted, (cudaStream_t)stream, 0, 1, 0, w, nullptr);
}

static int check_fd(const emri_fdprop* fd) {
  if (!fd) return EMRI_OK;
  if (fd->q_m < 0 || fd->q_m > 3 || fd->q_t < 0 || fd->q_t > 3)
    return set_err(EMRI_EINVAL, "q_m and q_t must be in [0, 3]");
  if (!(fd->f_star > 0) || !isfinite(fd->f_star)) return set_err(EMRI_EINVAL, "f_star must be positive and finite");
  if (fd->q_m + fd->q_t > 0 && !fd->coef_dev) return set_err(EMRI_EINVAL, "NULL propagation coefficients");
  return EMRI_OK;
}

extern "C" int emri_stretch_step_fd(emri_ctx* ctx, const emri_dataset* ds, double* theta, double* lnp, int w,
                                    const emri_opts* opts, const emri_stretch_cfg* cfg, const emri_fdprop* fd,
                                    const double* u, int32_t* accepted, void* stream) {
  if (!ctx || !ds || !cfg || !fd) return set_err(EMRI_EINVAL, "NULL context, dataset, configuration or model");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 0) return set_err(EMRI_EINVAL, "w must be >= 0");
  if (w == 0) return EMRI_OK;
  if (w < 2) return set_err(EMRI_EINVAL, "the stretch move needs at least 2 walkers");
  if (!theta || !lnp || !u) return set_err(EMRI_EINVAL, "NULL pointer");
  int rc = check_fd(fd);
  if (rc) return rc;
  StretchArgs sa;
  if ((rc = stretch_args(cfg, &sa))) return rc;
  return stretch_run(ctx, ds, theta, lnp, w, opts, sa, u, accepted, (cudaStream_t)stream, 0, 1, 0, w, fd);
}

extern "C" int emri_stretch_half(emri_ctx* ctx, const emri_dataset* ds, double* theta, double* lnp, int w, int half,
                                 int k0, int k1, const emri_opts* opts, const emri_stretch_cfg* cfg,
                                 const emri_fdprop* fd, const double* u, int32_t* accepted, void* stream) {
  if (!ctx || !ds || !cfg) return set_err(EMRI_EINVAL, "NULL context, dataset or configuration");
  if (ds->ctx != ctx) return set_err(EMRI_EINVAL, "dataset belongs to another context");
  if (w < 2) return set_err(EMRI_EINVAL, "the stretch move needs at least 2 walkers");
  if (half != 0 && half != 1) return set_err(EMRI_EINVAL, "half must be 0 or 1");
  const int lo = half == 0 ? 0 : w / 2, hi = half == 0 ? w / 2 : w;
  if (k0 < lo || k1 > hi || k0 > k1)
    return set_err(EMRI_EINVAL, "walker block [%d, %d) is not inside half %d = [%d, %d)", k0, k1, half, lo, hi);
  if (k0 == k1) return EMRI_OK;
  if (!theta || !lnp || !u) return set_err(EMRI_EINVAL, "NULL pointer");
  int rc = check_fd(fd);
  if (rc) return rc;
  StretchArgs sa;
  if ((rc = stretch_args(cfg, &sa))) return rc;
  return stretch_run(ctx, ds, theta, lnp, w, opts, sa, u, accepted, (cudaStream_t)stream, half, half, k0, k1, fd);
}
