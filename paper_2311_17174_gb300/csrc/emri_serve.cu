// emri_serve.cu -- placeholder for serving, autotuning and multi-chain launches.
#include "../../include/emri.h"
#include "emri_api_internal.h"
#include "emri_common.cuh"

using namespace emri;

namespace emri {
int ctx_plan_wave(emri_ctx* ctx, int64_t n, const OptsN& o) {
  auto it = ctx->plans.find(std::make_tuple(n, o.n_max, o.precision));
  return it == ctx->plans.end() ? 0 : it->second.wave;
}
void serve_shutdown(emri_ctx*) {}
}  // namespace emri

extern "C" int emri_loglike_multi(emri_ctx*, const emri_work*, int, void*) { return set_err(EMRI_EINVAL, "not built"); }
extern "C" int emri_serve_start(emri_ctx*, const emri_serve_cfg*) { return set_err(EMRI_EINVAL, "not built"); }
extern "C" int emri_serve_stop(emri_ctx*) { return set_err(EMRI_EINVAL, "not built"); }
extern "C" int emri_serve_submit(emri_ctx*, const emri_dataset*, const double*, int, const emri_opts*, uint64_t*) { return set_err(EMRI_EINVAL, "not built"); }
extern "C" int emri_serve_poll(emri_ctx*, uint64_t, double*, uint32_t*, emri_req_stats*, int64_t) { return set_err(EMRI_EINVAL, "not built"); }
extern "C" int emri_autotune(emri_ctx*, const emri_grid*, int, int, const char*, int64_t*) { return set_err(EMRI_EINVAL, "not built"); }
