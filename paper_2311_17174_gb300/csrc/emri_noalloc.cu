// emri_noalloc.cu -- emri_fft_batch_noalloc: the batched FFT of
// emri_fft_batch for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or must not be
// called -- a plugin that may only use memory its host application hands it,
// a process whose device memory is already fully reserved by another
// allocator, or a real-time loop that must never enter the allocator.  Such
// callers cannot create an emri_ctx (its creation allocates tables and
// workspaces), so this entry point takes no context at all.
//
// How: the FFT's second pass writes out of place into scratch memory.  That
// scratch (32 MiB, at least one whole sequence: 2^21 double2 or 2^22 float2
// values, and several sequences per pass when they are shorter) and the
// twiddle tables the passes read are file-scope static device arrays of
// fixed size, present on every GPU that loads the library until the process
// exits.  Their device addresses are looked up once per device
// (cudaGetSymbolAddress, with that device current) the first time the entry
// point runs there; that first call also fills the twiddle tables and
// synchronises the stream, so it must not be made while the stream is being
// captured (it is refused with EMRI_EINVAL then; later calls may be).
// Nothing here calls cudaMalloc, cudaFree or an allocating
// library routine.  Every call on a device shares the same scratch, so calls
// whose work overlaps on the GPU (different streams, or host threads without
// ordering) race; the scratch is fully overwritten by each call, so nothing
// in it needs clearing.
#include <mutex>

#include "../../include/emri.h"
#include "emri_api_internal.h"
#include "emri_common.cuh"
#include "emri_internal.h"

using namespace emri;

// Scratch of EMRI_NOALLOC_SCRATCH_BYTES (32 MiB): at least one sequence
// (2^21 double2 or 2^22 float2 values), more when they are shorter.
static __device__ __align__(256) unsigned char g_noalloc_scratch[EMRI_NOALLOC_SCRATCH_BYTES];
// Twiddle tables: ta64[4096], tb64[1024], ta32[4096], tb32[1024], tc64[4096], tt32[4096].
static __device__ __align__(256) unsigned char g_noalloc_tables[4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8 +
                                                                4096 * 16 + 4096 * 8];

namespace {

constexpr int kMaxDevices = 64;

struct DevState {
  bool ready = false;
  unsigned char* scratch = nullptr;
  Twiddles tw{};
};

std::mutex g_mu;
DevState g_dev[kMaxDevices];

// Resolve the arrays' device addresses on the current device and fill the
// twiddle tables (first call on a device only).
int setup_device(int dev, cudaStream_t s, DevState** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& st = g_dev[dev];
  if (!st.ready) {
    // the set-up below synchronises the stream, which a capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
      return set_err(EMRI_EINVAL,
                     "emri_fft_batch_noalloc: the first call on a device sets up its tables and must not be made "
                     "while the stream is being captured");
    void* sp = nullptr;
    void* tp = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&sp, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
    e = cudaGetSymbolAddress(&tp, g_noalloc_tables);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(tables)");
    unsigned char* t = (unsigned char*)tp;
    st.tw.ta64 = (double2*)t;
    st.tw.tb64 = (double2*)(t + 4096 * 16);
    st.tw.ta32 = (float2*)(t + 4096 * 16 + 1024 * 16);
    st.tw.tb32 = (float2*)(t + 4096 * 16 + 1024 * 16 + 4096 * 8);
    st.tw.tc64 = (double2*)(t + 4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8);
    st.tw.tt32 = (float2*)(t + 4096 * 16 + 1024 * 16 + 4096 * 8 + 1024 * 8 + 4096 * 16);
    launch_twiddle_init(st.tw, s);
    fft_set_smem_limits();
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "no-alloc FFT set-up");
    st.scratch = (unsigned char*)sp;
    st.ready = true;
  }
  *out = &st;
  return EMRI_OK;
}

}  // namespace

extern "C" int emri_fft_batch_noalloc(void* z, int64_t n, int batch, int precision, int direction, void* stream) {
  emri_grid g{n, 1.0, 0.0};
  int rc = check_grid(&g);
  if (rc) return rc;
  if (batch < 0) return set_err(EMRI_EINVAL, "batch must be >= 0");
  if (precision != EMRI_FP64 && precision != EMRI_MIXED) return set_err(EMRI_EINVAL, "bad precision");
  if (direction != -1 && direction != 1) return set_err(EMRI_EINVAL, "direction must be -1 or +1");
  const size_t cs = precision == EMRI_MIXED ? sizeof(float2) : sizeof(double2);
  if ((size_t)n * cs > (size_t)EMRI_NOALLOC_SCRATCH_BYTES)
    return set_err(EMRI_EINVAL,
                   "emri_fft_batch_noalloc: one sequence of %lld %s values (%zu bytes) exceeds the fixed scratch of "
                   "%u bytes; use emri_fft_batch",
                   (long long)n, precision == EMRI_MIXED ? "float2" : "double2", (size_t)n * cs,
                   (unsigned)EMRI_NOALLOC_SCRATCH_BYTES);
  if (batch == 0) return EMRI_OK;
  if (!z) return set_err(EMRI_EINVAL, "NULL pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_err(EMRI_EINVAL, "device index %d not supported", dev);
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = nullptr;
  if ((rc = setup_device(dev, s, &st))) return rc;
  const bool f32 = precision == EMRI_MIXED;
  const FftPlan p = make_fft_plan(n);
  const int chunk = (int)((size_t)EMRI_NOALLOC_SCRATCH_BYTES / ((size_t)n * cs));
  for (int b0 = 0; b0 < batch; b0 += chunk) {
    const int bb = batch - b0 < chunk ? batch - b0 : chunk;
    char* zb = (char*)z + (size_t)b0 * n * cs;
    launch_fft_pass1(zb, bb, p, f32, direction, st->tw, s);
    launch_fft_pass2_store(zb, st->scratch, bb, p, f32, direction, st->tw, s);
    e = cudaMemcpyAsync(zb, st->scratch, (size_t)bb * n * cs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(e, "no-alloc FFT copy-back");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "no-alloc FFT launch");
  return EMRI_OK;
}
