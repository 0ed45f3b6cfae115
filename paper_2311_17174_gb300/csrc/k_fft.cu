// k_fft.cu -- steps S5-S7: batched FFT and the fused noise-weighted inner
// products (paper Sec. 3: the time-domain waveform is Fourier transformed and
// compared with the data through the likelihood of Eq. (8)).
//
// n = n1 * n2 (four-step): element j = j1 + n1 j2, bin k = k2 + n2 k1.
//  pass 1: for each column j1, the n2-point DFT over j2, times the twiddle
//          exp(-2 pi i j1 k2 / n), written back in place (position j1 + n1 k2);
//  pass 2: for each row k2, the n1-point DFT over j1 gives bins k2 + n2 k1.
// Both passes are shared-memory Stockham FFTs (radix-4 stages, one radix-2
// stage when log2 of the length is odd), one CTA per column group / row.
// The likelihood path never writes the spectrum: pass 2 multiplies each bin
// by the GW-speed delay factor and accumulates
//   sum_k w_k Re(conj(D_k) H_k e^{-2 pi i k_s r})  and  sum_k w_k |H_k|^2
// against the data and weights stored in the same (k2-major) order, and
// writes one pair of partial sums per row.  A final kernel adds a walker's
// rows in a fixed order, so results are bitwise independent of the batch.
// Twiddles come from two FP64-built tables:
//   ta[i] = exp(-2 pi i i / 4096), tb[i] = exp(-2 pi i i / 2^22),
// exp(-2 pi i m / 2^22) = ta[m >> 10] * tb[m & 1023].
#include "emri_common.cuh"
#include "emri_internal.h"

namespace emri {

constexpr int kFftThreads = 512;   // pass 1 (column groups)
constexpr int kPass2Threads = 256; // pass 2 (rows)

FftPlan make_fft_plan(int64_t n) {
  FftPlan p;
  p.n = n;
  int m = 0;
  while ((int64_t(1) << m) < n) ++m;
  p.log2n = m;
  int m2 = m / 2 < 10 ? m / 2 : 10;
  p.n2 = 1 << m2;
  p.n1 = (int)(n >> m2);
  return p;
}

// ------------------------------------------------------------ twiddles
__global__ void k_twiddle_init(double2* ta64, double2* tb64, float2* ta32, float2* tb32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 4096) {
    double s, c;
    sincospi(-2.0 * (double)i / 4096.0, &s, &c);
    ta64[i] = make_double2(c, s);
    ta32[i] = make_float2((float)c, (float)s);
  }
  if (i < 1024) {
    double s, c;
    sincospi(-2.0 * (double)i / 4194304.0, &s, &c);
    tb64[i] = make_double2(c, s);
    tb32[i] = make_float2((float)c, (float)s);
  }
}

void launch_twiddle_init(Twiddles t, cudaStream_t s) {
  k_twiddle_init<<<16, 256, 0, s>>>(t.ta64, t.tb64, t.ta32, t.tb32);
}

// ----------------------------------------------------- complex helpers
template <typename C2>
struct CT;
template <>
struct CT<double2> {
  using T = double;
  __device__ static double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct CT<float2> {
  using T = float;
  __device__ static float2 make(float x, float y) { return make_float2(x, y); }
};

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return CT<C2>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C2>
__device__ __forceinline__ C2 cadd(C2 a, C2 b) {
  return CT<C2>::make(a.x + b.x, a.y + b.y);
}
template <typename C2>
__device__ __forceinline__ C2 csub(C2 a, C2 b) {
  return CT<C2>::make(a.x - b.x, a.y - b.y);
}
template <typename C2>
__device__ __forceinline__ C2 conj_if(C2 a, int sign) {
  return sign > 0 ? CT<C2>::make(a.x, -a.y) : a;
}

// exp(sign * 2 pi i * m / 2^22), m < 2^22
template <typename C2>
__device__ __forceinline__ C2 twiddle22(const C2* __restrict__ ta, const C2* __restrict__ tb, uint32_t m,
                                        int sign) {
  return conj_if(cmul(ta[m >> 10], tb[m & 1023u]), sign);
}

// ------------------------------------------------- shared-memory Stockham
// nb transforms of length L (power of two, <= 4096); element i of transform
// c lives at buf[i*sj + c*sc].  Butterfly b works on transform b % nb, so
// consecutive threads touch consecutive transforms when sc = 1 (row-major
// tiles: conflict-free) or consecutive elements when nb = 1.  Each thread
// stages its outputs in registers so a stage reads everything before
// anything is overwritten.
template <typename C2, int MAXB>
__device__ void smem_fft(C2* buf, int L, int nb, int sj, int sc, int sign, const C2* __restrict__ ta) {
  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  const int nr4 = lg / 2;
  int ns = 1;
  for (int st = 0; st < nr4; ++st) {
    const int q4 = L / 4;
    const int nbf = nb * q4;
    C2 y[MAXB][4];
    int dst[MAXB];
#pragma unroll
    for (int r = 0; r < MAXB; ++r) {
      const int b = tid + r * nth;
      dst[r] = -1;
      if (b < nbf) {
        const int c = b % nb, j = b / nb;
        const int k = j & (ns - 1);
        C2* col = buf + c * sc;
        C2 a0 = col[j * sj], a1 = col[(j + q4) * sj], a2 = col[(j + 2 * q4) * sj], a3 = col[(j + 3 * q4) * sj];
        if (ns > 1) {
          const int u = (k * 4096) / (ns * 4);   // twiddle step in 1/4096 cycles
          a1 = cmul(a1, conj_if(ta[u], sign));
          a2 = cmul(a2, conj_if(ta[(2 * u) & 4095], sign));
          a3 = cmul(a3, conj_if(ta[(3 * u) & 4095], sign));
        }
        const C2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
        C2 d = csub(a1, a3);
        // times -i (forward) or +i (inverse)
        const C2 b3 = sign < 0 ? CT<C2>::make(d.y, -d.x) : CT<C2>::make(-d.y, d.x);
        y[r][0] = cadd(b0, b2);
        y[r][1] = cadd(b1, b3);
        y[r][2] = csub(b0, b2);
        y[r][3] = csub(b1, b3);
        dst[r] = c * sc + ((j / ns) * ns * 4 + k) * sj;
      }
    }
    __syncthreads();
    const int step = ns * sj;
#pragma unroll
    for (int r = 0; r < MAXB; ++r) {
      if (dst[r] >= 0) {
        buf[dst[r]] = y[r][0];
        buf[dst[r] + step] = y[r][1];
        buf[dst[r] + 2 * step] = y[r][2];
        buf[dst[r] + 3 * step] = y[r][3];
      }
    }
    __syncthreads();
    ns *= 4;
  }
  if (lg & 1) {
    const int h2 = L / 2;
    const int nbf = nb * h2;
    C2 y[2 * MAXB][2];
    int dst[2 * MAXB];
#pragma unroll
    for (int r = 0; r < 2 * MAXB; ++r) {
      const int b = tid + r * nth;
      dst[r] = -1;
      if (b < nbf) {
        const int c = b % nb, j = b / nb;
        const int k = j & (ns - 1);
        C2* col = buf + c * sc;
        C2 a0 = col[j * sj], a1 = col[(j + h2) * sj];
        if (ns > 1) a1 = cmul(a1, conj_if(ta[(k * 4096) / (ns * 2)], sign));
        y[r][0] = cadd(a0, a1);
        y[r][1] = csub(a0, a1);
        dst[r] = c * sc + ((j / ns) * ns * 2 + k) * sj;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2 * MAXB; ++r) {
      if (dst[r] >= 0) {
        buf[dst[r]] = y[r][0];
        buf[dst[r] + ns * sj] = y[r][1];
      }
    }
    __syncthreads();
  }
}

// Copy nrow rows of rowlen contiguous complex values (global row stride gs)
// to/from a row-major shared tile, with LPT independent 16-byte accesses per
// thread in flight (rowlen * sizeof(C2) must be a multiple of 16).
template <typename C2, int LPT>
__device__ __forceinline__ void tile_load(C2* __restrict__ buf, const C2* __restrict__ g, int64_t gs, int rowlen,
                                          int nrow) {
  const int per = rowlen * (int)sizeof(C2) / 16;       // 16-byte vectors per row
  const int total = per * nrow;
  const int nth = blockDim.x;
  for (int base = threadIdx.x; base < total; base += LPT * nth) {
    float4 v[LPT];
#pragma unroll
    for (int r = 0; r < LPT; ++r) {
      const int i = base + r * nth;
      if (i < total) {
        const int row = i / per, q = i - row * per;
        v[r] = reinterpret_cast<const float4*>(g + (int64_t)row * gs)[q];
      }
    }
#pragma unroll
    for (int r = 0; r < LPT; ++r) {
      const int i = base + r * nth;
      if (i < total) reinterpret_cast<float4*>(buf)[i] = v[r];
    }
  }
}

template <typename C2>
struct FftCfg;
template <>
struct FftCfg<double2> {
  static constexpr int kCols = 8;    // columns per pass-1 CTA (8 x 16 B = 128 B rows)
  static constexpr int kMaxB = 4;    // kCols * 1024/4 / 512
};
template <>
struct FftCfg<float2> {
  static constexpr int kCols = 16;   // 16 x 8 B = 128 B rows
  static constexpr int kMaxB = 8;
};

// ------------------------------------------------------------- pass 1
// CTA = ncol adjacent columns j1, all n2 rows: the tile is staged row-major
// (rows of ncol contiguous elements), transformed along the rows index, and
// written back in place with the inter-pass twiddle.
template <typename C2>
__global__ void __launch_bounds__(kFftThreads) k3_pass1(C2* __restrict__ z, int64_t n, int n1, int n2, int ncol,
                                                        int sign, int shift22, const C2* __restrict__ ta,
                                                        const C2* __restrict__ tb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* buf = reinterpret_cast<C2*>(smraw);
  C2* zw = z + (int64_t)blockIdx.y * n;
  const int j10 = blockIdx.x * ncol;
  tile_load<C2, 8>(buf, zw + j10, n1, ncol, n2);
  __syncthreads();
  smem_fft<C2, FftCfg<C2>::kMaxB>(buf, n2, ncol, ncol, 1, sign, ta);
  for (int idx = threadIdx.x; idx < ncol * n2; idx += blockDim.x) {
    const int c = idx % ncol, k2 = idx / ncol;
    const uint32_t m = (uint32_t)((j10 + c) * k2) << shift22;
    zw[j10 + c + (int64_t)n1 * k2] = cmul(buf[idx], twiddle22(ta, tb, m, sign));
  }
}

// --------------------------------------------------- pass 2, natural order
template <typename C2>
__global__ void __launch_bounds__(kPass2Threads, 2) k4_pass2_store(const C2* __restrict__ y, C2* __restrict__ out,
                                                              int64_t n, int n1, int n2, int sign,
                                                              const C2* __restrict__ ta) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* buf = reinterpret_cast<C2*>(smraw);
  const int k2 = blockIdx.x;
  const C2* row = y + (int64_t)blockIdx.y * n + (int64_t)n1 * k2;
  tile_load<C2, 4>(buf, row, 0, n1, 1);
  __syncthreads();
  smem_fft<C2, FftCfg<C2>::kMaxB>(buf, n1, 1, 1, 1, sign, ta);
  C2* o = out + (int64_t)blockIdx.y * n;
  for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) o[k2 + (int64_t)n2 * k1] = buf[k1];
}

// -------------------------------------------- pass 2 fused with the IP
// FP64: plain double accumulation.  FP32: TwoSum-compensated float pairs.
struct AccD {
  double dh, hh;
  __device__ void init() { dh = 0.0; hh = 0.0; }
  __device__ void add(double a, double b) { dh += a; hh += b; }
  __device__ double2 get() const { return make_double2(dh, hh); }
  __device__ void shfl_merge(int off) {
    dh += __shfl_xor_sync(0xffffffffu, dh, off);
    hh += __shfl_xor_sync(0xffffffffu, hh, off);
  }
  __device__ void merge(double2 o) { dh += o.x; hh += o.y; }
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct AccF {
  float dh, dhc, hh, hhc;   // value = x + xc
  __device__ void init() { dh = dhc = hh = hhc = 0.f; }
  __device__ void add2(float& x, float& xc, float v) {
    float s, e;
    two_sum_f(x, v, s, e);
    x = s;
    xc += e;
  }
  __device__ void add(float a, float b) { add2(dh, dhc, a); add2(hh, hhc, b); }
  __device__ double2 get() const { return make_double2((double)dh + (double)dhc, (double)hh + (double)hhc); }
  __device__ void shfl_merge(int off) {
    const float o0 = __shfl_xor_sync(0xffffffffu, dh, off), o1 = __shfl_xor_sync(0xffffffffu, dhc, off);
    const float o2 = __shfl_xor_sync(0xffffffffu, hh, off), o3 = __shfl_xor_sync(0xffffffffu, hhc, off);
    add2(dh, dhc, o0);
    dhc += o1;
    add2(hh, hhc, o2);
    hhc += o3;
  }
};

template <typename C2, typename WT, typename Acc>
__global__ void __launch_bounds__(kPass2Threads, 2) k4_pass2_ip(const C2* __restrict__ y, int64_t n, int n1, int n2,
                                                           const C2* __restrict__ ta, const WalkerC* __restrict__ wcs,
                                                           const C2* __restrict__ dtab, const C2* __restrict__ dperm,
                                                           const WT* __restrict__ wperm, double2* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* buf = reinterpret_cast<C2*>(smraw);
  __shared__ double2 afac;
  __shared__ double2 red[kPass2Threads / 32];
  using T = typename CT<C2>::T;
  const int k2 = blockIdx.x, wk = blockIdx.y;
  const C2* row = y + (int64_t)wk * n + (int64_t)n1 * k2;
  tile_load<C2, 4>(buf, row, 0, n1, 1);
  if (threadIdx.x == 0) {
    // exp(-2 pi i frac(k2 r))
    const double rh = wcs[wk].r_hi, rl = wcs[wk].r_lo;
    dd p = dd_add_d(two_prod((double)k2, rh), (double)k2 * rl);
    dd f = dd_frac(p);
    double s, c;
    sincospi(2.0 * f.hi, &s, &c);
    afac = make_double2(c, -s);
  }
  __syncthreads();
  smem_fft<C2, FftCfg<C2>::kMaxB>(buf, n1, 1, 1, 1, -1, ta);
  const C2 a = CT<C2>::make((T)afac.x, (T)afac.y);
  const C2 cn = CT<C2>::make((T)wcs[wk].cn_re, (T)wcs[wk].cn_im);
  const C2* tabw = dtab + (int64_t)wk * n1;
  const int64_t base = (int64_t)k2 * n1;
  Acc acc;
  acc.init();
  for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) {
    const C2 H = buf[k1];
    const T wv = (T)wperm[base + k1];
    const C2 D = dperm[base + k1];
    C2 f = cmul(a, tabw[k1]);
    if (2 * k1 > n1 || (2 * k1 == n1 && k2 > 0)) f = cmul(f, cn);   // signed index k - n
    const C2 Hd = cmul(H, f);
    acc.add(wv * (D.x * Hd.x + D.y * Hd.y), wv * (H.x * H.x + H.y * H.y));
  }
  // fixed-shape reduction: warp xor tree, then warp 0 over the warp sums
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc.shfl_merge(off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc.get();
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    double2 v = lane < nw ? red[lane] : make_double2(0.0, 0.0);
    AccD r{v.x, v.y};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r.shfl_merge(off);
    if (lane == 0) partial[(int64_t)wk * n2 + k2] = r.get();
  }
}

// --------------------------------------------------------------- finalize
__global__ void k5_finalize(const double2* __restrict__ partial, int n2, const WalkerC* __restrict__ wcs, int w,
                            double dh_scale, double hh_scale, double* __restrict__ lnl, double* __restrict__ dh,
                            double* __restrict__ hh, uint32_t* __restrict__ status) {
  const int wk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (wk >= w) return;
  double sd = 0.0, sh = 0.0;
  for (int i = lane; i < n2; i += 32) {
    const double2 p = partial[(int64_t)wk * n2 + i];
    sd += p.x;
    sh += p.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, off);
    sh += __shfl_xor_sync(0xffffffffu, sh, off);
  }
  if (lane == 0) {
    const WalkerC& c = wcs[wk];
    const double as = c.amp_scale;
    const double dhu = sd * dh_scale * as;
    const double hhu = sh * hh_scale * as * as;
    double l = dhu / c.d_gw - 0.5 * hhu / (c.d_gw * c.d_gw);
    if (c.status & ST_BADPARAM) l = 0.0;
    lnl[wk] = l;
    if (dh) dh[wk] = dhu;
    if (hh) hh[wk] = hhu;
    if (status) status[wk] = c.status;
  }
}

// ------------------------------------------------------------ datasets
__global__ void k_weights(const double* __restrict__ psd, int64_t n, double dt, double fmin, double fmax,
                          double* __restrict__ w) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t kk = k <= n / 2 ? k : n - k;
  const double df = 1.0 / ((double)n * dt);
  const double f = (double)kk * df;
  const bool in = kk > 0 && 2 * kk < n && f >= fmin && f <= fmax;
  w[k] = in ? 2.0 * dt * dt * df / psd[kk] : 0.0;
}

__global__ void k_permute(const double2* __restrict__ d, const double* __restrict__ w, int n1, int n2,
                          double2* __restrict__ dp, double* __restrict__ wp, float2* __restrict__ dp32,
                          float* __restrict__ wp32, double ds, double ws) {
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y;
  if (k1 >= n1) return;
  const int64_t src = k2 + (int64_t)n2 * k1, dst = (int64_t)k2 * n1 + k1;
  const double2 v = d[src];
  dp[dst] = v;
  wp[dst] = w[src];
  dp32[dst] = make_float2((float)(v.x * ds), (float)(v.y * ds));
  wp32[dst] = (float)(w[src] * ws);
}

__global__ void k_pack(const double* __restrict__ d2, int64_t n, double2* __restrict__ z) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) z[j] = make_double2(d2[j], d2[n + j]);
}

__global__ void k_inner_dd(const double2* __restrict__ d, const double* __restrict__ w, int64_t n,
                           double* __restrict__ out) {
  __shared__ double red[1024 / 32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += w[k] * (d[k].x * d[k].x + d[k].y * d[k].y);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) *out = v;
  }
}

// ------------------------------------------------------------ launchers
static size_t pass1_smem(const FftPlan& p, bool fp32, int& ncol) {
  ncol = fp32 ? FftCfg<float2>::kCols : FftCfg<double2>::kCols;
  if (ncol > p.n1) ncol = p.n1;
  return (size_t)ncol * p.n2 * (fp32 ? sizeof(float2) : sizeof(double2));
}

void launch_fft_pass1(void* z, int batch, const FftPlan& p, bool fp32, int sign, const Twiddles& t,
                      cudaStream_t s) {
  if (batch <= 0) return;
  int ncol;
  const size_t sm = pass1_smem(p, fp32, ncol);
  dim3 g(p.n1 / ncol, batch);
  const int shift = 22 - p.log2n;
  if (fp32)
    k3_pass1<float2><<<g, kFftThreads, sm, s>>>((float2*)z, p.n, p.n1, p.n2, ncol, sign, shift, t.ta32, t.tb32);
  else
    k3_pass1<double2><<<g, kFftThreads, sm, s>>>((double2*)z, p.n, p.n1, p.n2, ncol, sign, shift, t.ta64, t.tb64);
}

void launch_fft_pass2_store(const void* y, void* out, int batch, const FftPlan& p, bool fp32, int sign,
                            const Twiddles& t, cudaStream_t s) {
  if (batch <= 0) return;
  dim3 g(p.n2, batch);
  if (fp32)
    k4_pass2_store<float2><<<g, kPass2Threads, p.n1 * sizeof(float2), s>>>((const float2*)y, (float2*)out, p.n, p.n1,
                                                                          p.n2, sign, t.ta32);
  else
    k4_pass2_store<double2><<<g, kPass2Threads, p.n1 * sizeof(double2), s>>>((const double2*)y, (double2*)out, p.n,
                                                                            p.n1, p.n2, sign, t.ta64);
}

void launch_fft_pass2_ip(const void* y, int w, const FftPlan& p, bool fp32, const Twiddles& t, const WalkerC* wc,
                         const void* delay_tab, const void* data_perm, const void* wt_perm, double2* partial,
                         cudaStream_t s) {
  if (w <= 0) return;
  dim3 g(p.n2, w);
  if (fp32)
    k4_pass2_ip<float2, float, AccF><<<g, kPass2Threads, p.n1 * sizeof(float2), s>>>(
        (const float2*)y, p.n, p.n1, p.n2, t.ta32, wc, (const float2*)delay_tab, (const float2*)data_perm,
        (const float*)wt_perm, partial);
  else
    k4_pass2_ip<double2, double, AccD><<<g, kPass2Threads, p.n1 * sizeof(double2), s>>>(
        (const double2*)y, p.n, p.n1, p.n2, t.ta64, wc, (const double2*)delay_tab, (const double2*)data_perm,
        (const double*)wt_perm, partial);
}

void launch_finalize(const double2* partial, int n2, const WalkerC* wc, int w, double dh_scale, double hh_scale,
                     double* lnl, double* dh, double* hh, uint32_t* status, cudaStream_t s) {
  if (w <= 0) return;
  k5_finalize<<<(w + 7) / 8, 256, 0, s>>>(partial, n2, wc, w, dh_scale, hh_scale, lnl, dh, hh, status);
}

void launch_weights(const double* psd, int64_t n, double dt, double fmin, double fmax, double* w, cudaStream_t s) {
  k_weights<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(psd, n, dt, fmin, fmax, w);
}

void launch_dataset_permute(const double2* d_nat, const double* w_nat, const FftPlan& p, double2* d_perm,
                            double* w_perm, float2* d_perm32, float* w_perm32, double d_scale, double w_scale,
                            cudaStream_t s) {
  dim3 g((p.n1 + 255) / 256, p.n2);
  k_permute<<<g, 256, 0, s>>>(d_nat, w_nat, p.n1, p.n2, d_perm, w_perm, d_perm32, w_perm32, d_scale, w_scale);
}

void launch_pack_time_series(const double* d2, int64_t n, double2* z, cudaStream_t s) {
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d2, n, z);
}

void launch_inner_dd(const double2* d, const double* w, int64_t n, double* out, cudaStream_t s) {
  k_inner_dd<<<1, 1024, 0, s>>>(d, w, n, out);
}

// Raise the dynamic shared-memory limit of the FFT kernels (once per device).
void fft_set_smem_limits() {
  const int lim = 200 * 1024;
  cudaFuncSetAttribute(k3_pass1<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k3_pass1<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k4_pass2_store<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k4_pass2_store<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k4_pass2_ip<double2, double, AccD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k4_pass2_ip<float2, float, AccF>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

}  // namespace emri
