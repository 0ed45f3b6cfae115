// k_fft.cu -- steps S5-S7: batched FFT and the fused noise-weighted inner
// products (paper Sec. 3: the time-domain waveform is Fourier transformed and
// compared with the data through the likelihood of Eq. (8)).
//
// n = n1 * n2 (four-step): element j = j1 + n1 j2, bin k = k2 + n2 k1.
//  pass 1: for each column j1, the n2-point DFT over j2, times the twiddle
//          exp(-2 pi i j1 k2 / n), written back in place (position j1 + n1 k2);
//  pass 2: for each row k2, the n1-point DFT over j1 gives bins k2 + n2 k1.
// Both passes are shared-memory Stockham FFTs, one CTA per column group /
// row: radix-4 stages (one radix-2 stage when log2 of the length is odd) in
// FP64, radix-8 stages (then one radix-4 or radix-2) in FP32.
// The likelihood path never writes the spectrum: pass 2 multiplies each bin
// by the GW-speed delay factor and accumulates
//   sum_k w_k Re(conj(D_k) H_k e^{-2 pi i k_s r})  and  sum_k w_k |H_k|^2
// against the data and weights stored in the same (k2-major) order, and
// writes one pair of partial sums per row.  A final kernel adds a walker's
// rows in a fixed order, so results are bitwise independent of the batch.
// Twiddles come from FP64-built tables:
//   ta[i] = exp(-2 pi i i / 4096), tb[i] = exp(-2 pi i i / 2^22),
// exp(-2 pi i m / 2^22) = ta[m >> 10] * tb[m & 1023]; the FP64 butterflies
// read tc[i] = (cos, tan) of the same angles.
#include "emri_common.cuh"
#include "emri_internal.h"

namespace emri {

constexpr int kFftThreads = 512;   // pass 1 (column groups)
constexpr int kPass2Threads = 256; // pass 2 (rows)

FftPlan make_fft_plan(int64_t n, int n2) {
  FftPlan p;
  p.n = n;
  int m = 0;
  while ((int64_t(1) << m) < n) ++m;
  p.log2n = m;
  int m2 = m / 2 < 10 ? m / 2 : 10;
  if (n2 > 0) {
    int q = 0;
    while ((1 << q) < n2) ++q;
    m2 = q;
  }
  p.n2 = 1 << m2;
  p.n1 = (int)(n >> m2);
  return p;
}

// ------------------------------------------------------------ twiddles
// tc64[i] = (cos, tan) of -2 pi i / 4096 for the FMA-folded FP64 butterflies;
// where the cosine is zero (a quarter turn) it is replaced by 2^-60 and the
// tangent by sin * 2^60, so c * t = sin exactly and the stray c * Re part is
// below 1e-18 relative.
// tt32[M/2 + k] = exp(-2 pi i k / M) for M = 2, 4, ..., 4096 and k < M/2: the
// twiddles of one FFT stage of size M in consecutive entries (the same values
// as ta32[k 4096 / M]), so the threads of a stage read them coalesced.
__global__ void k_twiddle_init(double2* ta64, double2* tb64, float2* ta32, float2* tb32, double2* tc64,
                               float2* tt32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 4096) {
    double s, c;
    sincospi(-2.0 * (double)i / 4096.0, &s, &c);
    ta64[i] = make_double2(c, s);
    ta32[i] = make_float2((float)c, (float)s);
    const double cf = fabs(c) < 0x1p-60 ? 0x1p-60 : c;
    tc64[i] = make_double2(cf, s / cf);
    if (i == 0) {
      tt32[0] = make_float2(1.f, 0.f);
    } else {
      const int half = 1 << (31 - __clz(i));   // M / 2
      double ts, tc;
      sincospi(-2.0 * (double)(i - half) / (double)(2 * half), &ts, &tc);
      tt32[i] = make_float2((float)tc, (float)ts);
    }
  }
  if (i < 1024) {
    double s, c;
    sincospi(-2.0 * (double)i / 4194304.0, &s, &c);
    tb64[i] = make_double2(c, s);
    tb32[i] = make_float2((float)c, (float)s);
  }
}

void launch_twiddle_init(Twiddles t, cudaStream_t s) {
  k_twiddle_init<<<16, 256, 0, s>>>(t.ta64, t.tb64, t.ta32, t.tb32, t.tc64, t.tt32);
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
// FP32: one paired (f32x2) instruction each (a - b as fma(b, -1, a), rounded
// once).  Unlike scalar additions they are not contracted with a preceding
// product into one FMA, so the FP32 tile transforms round differently in the
// last bit than with scalar forms; FP32 pass 1 takes 7.81 instead of 8.19 ms
// per 1024-walker 2^21 step with them.
template <>
__device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
template <>
__device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
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

// x with its sign flipped when sign > 0 (the inverse transform's conjugate
// twiddles), by an integer XOR on the high word: no FP64 instruction
__device__ __forceinline__ double flip_sign(double x, int sign) {
  return __longlong_as_double(__double_as_longlong(x) ^ (sign > 0 ? (long long)0x8000000000000000ULL : 0LL));
}

// ------------------------------------------------- shared-memory Stockham
// NB transforms of length L = 2^LG (compile-time), element i of transform c at
// buf[i*NB + c] (row-major tile; NB = 1 for a single contiguous transform).
// Butterfly b works on transform b % NB, element b / NB, so consecutive
// threads touch consecutive addresses.  Each thread stages its outputs in
// registers so a stage reads everything before anything is overwritten.
// FP64 only (C2 = double2); tf[i] = (cos, tan) of -2 pi i / 4096.
template <typename C2, int LG, int NB, int NTH>
__device__ __forceinline__ void smem_fft(C2* buf, int sign, const C2* __restrict__ tf) {
  static_assert(sizeof(C2) == 16, "FP64 transform");
  constexpr int L = 1 << LG;
  constexpr int NR4 = LG / 2;
  constexpr int NBF4 = NB * (L / 4);
  constexpr int MB4 = (NBF4 + NTH - 1) / NTH;
  const int tid = threadIdx.x;
#pragma unroll
  for (int st = 0; st < NR4; ++st) {
    const int ns = 1 << (2 * st);
    constexpr int Q4 = L / 4;
    C2 y[MB4][4];
    int dst[MB4];
#pragma unroll
    for (int r = 0; r < MB4; ++r) {
      const int b = tid + r * NTH;
      dst[r] = -1;
      if (NBF4 % NTH == 0 || b < NBF4) {
        const int c = b % NB, j = b / NB;
        const int k = j & (ns - 1);
        C2* col = buf + c;
        C2 a0 = col[j * NB], a1 = col[(j + Q4) * NB], a2 = col[(j + 2 * Q4) * NB], a3 = col[(j + 3 * Q4) * NB];
        if (st > 0) {
          // FMA-folded butterfly (after Goedecker): with w = c (1 + i t),
          // w1 = W^u, w2 = W^2u, w3 = w1 w2,
          //   y0, y2 = (a0 + w2 a2) +- w1 (a1 + w2 a3)
          //   y1, y3 = (a0 - w2 a2) -+ i w1 (a1 - w2 a3)   (forward)
          // in 24 FMAs instead of three products and eight sums (28)
          const int u = (k * 4096) >> (2 * st + 2);
          const double2 w1 = tf[u], w2 = tf[2 * u];
          const double t1 = flip_sign(w1.y, sign), t2 = flip_sign(w2.y, sign), c1 = w1.x, c2 = w2.x;
          const double2 v2 = make_double2(fma(-t2, a2.y, a2.x), fma(t2, a2.x, a2.y));
          const double2 v3 = make_double2(fma(-t2, a3.y, a3.x), fma(t2, a3.x, a3.y));
          const double2 pp = make_double2(fma(c2, v2.x, a0.x), fma(c2, v2.y, a0.y));
          const double2 pm = make_double2(fma(-c2, v2.x, a0.x), fma(-c2, v2.y, a0.y));
          const double2 qp = make_double2(fma(c2, v3.x, a1.x), fma(c2, v3.y, a1.y));
          const double2 qm = make_double2(fma(-c2, v3.x, a1.x), fma(-c2, v3.y, a1.y));
          const double2 e = make_double2(fma(-t1, qp.y, qp.x), fma(t1, qp.x, qp.y));
          const double2 f = make_double2(fma(-t1, qm.y, qm.x), fma(t1, qm.x, qm.y));
          const double c1s = flip_sign(c1, sign);
          y[r][0] = make_double2(fma(c1, e.x, pp.x), fma(c1, e.y, pp.y));
          y[r][2] = make_double2(fma(-c1, e.x, pp.x), fma(-c1, e.y, pp.y));
          y[r][1] = make_double2(fma(c1s, f.y, pm.x), fma(-c1s, f.x, pm.y));
          y[r][3] = make_double2(fma(-c1s, f.y, pm.x), fma(c1s, f.x, pm.y));
        } else {
          const C2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
          const C2 d = csub(a1, a3);
          const C2 b3 = sign < 0 ? CT<C2>::make(d.y, -d.x) : CT<C2>::make(-d.y, d.x);   // -i d or +i d
          y[r][0] = cadd(b0, b2);
          y[r][1] = cadd(b1, b3);
          y[r][2] = csub(b0, b2);
          y[r][3] = csub(b1, b3);
        }
        dst[r] = c + (((j >> (2 * st)) << (2 * st + 2)) + k) * NB;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MB4; ++r) {
      if (dst[r] >= 0) {
        buf[dst[r]] = y[r][0];
        buf[dst[r] + ns * NB] = y[r][1];
        buf[dst[r] + 2 * ns * NB] = y[r][2];
        buf[dst[r] + 3 * ns * NB] = y[r][3];
      }
    }
    __syncthreads();
  }
  if (LG & 1) {
    constexpr int H2 = L / 2;
    constexpr int NBF2 = NB * H2;
    constexpr int MB2 = (NBF2 + NTH - 1) / NTH;
    constexpr int NS = 1 << (2 * NR4);
    C2 y[MB2][2];
    int dst[MB2];
#pragma unroll
    for (int r = 0; r < MB2; ++r) {
      const int b = tid + r * NTH;
      dst[r] = -1;
      if (NBF2 % NTH == 0 || b < NBF2) {
        const int c = b % NB, j = b / NB;
        const int k = j & (NS - 1);
        C2* col = buf + c;
        const C2 a0 = col[j * NB], a1 = col[(j + H2) * NB];
        // a0 +- w a1 with w = c (1 + i t): 6 FMAs
        const double2 w = tf[(k * 4096) / (NS * 2)];
        const double t = flip_sign(w.y, sign);
        const double2 v = make_double2(fma(-t, a1.y, a1.x), fma(t, a1.x, a1.y));
        y[r][0] = make_double2(fma(w.x, v.x, a0.x), fma(w.x, v.y, a0.y));
        y[r][1] = make_double2(fma(-w.x, v.x, a0.x), fma(-w.x, v.y, a0.y));
        dst[r] = c + (((j / NS) * NS * 2) + k) * NB;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MB2; ++r) {
      if (dst[r] >= 0) {
        buf[dst[r]] = y[r][0];
        buf[dst[r] + NS * NB] = y[r][1];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------ radix-8 Stockham (FP32 path)
// The same Stockham layout as smem_fft, with radix-8 stages (then one radix-4
// or radix-2 stage for the remaining bits): a 2048-point transform takes four
// shared-memory round trips instead of six.  Used for float2 only: in FP64
// the radix-8 butterfly costs slightly more FP64 operations per point than
// radix 4, and the FP64 passes are bound by the FP64 pipe.
template <typename C2>
__device__ __forceinline__ C2 mul_i(C2 d, int sign) {   // -i d (sign < 0) or +i d
  return sign < 0 ? CT<C2>::make(d.y, -d.x) : CT<C2>::make(-d.y, d.x);
}

template <typename C2>
__device__ __forceinline__ void dft4_inplace(C2& a0, C2& a1, C2& a2, C2& a3, int sign) {
  const C2 s0 = cadd(a0, a2), s1 = csub(a0, a2), s2 = cadd(a1, a3), s3 = mul_i(csub(a1, a3), sign);
  a0 = cadd(s0, s2);
  a2 = csub(s0, s2);
  a1 = cadd(s1, s3);
  a3 = csub(s1, s3);
}

// X_q = sum_r a_r w^(q r), w = exp(sign 2 pi i / R), R = 2, 4, 8; in place
template <typename C2, int R>
__device__ __forceinline__ void dft_r(C2* a, int sign) {
  using T = typename CT<C2>::T;
  if constexpr (R == 2) {
    const C2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if constexpr (R == 4) {
    dft4_inplace(a[0], a[1], a[2], a[3], sign);
  } else if constexpr (R == 16) {
    // even and odd halves (8-point transforms), then the W16^q combination
    C2 e[8], o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      e[q] = a[2 * q];
      o[q] = a[2 * q + 1];
    }
    dft_r<C2, 8>(e, sign);
    dft_r<C2, 8>(o, sign);
    // W16^q = (cos(pi q/8), -+sin(pi q/8)); q = 4 is -+i
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), h = T(0.70710678118654752440);
    const T cq[8] = {T(1), c1, h, s1, T(0), -s1, -h, -c1};
    const T sq[8] = {T(0), s1, h, c1, T(1), c1, h, s1};
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      if (q == 4) o[q] = mul_i(o[q], sign);
      else o[q] = cmul(o[q], CT<C2>::make(cq[q], sign < 0 ? -sq[q] : sq[q]));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      a[q] = cadd(e[q], o[q]);
      a[q + 8] = csub(e[q], o[q]);
    }
  } else {
    // even and odd halves, then the W8^q combination
    C2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4_inplace(e0, e1, e2, e3, sign);
    dft4_inplace(o0, o1, o2, o3, sign);
    const T h = T(0.70710678118654752440);
    // W8 = h (1 - i) for sign < 0, h (1 + i) for sign > 0
    o1 = sign < 0 ? CT<C2>::make(h * (o1.x + o1.y), h * (o1.y - o1.x))
                  : CT<C2>::make(h * (o1.x - o1.y), h * (o1.x + o1.y));
    o2 = mul_i(o2, sign);
    o3 = sign < 0 ? CT<C2>::make(h * (o3.y - o3.x), -h * (o3.x + o3.y))
                  : CT<C2>::make(-h * (o3.x + o3.y), h * (o3.x - o3.y));
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
  }
}

// One radix-R stage on NB interleaved transforms of length L, sub-transform
// length NS so far.  Twiddles W_{R NS}^{k r}: W^k from the table ta (4096
// points per cycle), its powers by complex products (at most three deep).
// One table load per butterfly instead of R-1: the scattered table loads
// (up to 32 L1 wavefronts each) were the stage's bottleneck; the products
// raise the FP32 transform's rms error from 1.3e-7 to 2.0e-7 relative
// (2048 points), well below the FP32 waveform's own error.
template <typename C2, int R, int NB, int NTH, int L, int NS>
__device__ __forceinline__ void stage_r(C2* buf, int sign, const C2* __restrict__ ta) {
  constexpr int Q = L / R;
  constexpr int NBF = NB * Q;
  constexpr int MB = (NBF + NTH - 1) / NTH;
  constexpr int STEP = 4096 / (R * NS);
  const int tid = threadIdx.x;
  C2 y[MB][R];
  int dst[MB];
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = tid + m * NTH;
    dst[m] = -1;
    if (NBF % NTH == 0 || b < NBF) {
      const int c = b % NB, j = b / NB;
      const int k = j & (NS - 1);
#pragma unroll
      for (int q = 0; q < R; ++q) y[m][q] = buf[(j + q * Q) * NB + c];
      if (NS > 1) {
        C2 w[R];
        w[1] = conj_if(ta[k * STEP], sign);
        if constexpr (R >= 4) {
          w[2] = cmul(w[1], w[1]);
          w[3] = cmul(w[2], w[1]);
        }
        if constexpr (R >= 8) {
          w[4] = cmul(w[2], w[2]);
          w[5] = cmul(w[4], w[1]);
          w[6] = cmul(w[4], w[2]);
          w[7] = cmul(w[4], w[3]);
        }
        if constexpr (R == 16) {
          w[8] = cmul(w[4], w[4]);
#pragma unroll
          for (int q = 9; q < 16; ++q) w[q] = cmul(w[8], w[q - 8]);
        }
#pragma unroll
        for (int q = 1; q < R; ++q) y[m][q] = cmul(y[m][q], w[q]);
      }
      dft_r<C2, R>(y[m], sign);
      dst[m] = c + (((j / NS) * NS * R) + k) * NB;
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < MB; ++m)
    if (dst[m] >= 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) buf[dst[m] + q * NS * NB] = y[m][q];
    }
  __syncthreads();
}

// Radix-8 stages, then radix 4 (LG = 3k + 2) or, for LG = 3k + 1, one
// radix-16 stage in place of the last radix-8 and a radix-2 stage (one
// shared-memory round trip fewer; 2^4 alone keeps radix 8 + 2).
template <typename C2, int LG, int NB, int NTH, int ST>
__device__ __forceinline__ void r8_stages(C2* buf, int sign, const C2* __restrict__ ta) {
  constexpr int L = 1 << LG;
  constexpr bool R16 = LG % 3 == 1 && LG >= 7;
  constexpr int N8 = R16 ? LG / 3 - 1 : LG / 3;
  if constexpr (ST < N8) {
    stage_r<C2, 8, NB, NTH, L, (1 << (3 * ST))>(buf, sign, ta);
    r8_stages<C2, LG, NB, NTH, ST + 1>(buf, sign, ta);
  } else {
    constexpr int NS = 1 << (3 * N8);
    if constexpr (LG % 3 == 2) stage_r<C2, 4, NB, NTH, L, NS>(buf, sign, ta);
    if constexpr (R16) stage_r<C2, 16, NB, NTH, L, NS>(buf, sign, ta);
    if constexpr (LG % 3 == 1 && !R16) stage_r<C2, 2, NB, NTH, L, NS>(buf, sign, ta);
  }
}

// The transform of a shared tile: radix-8 stages in FP32 (tf = (cos, sin)
// table), FMA-folded radix-4 in FP64 (tf = (cos, tan) table).
template <typename C2, int LG, int NB, int NTH>
__device__ __forceinline__ void tile_fft(C2* buf, int sign, const C2* __restrict__ tf) {
  if constexpr (sizeof(C2) == 8)
    r8_stages<C2, LG, NB, NTH, 0>(buf, sign, tf);
  else
    smem_fft<C2, LG, NB, NTH>(buf, sign, tf);
}

template <typename C2>
__device__ __forceinline__ C2 cn_factor(const WalkerC& c);
template <>
__device__ __forceinline__ double2 cn_factor<double2>(const WalkerC& c) { return make_double2(c.cn_re, c.cn_im); }
template <>
__device__ __forceinline__ float2 cn_factor<float2>(const WalkerC& c) { return make_float2(c.cnf[0], c.cnf[1]); }

// 16-byte asynchronous global -> shared copies (cp.async, L2 only) and their
// group fences: the copies of a row are issued before the FFT and waited for
// after it, so their latency overlaps the butterflies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// bytes (a multiple of 16, both addresses 16-byte aligned) by all threads
__device__ __forceinline__ void row_async(void* smem, const void* gmem, int bytes) {
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x)
    cp_async16((char*)smem + 16 * i, (const char*)gmem + 16 * (size_t)i);
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
  static constexpr int kCols = 8;    // 8 x 8 B = 64 B rows; 64 KB tiles, two CTAs per SM
  static constexpr int kMaxB = 4;
};

// ------------------------------- FP32 pass 2 fused with the IP, in registers
// Row FFT of N1 = 2^LG points (LG 8..12) by T = N1/8 threads with eight
// points each in registers: radix-8 Stockham stages, then one radix-4 or
// radix-2 stage for the remaining bits.  At the start of every stage thread
// t holds the points t + q T (q < 8) of the stage's input; the first stage
// loads them from the row in global memory, later ones from a shared buffer
// the previous stage wrote (element i at i + i/16, which keeps the stride-8
// writes of the first stage free of bank conflicts), and the last stage
// leaves the bins k1 = t + q T in registers, where the inner products take
// them (a thread's bins in FP32, the row's threads in TwoSum-compensated
// FP32 pairs).  Complex additions run as paired FP32 instructions (f32x2).  The
// stage twiddles W_M^k (M = R NS) come from the stage table tt, W^2..W^7 by
// complex products.
namespace r8 {

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// plain componentwise complex add / subtract as paired FP32 instructions
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// complex a b in scalar FMAs (a paired form would need swizzled operand pairs)
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// X_q = sum_r a_r exp(-2 pi i q r / 4), in place; the -i rotation in scalar adds
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s0 = add(a0, a2), s1 = sub(a0, a2), s2 = add(a1, a3), d = sub(a1, a3);
  a0 = add(s0, s2);
  a2 = sub(s0, s2);
  a1 = make_float2(s1.x + d.y, s1.y - d.x);   // s1 - i d
  a3 = make_float2(s1.x - d.y, s1.y + d.x);   // s1 + i d
}

// X_q = sum_r a_r exp(-2 pi i q r / 8), in place (natural order): split in
// halves b_r = a_r + a_{r+4} (even outputs) and c_r = (a_r - a_{r+4}) W8^r
// (odd outputs), then two 4-point DFTs; c_2 = -i d_2 enters the second one
// in scalar adds.
__device__ __forceinline__ void dft8(float2 (&a)[8]) {
  constexpr float h = 0.70710678118654752440f;
  float2 b0 = add(a[0], a[4]), b1 = add(a[1], a[5]), b2 = add(a[2], a[6]), b3 = add(a[3], a[7]);
  const float2 d0 = sub(a[0], a[4]), d1 = sub(a[1], a[5]), d2 = sub(a[2], a[6]), d3 = sub(a[3], a[7]);
  // W8 d1 = h (d1.x + d1.y, d1.y - d1.x); W8^3 d3 = h (d3.y - d3.x, -(d3.x + d3.y))
  const float2 c1 = __fmul2_rn(make_float2(h, h), make_float2(d1.x + d1.y, d1.y - d1.x));
  const float2 c3 = __fmul2_rn(make_float2(h, h), make_float2(d3.y - d3.x, -(d3.x + d3.y)));
  dft4(b0, b1, b2, b3);
  // 4-point DFT of (d0, c1, -i d2, c3)
  const float2 s0 = make_float2(d0.x + d2.y, d0.y - d2.x);   // d0 + (-i d2)
  const float2 s1 = make_float2(d0.x - d2.y, d0.y + d2.x);   // d0 - (-i d2)
  const float2 s2 = add(c1, c3), dd = sub(c1, c3);
  a[0] = b0; a[2] = b1; a[4] = b2; a[6] = b3;
  a[1] = add(s0, s2);
  a[5] = sub(s0, s2);
  a[3] = make_float2(s1.x + dd.y, s1.y - dd.x);
  a[7] = make_float2(s1.x - dd.y, s1.y + dd.x);
}

// multiply a[q] by w^q, q = 1..7 (w^2..w^7 by products)
__device__ __forceinline__ void twiddle8(float2 (&a)[8], float2 w1) {
  const float2 w2 = mul(w1, w1), w3 = mul(w2, w1), w4 = mul(w2, w2);
  const float2 w5 = mul(w4, w1), w6 = mul(w4, w2), w7 = mul(w4, w3);
  a[1] = mul(a[1], w1); a[2] = mul(a[2], w2); a[3] = mul(a[3], w3); a[4] = mul(a[4], w4);
  a[5] = mul(a[5], w5); a[6] = mul(a[6], w6); a[7] = mul(a[7], w7);
}

// Radix-8 stage S (sub-transform length NS = 8^S) of an N-point transform
// whose element i sits at xb[pad16(i)]; t is the thread's index.  The
// padded positions of a thread's writes d0 + q NS and reads t + q T are
// pad16(base) plus the compile-time offsets q NS + (q NS >> 4) and
// q (T + T/16): the low four bits of base and of q NS never carry into
// bit 4 (d0 mod 16 + q NS mod 16 < 16 for NS = 1, 8 and every larger NS).
template <int LG, int S>
__device__ __forceinline__ void stage8(float2 (&v)[8], float2* xb, const float2* __restrict__ tt, int t) {
  constexpr int N = 1 << LG, T = N / 8, NS = 1 << (3 * S);
  static_assert(T % 16 == 0, "eight points per thread and at least 16 threads per transform");
  const int k = t & (NS - 1);
  if constexpr (NS > 1) twiddle8(v, tt[4 * NS + k]);   // W_{8 NS}^k
  dft8(v);
  if constexpr (8 * NS < N) {
    float2* wp = xb + pad16((t / NS) * NS * 8 + k);
#pragma unroll
    for (int q = 0; q < 8; ++q) wp[q * NS + ((q * NS) >> 4)] = v[q];
    __syncthreads();
    const float2* rp = xb + pad16(t);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = rp[q * (T + T / 16)];
    __syncthreads();   // every read done before the next stage writes
  }
}

template <int LG, int S>
__device__ __forceinline__ void stages8(float2 (&v)[8], float2* xb, const float2* __restrict__ tt, int t) {
  if constexpr (S < LG / 3) {
    stage8<LG, S>(v, xb, tt, t);
    stages8<LG, S + 1>(v, xb, tt, t);
  }
}

// The last stage for LG % 3 != 0: radix 4 (two butterflies per thread) or
// radix 2 (four).  Slot q of v holds bin t + q T afterwards.
template <int LG>
__device__ __forceinline__ void last_stage(float2 (&v)[8], const float2* __restrict__ tt, int t) {
  constexpr int N1 = 1 << LG, T = N1 / 8;
  if constexpr (LG % 3 == 2) {        // NS = N1/4: butterflies t and t + T over v[0,2,4,6] and v[1,3,5,7]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2 w1 = tt[N1 / 2 + t + h * T];   // W_{N1}^k, k = t + h T
      const float2 w2 = mul(w1, w1), w3 = mul(w2, w1);
      float2 a0 = v[h], a1 = mul(v[h + 2], w1), a2 = mul(v[h + 4], w2), a3 = mul(v[h + 6], w3);
      dft4(a0, a1, a2, a3);
      v[h] = a0; v[h + 2] = a1; v[h + 4] = a2; v[h + 6] = a3;
    }
  } else if constexpr (LG % 3 == 1) { // NS = N1/2: butterflies t + i T over v[i], v[i + 4]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 b = mul(v[i + 4], tt[N1 / 2 + t + i * T]);
      const float2 a = v[i];
      v[i] = add(a, b);
      v[i + 4] = sub(a, b);
    }
  }
}

}  // namespace r8

// ------------------------------------------------------------- pass 1
// CTA = NB adjacent columns j1, all n2 = 2^LG rows: the tile is staged
// row-major (rows of NB contiguous elements), transformed along the rows
// index, and written back in place with the inter-pass twiddle.
template <typename C2, int LG, int NB>
__global__ void __launch_bounds__(kFftThreads, sizeof(C2) == 8 ? 2 : 1) k3_pass1(C2* __restrict__ z, int64_t n, int n1, int sign, int shift22,
                                                        const C2* __restrict__ ta, const C2* __restrict__ tb,
                                                        const C2* __restrict__ tf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* buf = reinterpret_cast<C2*>(smraw);
  constexpr int N2 = 1 << LG;
  C2* zw = z + (int64_t)blockIdx.y * n;
  const int j10 = blockIdx.x * NB;
  if constexpr (sizeof(C2) == 8) {
    // the tile's rows (NB * 8 bytes each) by cp.async: all of it in flight,
    // no registers held (with two CTAs per SM this took pass 1 from 9.65 to
    // 8.62 ms per 1024-walker 2^21 step against register-staged loads)
    constexpr int VR = NB * 8 / 16, V = VR * N2;   // 16-byte copies per row, per tile
#pragma unroll
    for (int i0 = 0; i0 < V; i0 += kFftThreads) {
      const int i = i0 + (int)threadIdx.x;
      if (V % kFftThreads == 0 || i < V) {         // small tiles: fewer copies than threads
        const int row = i / VR, q = i - row * VR;
        cp_async16(buf + row * NB + 2 * q, zw + j10 + (int64_t)row * n1 + 2 * q);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
  } else {
    tile_load<C2, 8>(buf, zw + j10, n1, NB, N2);
  }
  __syncthreads();
  tile_fft<C2, LG, NB, kFftThreads>(buf, sign, tf);
  // write-back with the inter-pass twiddle W_n^{j1 k2}: a thread keeps its
  // column (kFftThreads is a multiple of NB) and steps k2 by kFftThreads/NB,
  // so the twiddle advances by a fixed factor; it is re-read from the table
  // every 4th element (error at most a few ulp, loads 0.6 per element)
  static_assert(kFftThreads % NB == 0, "threads per column");
  const int c = threadIdx.x % NB;
  const C2 wstep = twiddle22(ta, tb, (uint32_t)((j10 + c) * (kFftThreads / NB)) << shift22, sign);
  C2 w = CT<C2>::make(1, 0);
  int i = 0;
  for (int idx = threadIdx.x; idx < NB * N2; idx += kFftThreads, ++i) {
    const int k2 = idx / NB;
    w = (i & 3) == 0 ? twiddle22(ta, tb, (uint32_t)((j10 + c) * k2) << shift22, sign) : cmul(w, wstep);
    zw[j10 + c + (int64_t)n1 * k2] = cmul(buf[idx], w);
  }
}

// --------------------------------------------------- pass 2, natural order
template <typename C2, int LG>
__global__ void __launch_bounds__(kPass2Threads, 2) k4_pass2_store(const C2* __restrict__ y, C2* __restrict__ out,
                                                                   int64_t n, int n2, int sign,
                                                                   const C2* __restrict__ tf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* buf = reinterpret_cast<C2*>(smraw);
  constexpr int N1 = 1 << LG;
  const int k2 = blockIdx.x;
  const C2* row = y + (int64_t)blockIdx.y * n + (int64_t)N1 * k2;
  tile_load<C2, 4>(buf, row, 0, N1, 1);
  __syncthreads();
  tile_fft<C2, LG, 1, kPass2Threads>(buf, sign, tf);
  C2* o = out + (int64_t)blockIdx.y * n;
  for (int k1 = threadIdx.x; k1 < N1; k1 += kPass2Threads) o[k2 + (int64_t)n2 * k1] = buf[k1];
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

// 128-bit fixed-point fractions (mod 1) for the frequency-dependent phase:
// value = (hi 2^64 + lo) / 2^128; products with a small integer and sums wrap
// mod 2^128, which is exactly the reduction mod 1 cycle.
struct U128 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ U128 mul128_small(U128 a, unsigned long long k) {
  U128 r;
  r.lo = a.lo * k;
  r.hi = a.hi * k + __umul64hi(a.lo, k);
  return r;
}
__device__ __forceinline__ U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 neg128(U128 a) {
  U128 r;
  r.lo = ~a.lo + 1ull;
  r.hi = ~a.hi + (r.lo == 0ull ? 1ull : 0ull);
  return r;
}

// exp(-2 pi i phi) of a phase fraction given by the top 64 bits (signed,
// [-1/2, 1/2) cycle)
__device__ __forceinline__ void phase_factor(long long top, double& c, double& s) {
  const double ph = (double)top * 5.421010862427522e-20;   // 2^-64
  double sn, cs;
  sincospi(2.0 * ph, &sn, &cs);
  c = cs;
  s = -sn;
}
__device__ __forceinline__ void phase_factor(long long top, float& c, float& s) {
  const float ph = (float)(int)(top >> 32) * 2.3283064365386963e-10f;   // 2^-32
  float sn, cs;
  __sincosf(6.283185307179586f * ph, &sn, &cs);
  c = cs;
  s = -sn;
}
__device__ __forceinline__ double fd_exp(double x) { return exp(x); }
__device__ __forceinline__ float fd_exp(float x) { return __expf(x); }

// Frequency-dependent factor of bin |k_s| = a: amplitude A (returned) and
// the phase factor (c, s) = exp(-2 pi i sgn(k_s) sum beta_m a^(m+1)).
template <typename T>
__device__ __forceinline__ T fd_factor(const FdW& f, unsigned long long a, bool neg, T& c, T& s) {
  T A = T(1);
  if (f.qm > 0) {
    const T x = (T)a * (T)f.xs;
    T am = (T)f.a[f.qm - 1];
    for (int m = f.qm - 2; m >= 0; --m) am = am * x + (T)f.a[m];
    A = fd_exp((T)f.nlz_half * am * x);
  }
  if (f.qt > 0) {
    U128 acc{f.bhi[f.qt - 1], f.blo[f.qt - 1]};
    for (int m = f.qt - 2; m >= 0; --m) acc = add128(mul128_small(acc, a), U128{f.bhi[m], f.blo[m]});
    acc = mul128_small(mul128_small(acc, a), a);
    if (neg) acc = neg128(acc);
    phase_factor((long long)acc.hi, c, s);
  } else {
    c = T(1);
    s = T(0);
  }
  return A;
}

// Shared memory of one pass-2 row: the row itself, then (when they fit in
// 160 KB together) the row's data, delay factors and weights, prefetched.
template <typename C2, typename WT, int LG>
struct P2Smem {
  static constexpr int N1 = 1 << LG;
  static constexpr bool kPrefetch = (size_t)N1 * (3 * sizeof(C2) + sizeof(WT)) <= 160 * 1024;
  static constexpr size_t bytes() {
    return kPrefetch ? (size_t)N1 * (3 * sizeof(C2) + sizeof(WT)) : (size_t)N1 * sizeof(C2);
  }
};

template <typename C2, typename WT, typename Acc, int LG, bool FD>
__global__ void __launch_bounds__(kPass2Threads, sizeof(C2) == 8 ? 4 : 2)
    k4_pass2_ip(const C2* __restrict__ y, int64_t n, int n2, const C2* __restrict__ tf,
                const WalkerC* __restrict__ wcs, const C2* __restrict__ dtab, const C2* __restrict__ rtab,
                const C2* __restrict__ dperm, const WT* __restrict__ wperm, double2* __restrict__ partial,
                const FdW* __restrict__ fdw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using SM = P2Smem<C2, WT, LG>;
  C2* buf = reinterpret_cast<C2*>(smraw);
  C2* ds = buf + SM::N1;
  C2* ts = ds + SM::N1;
  WT* ws = reinterpret_cast<WT*>(ts + SM::N1);
  __shared__ Acc red[kPass2Threads / 32];
  using T = typename CT<C2>::T;
  constexpr int N1 = 1 << LG;
  const int k2 = blockIdx.x, wk = blockIdx.y;
  const C2* row = y + (int64_t)wk * n + (int64_t)N1 * k2;
  const int64_t base = (int64_t)k2 * N1;
  const C2* tabw = dtab + (int64_t)wk * N1;
  row_async(buf, row, N1 * (int)sizeof(C2));
  cp_async_commit();
  if (SM::kPrefetch) {
    row_async(ds, dperm + base, N1 * (int)sizeof(C2));
    row_async(ts, tabw, N1 * (int)sizeof(C2));
    row_async(ws, wperm + base, N1 * (int)sizeof(WT));
  }
  cp_async_commit();
  const C2 a = rtab[(int64_t)wk * n2 + k2];                 // exp(-2 pi i frac(k2 r))
  const C2 cnv = cn_factor<C2>(wcs[wk]);
  cp_async_wait<1>();
  __syncthreads();
  tile_fft<C2, LG, 1, kPass2Threads>(buf, -1, tf);
  cp_async_wait<0>();
  __syncthreads();
  // a thread's own bins (N1/256 of them) in plain arithmetic; the
  // compensated accumulator then merges the threads in a fixed order.
  // The bin's delay factor is a * ts[k1] (times cn for negative
  // frequencies; the table carries it for k1 > N1/2), and the row factor a
  // is common to the row: <d|h> collects Z = sum g ts H and takes Re(a Z).
  T zr = T(0), zi = T(0), shh = T(0);
  FdW fd;
  if (FD) fd = fdw[wk];
  for (int k1 = threadIdx.x; k1 < N1; k1 += kPass2Threads) {
    const C2 H = buf[k1];
    const T wv = SM::kPrefetch ? (T)ws[k1] : (T)wperm[base + k1];
    const C2 G = SM::kPrefetch ? ds[k1] : dperm[base + k1];
    C2 P = cmul(H, SM::kPrefetch ? ts[k1] : tabw[k1]);
    if (2 * k1 == N1 && k2 > 0) P = cmul(P, cnv);   // the one negative bin of this column not in the table
    T A2 = T(1);
    if (FD) {
      const bool neg = 2 * k1 > N1 || (2 * k1 == N1 && k2 > 0);
      const long long kk = (long long)k2 + (long long)n2 * k1;
      const unsigned long long ak = (unsigned long long)(neg ? n - kk : kk);
      T c, sn;
      const T A = fd_factor<T>(fd, ak, neg, c, sn);
      P = cmul(P, CT<C2>::make(A * c, A * sn));
      A2 = A * A;
    }
    zr += G.x * P.x - G.y * P.y;
    zi += G.x * P.y + G.y * P.x;
    shh += wv * (H.x * H.x + H.y * H.y) * A2;
  }
  const T sdh = a.x * zr - a.y * zi;
  Acc acc;
  acc.init();
  acc.add(sdh, shh);
  // fixed-shape reduction in the accumulator's own arithmetic: warp xor tree,
  // then warp 0 over the warp partials
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc.shfl_merge(off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = kPass2Threads / 32;
    Acc r;
    if (lane < NW) r = red[lane];
    else r.init();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r.shfl_merge(off);
    if (lane == 0) partial[(int64_t)wk * n2 + k2] = r.get();
  }
}


template <int LG, bool FD>
__global__ void __launch_bounds__((1 << LG) / 8)
    k4_pass2_ip_r8(const float2* __restrict__ y, int64_t n, int n2, const float2* __restrict__ tt,
                   const WalkerC* __restrict__ wcs, const float2* __restrict__ dtab, const float2* __restrict__ rtab,
                   const float2* __restrict__ dperm, const float* __restrict__ wperm, double2* __restrict__ partial,
                   const FdW* __restrict__ fdw) {
  constexpr int N1 = 1 << LG, T = N1 / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* xb = reinterpret_cast<float2*>(smraw);   // stage exchange, padded
  __shared__ AccF red[T / 32];
  const int t = threadIdx.x;
  const int k2 = blockIdx.x, wk = blockIdx.y;
  const int64_t base = (int64_t)k2 * N1;
  // the inner product's operands, read where they are used (the row's
  // dataset entries from L2, the walker's delay factors from L1/L2): shared
  // memory holds only the exchange buffer (17 KB at 2048 points), and the
  // registers, not shared memory, bound the CTAs per SM.  Staging the three
  // rows in shared memory by cp.async (57 KB, three CTAs per SM) took
  // 8.42 ms per 1024-walker 2^21 step against 6.67 ms.
  const float2* ds = dperm + base;                  // the row's g = w conj(D)
  const float2* ts = dtab + (int64_t)wk * N1;       // the walker's delay factors
  const float* ws = wperm + base;                   // the row's weights
  const float2* row = y + (int64_t)wk * n + (int64_t)N1 * k2;
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = row[t + q * T];
  const float2 a = rtab[(int64_t)wk * n2 + k2];   // exp(-2 pi i frac(k2 r))
  const float2 cnv = make_float2(wcs[wk].cnf[0], wcs[wk].cnf[1]);
  r8::stages8<LG, 0>(v, xb, tt, t);
  r8::last_stage<LG>(v, tt, t);
  // the thread's bins k1 = t + q T in plain FP32, then the compensated tree
  float zr = 0.f, zi = 0.f, shh = 0.f;
  FdW fd;
  if (FD) fd = fdw[wk];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k1 = t + q * T;
    const float2 H = v[q];
    const float wv = ws[k1];
    const float2 G = ds[k1];
    float2 P = cmul(H, ts[k1]);
    // the one negative bin of this column not in the table: k1 = N1/2 = 4 T,
    // i.e. slot 4 of thread 0
    if (q == 4 && t == 0 && k2 > 0) P = cmul(P, cnv);
    float A2 = 1.f;
    if (FD) {
      const bool neg = q > 4 || (q == 4 && t > 0) || (q == 4 && t == 0 && k2 > 0);
      const long long kk = (long long)k2 + (long long)n2 * k1;
      const unsigned long long ak = (unsigned long long)(neg ? n - kk : kk);
      float c, sn;
      const float A = fd_factor<float>(fd, ak, neg, c, sn);
      P = cmul(P, make_float2(A * c, A * sn));
      A2 = A * A;
    }
    zr += G.x * P.x - G.y * P.y;
    zi += G.x * P.y + G.y * P.x;
    shh += wv * (H.x * H.x + H.y * H.y) * A2;
  }
  // fixed-shape reduction in TwoSum-compensated FP32 pairs: warp xor tree,
  // then warp 0 over the warp partials
  AccF acc;
  acc.init();
  acc.add(a.x * zr - a.y * zi, shh);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc.shfl_merge(off);
  const int lane = t & 31, wid = t >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = T / 32;
    AccF r;
    if (lane < NW) r = red[lane];
    else r.init();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r.shfl_merge(off);
    if (lane == 0) partial[(int64_t)wk * n2 + k2] = r.get();
  }
}

template <int LG>
constexpr size_t r8_smem() {
  return (size_t)((1 << LG) + (1 << LG) / 16) * sizeof(float2);
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

// Dataset arrays in pass-2 order (bin k2 + n2 k1 at k2 * n1 + k1): the
// weighted conjugate data g = w conj(D) (the inner product needs only this
// product) and the weights w, in FP64 and scaled FP32 (g by ds ws, w by ws).
__global__ void k_permute(const double2* __restrict__ d, const double* __restrict__ w, int n1, int n2,
                          double2* __restrict__ gp, double* __restrict__ wp, float2* __restrict__ gp32,
                          float* __restrict__ wp32, double ds, double ws) {
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y;
  if (k1 >= n1) return;
  const int64_t src = k2 + (int64_t)n2 * k1, dst = (int64_t)k2 * n1 + k1;
  const double2 v = d[src];
  const double wv = w[src];
  const double2 g = make_double2(wv * v.x, -(wv * v.y));
  gp[dst] = g;
  wp[dst] = wv;
  const double sc = ds * ws;
  gp32[dst] = make_float2((float)(g.x * sc), (float)(g.y * sc));
  wp32[dst] = (float)(wv * ws);
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
template <typename C2>
static size_t csize() { return sizeof(C2); }

template <typename C2, int NB, int LG>
static void pass1_inst(C2* z, int batch, const FftPlan& p, int sign, int shift, const C2* ta, const C2* tb,
                       const C2* tf, cudaStream_t s) {
  dim3 g(p.n1 / NB, batch);
  k3_pass1<C2, LG, NB><<<g, kFftThreads, (size_t)NB * (1 << LG) * sizeof(C2), s>>>(z, p.n, p.n1, sign, shift, ta, tb,
                                                                                    tf);
}

template <typename C2, int NB>
static void pass1_dispatch(C2* z, int batch, const FftPlan& p, int sign, const C2* ta, const C2* tb, const C2* tf,
                           cudaStream_t s) {
  const int shift = 22 - p.log2n;
  int lg = 0;
  while ((1 << lg) < p.n2) ++lg;
  switch (lg) {
    case 5: pass1_inst<C2, NB, 5>(z, batch, p, sign, shift, ta, tb, tf, s); break;
    case 6: pass1_inst<C2, NB, 6>(z, batch, p, sign, shift, ta, tb, tf, s); break;
    case 7: pass1_inst<C2, NB, 7>(z, batch, p, sign, shift, ta, tb, tf, s); break;
    case 8: pass1_inst<C2, NB, 8>(z, batch, p, sign, shift, ta, tb, tf, s); break;
    case 9: pass1_inst<C2, NB, 9>(z, batch, p, sign, shift, ta, tb, tf, s); break;
    default: pass1_inst<C2, NB, 10>(z, batch, p, sign, shift, ta, tb, tf, s); break;
  }
}

static int log2i(int v) {
  int lg = 0;
  while ((1 << lg) < v) ++lg;
  return lg;
}


void launch_fft_pass1(void* z, int batch, const FftPlan& p, bool fp32, int sign, const Twiddles& t,
                      cudaStream_t s) {
  if (batch <= 0) return;
  if (fp32)
    pass1_dispatch<float2, FftCfg<float2>::kCols>((float2*)z, batch, p, sign, t.ta32, t.tb32, t.ta32, s);
  else
    pass1_dispatch<double2, FftCfg<double2>::kCols>((double2*)z, batch, p, sign, t.ta64, t.tb64, t.tc64, s);
}

#define EMRI_LG_SWITCH(lg, CALL)  \
  switch (lg) {                   \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    case 7: CALL(7); break;       \
    case 8: CALL(8); break;       \
    case 9: CALL(9); break;       \
    case 10: CALL(10); break;     \
    case 11: CALL(11); break;     \
    default: CALL(12); break;     \
  }


void launch_fft_pass2_store(const void* y, void* out, int batch, const FftPlan& p, bool fp32, int sign,
                            const Twiddles& t, cudaStream_t s) {
  if (batch <= 0) return;
  dim3 g(p.n2, batch);
  const int lg = log2i(p.n1);
  if (fp32) {
#define CALL32(L) k4_pass2_store<float2, L><<<g, kPass2Threads, p.n1 * sizeof(float2), s>>>( \
      (const float2*)y, (float2*)out, p.n, p.n2, sign, t.ta32)
    EMRI_LG_SWITCH(lg, CALL32)
#undef CALL32
  } else {
#define CALL64(L) k4_pass2_store<double2, L><<<g, kPass2Threads, p.n1 * sizeof(double2), s>>>( \
      (const double2*)y, (double2*)out, p.n, p.n2, sign, t.tc64)
    EMRI_LG_SWITCH(lg, CALL64)
#undef CALL64
  }
}

template <bool FD>
static void pass2_ip_dispatch(const void* y, int w, const FftPlan& p, bool fp32, const Twiddles& t,
                              const WalkerC* wc, const void* delay_tab, const void* row_tab, const void* data_perm,
                              const void* wt_perm, double2* partial, const FdW* fd, cudaStream_t s) {
  dim3 g(p.n2, w);
  const int lg = log2i(p.n1);
  if (fp32 && lg >= 8) {   // rows of 256..4096 points: register-resident radix-8 kernel
#define CALLR8(L) k4_pass2_ip_r8<L, FD><<<g, (1 << L) / 8, r8_smem<L>(), s>>>(                          \
      (const float2*)y, p.n, p.n2, t.tt32, wc, (const float2*)delay_tab, (const float2*)row_tab,   \
      (const float2*)data_perm, (const float*)wt_perm, partial, fd)
    switch (lg) {
      case 8: CALLR8(8); break;
      case 9: CALLR8(9); break;
      case 10: CALLR8(10); break;
      case 11: CALLR8(11); break;
      default: CALLR8(12); break;
    }
#undef CALLR8
  } else if (fp32) {
#define CALLI32(L) k4_pass2_ip<float2, float, AccF, L, FD><<<g, kPass2Threads, P2Smem<float2, float, L>::bytes(), s>>>( \
      (const float2*)y, p.n, p.n2, t.ta32, wc, (const float2*)delay_tab, (const float2*)row_tab,                \
      (const float2*)data_perm, (const float*)wt_perm, partial, fd)
    EMRI_LG_SWITCH(lg, CALLI32)
#undef CALLI32
  } else {
#define CALLI64(L) k4_pass2_ip<double2, double, AccD, L, FD><<<g, kPass2Threads, P2Smem<double2, double, L>::bytes(), s>>>( \
      (const double2*)y, p.n, p.n2, t.tc64, wc, (const double2*)delay_tab, (const double2*)row_tab,                 \
      (const double2*)data_perm, (const double*)wt_perm, partial, fd)
    EMRI_LG_SWITCH(lg, CALLI64)
#undef CALLI64
  }
}

void launch_fft_pass2_ip(const void* y, int w, const FftPlan& p, bool fp32, const Twiddles& t, const WalkerC* wc,
                         const void* delay_tab, const void* row_tab, const void* data_perm, const void* wt_perm,
                         double2* partial, cudaStream_t s, const FdW* fd) {
  if (w <= 0) return;
  if (fd)
    pass2_ip_dispatch<true>(y, w, p, fp32, t, wc, delay_tab, row_tab, data_perm, wt_perm, partial, fd, s);
  else
    pass2_ip_dispatch<false>(y, w, p, fp32, t, wc, delay_tab, row_tab, data_perm, wt_perm, partial, nullptr, s);
}

void launch_finalize(const double2* partial, int n2, const WalkerC* wc, int w, double dh_scale, double hh_scale,
                     double* lnl, double* dh, double* hh, uint32_t* status, cudaStream_t s) {
  if (w <= 0) return;
  k5_finalize<<<(w + 7) / 8, 256, 0, s>>>(partial, n2, wc, w, dh_scale, hh_scale, lnl, dh, hh, status);
}

void launch_weights(const double* psd, int64_t n, double dt, double fmin, double fmax, double* w, cudaStream_t s) {
  k_weights<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(psd, n, dt, fmin, fmax, w);
}

void launch_dataset_permute(const double2* d_nat, const double* w_nat, const FftPlan& p, double2* g_perm,
                            double* w_perm, float2* g_perm32, float* w_perm32, double d_scale, double w_scale,
                            cudaStream_t s) {
  dim3 g((p.n1 + 255) / 256, p.n2);
  k_permute<<<g, 256, 0, s>>>(d_nat, w_nat, p.n1, p.n2, g_perm, w_perm, g_perm32, w_perm32, d_scale, w_scale);
}

void launch_pack_time_series(const double* d2, int64_t n, double2* z, cudaStream_t s) {
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d2, n, z);
}

void launch_inner_dd(const double2* d, const double* w, int64_t n, double* out, cudaStream_t s) {
  k_inner_dd<<<1, 1024, 0, s>>>(d, w, n, out);
}

// Raise the dynamic shared-memory limit of the FFT kernels (once per device).
template <typename F>
static void raise(F f) {
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void fft_set_smem_limits() {
#define P1(L) raise(k3_pass1<double2, L, FftCfg<double2>::kCols>), raise(k3_pass1<float2, L, FftCfg<float2>::kCols>)
  P1(5); P1(6); P1(7); P1(8); P1(9); P1(10);
#undef P1
#define P2(L) raise(k4_pass2_store<double2, L>), raise(k4_pass2_store<float2, L>), \
              raise(k4_pass2_ip<double2, double, AccD, L, false>), raise(k4_pass2_ip<float2, float, AccF, L, false>), \
              raise(k4_pass2_ip<double2, double, AccD, L, true>), raise(k4_pass2_ip<float2, float, AccF, L, true>)
  P2(5); P2(6); P2(7); P2(8); P2(9); P2(10); P2(11); P2(12);
#undef P2
#define P3(L) raise(k4_pass2_ip_r8<L, false>), raise(k4_pass2_ip_r8<L, true>)
  P3(8); P3(9); P3(10); P3(11); P3(12);
#undef P3
}

}  // namespace emri
