// k_wave.cu -- steps S2-S4: dense orbit, LISA response and the
// Peters-Mathews harmonic sum of Eq. (2), one CTA per 256-sample tile (FP64)
// or per 1024-sample segment (mixed).
//
// Per tile (set-up, a few threads):
//  * the cubic Hermite interpolant of every orbit quantity over each knot
//    interval the tile touches (values and rates at both knots);
//  * the Bessel amplitudes of every harmonic at the tile's start, middle and
//    end, fitted by a quadratic in time.  The amplitudes depend on time only
//    through e(t), which moves by ~1e-4 relative per tile, so the quadratic
//    is exact to ~1e-11 and the per-sample cost of a harmonic drops from a
//    Bessel evaluation to a few FMAs;
//  * the four antenna patterns in a fixed sky polarisation basis at four
//    nodes, fitted by a cubic in time (they depend on time only through the
//    LISA orbital phase, a one-year period).
// Per sample (one thread each; four per thread in the mixed kernel):
//  * phases Phi_D (Doppler folded in), 2 gamma~ and alpha from the Hermite
//    polynomials, reduced modulo one cycle, and their sin/cos;
//  * the harmonic sum written as three running sums
//      C = sum_n n pa_n cos(n Phi), S = sum_n n sqrt(1-e^2) pb_n sin(n Phi),
//      R = sum_n 2 pc_n cos(n Phi),
//    with cos(n Phi), sin(n Phi) by the Chebyshev recurrence (or complex
//    rotation), Eq. (2)'s sum of A+_n and Ax_n regrouped;
//  * the response as a contraction in the fixed basis: (C, S) rotated by
//    2 gamma~, a quadratic form in the orbital-plane projections (linear in
//    cos alpha, sin alpha), times the fitted patterns -- identical to the
//    psi / beta form of the Barack-Cutler response, without either angle;
//  * z = h_I + i h_II.
// FP64 variant: everything in double.  Mixed variant: the three phases are
// evaluated in 64-bit fixed point (linear term) plus an FP32 correction, so
// no FP64 instruction runs per sample; the rest is FP32.
#include <vector>
#include "emri_common.cuh"
#include "emri_internal.h"

namespace emri {

constexpr int kTile = 256;

// --------------------------------------------------------------- Bessel
// J_m(x) by its power series (x/2)^m / m! * sum_k a_k y^k, y = x^2/4,
// a_k = (-1)^k m! / (k! (m+k)!), evaluated by Horner's rule (one FMA per
// term) over the first K = min(ceil(12 + 1.05 x), 48) terms.  Wherever the
// series is used (orders m >= n + 1 at x = n e, n <= 32, e < 0.999) the
// omitted tail is below 1e-16 of the sum.  bc[m * kBesselTerms + k] = a_k and
// ifact[m] = 1/m! are tables (host long double, rounded once).
template <typename T>
__device__ __forceinline__ T bessel_series(int m, T x, const T* __restrict__ bc, const T* __restrict__ ifact) {
  const T half = T(0.5) * x;
  T lead = T(1);
  T p = half;
  for (int k = m; k; k >>= 1) {     // (x/2)^m by squaring
    if (k & 1) lead *= p;
    p *= p;
  }
  lead *= ifact[m];
  const T y = half * half;
  int K = (int)(T(12) + T(1.05) * x) + 1;
  if (K > kBesselTerms) K = kBesselTerms;
  const T* a = bc + m * kBesselTerms;
  T sum = a[K - 1];
#pragma unroll 4
  for (int k = K - 2; k >= 0; --k) sum = fma(sum, y, a[k]);
  return lead * sum;
}

// Amplitudes of harmonic n at eccentricity e:
//   a = n pa, b = n sqrt(1-e^2) pb, c = 2 pc  with the Peters-Mathews brackets
//   pa = J_{n-2} - 2e J_{n-1} + (2/n) J_n + 2e J_{n+1} - J_{n+2},
//   pb = J_{n-2} - 2 J_n + J_{n+2},  pc = J_n   (argument x = n e).
// J_{n+2}, J_{n+1} by series, the lower orders by the (stable) downward
// recurrence J_{m-1} = (2m/x) J_m - J_{m+1}, which also gives J_{-1} = -J_1.
template <typename T>
__device__ __forceinline__ void harmonic_amps(int n, T e, T out[3], const T* __restrict__ bc,
                                              const T* __restrict__ ifact) {
  T jm2, jm1, j0, jp1, jp2;
  if (e < T(1e-12)) {               // J_m(0) = delta_m0
    jm2 = n == 2 ? T(1) : T(0);
    jm1 = n == 1 ? T(1) : T(0);
    j0 = jp1 = jp2 = T(0);
  } else {
    const T x = T(n) * e;
    const T ix = T(1) / x;
    jp2 = bessel_series<T>(n + 2, x, bc, ifact);
    jp1 = bessel_series<T>(n + 1, x, bc, ifact);
    j0 = T(2 * (n + 1)) * ix * jp1 - jp2;
    jm1 = T(2 * n) * ix * j0 - jp1;
    jm2 = T(2 * (n - 1)) * ix * jm1 - j0;
  }
  const T pa = jm2 - T(2) * e * jm1 + (T(2) / T(n)) * j0 + T(2) * e * jp1 - jp2;
  const T pb = jm2 - T(2) * j0 + jp2;
  out[0] = T(n) * pa;
  out[1] = T(n) * sqrt(T(1) - e * e) * pb;
  out[2] = T(2) * j0;
}

// Series tables (once per context): a_k(m) = a_{k-1}(m) * (-1) / (k (m+k))
// and 1/m! in long double, rounded once to double and to float.
int upload_bessel_tables(const BesselTab& t) {
  std::vector<double> c64((size_t)kBesselOrders * kBesselTerms), f64(kBesselOrders);
  std::vector<float> c32(c64.size()), f32(kBesselOrders);
  long double fact = 1.0L;
  for (int m = 0; m < kBesselOrders; ++m) {
    if (m > 0) fact *= (long double)m;
    f64[m] = (double)(1.0L / fact);
    f32[m] = (float)(1.0L / fact);
    long double a = 1.0L;
    for (int k = 0; k < kBesselTerms; ++k) {
      if (k > 0) a = -a / ((long double)k * (long double)(m + k));
      c64[(size_t)m * kBesselTerms + k] = (double)a;
      c32[(size_t)m * kBesselTerms + k] = (float)a;
    }
  }
  bool ok = cudaMemcpy(t.c64, c64.data(), c64.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(t.c32, c32.data(), c32.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(t.f64, f64.data(), f64.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(t.f32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
  return ok ? 0 : -1;
}

// exp(2 pi i k / 512), k = 0..511, for the FP64 sin/cos of phases in
// cycles; filled from the host (long double) at context creation.
constexpr int kExpLen = 512;
__device__ double2 g_exp512[kExpLen];

int upload_exp512() {
  double2 h[kExpLen];
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < kExpLen; ++k) {
    const long double a = 2.0L * pi * (long double)k / (long double)kExpLen;
    h[k] = make_double2((double)cosl(a), (double)sinl(a));
  }
  return cudaMemcpyToSymbol(g_exp512, h, sizeof(h)) == cudaSuccess ? 0 : -1;
}

// cos(2 pi f), sin(2 pi f) for a phase f in cycles (|f| < 2^20; whole cycles
// need not be removed first): f = k/512 + d with |d| <= 1/1024,
// exp(2 pi i k/512) from the table at k mod 512 and the Taylor polynomials
// of sin to x^5 and cos to x^4 at x = 2 pi d (|x| <= 0.00614: the first
// omitted terms, x^7/7! and x^6/6!, are below 7e-20 and 8e-17).  The
// nearest integer k of 512 f comes from adding 1.5 * 2^52: the sum rounds to
// an integer, its low word is k (two's complement) and subtracting the
// constant back gives k exactly, so no separate rounding or conversion
// instruction runs; d = f - k/512 is exact.  About 13 FP64 operations.
__device__ __forceinline__ void sincos2pi_tab(double f, const double2* __restrict__ tab, double& s, double& c) {
  constexpr double kRound = 6755399441055744.0;   // 1.5 * 2^52
  const double kb = fma(f, 512.0, kRound);
  const double kd = kb - kRound;
  const int k = __double2loint(kb);
  const double d = fma(kd, -0.001953125, f);   // exact
  const double x = d * 6.283185307179586;
  const double x2 = x * x;
  const double sx = fma(x2 * x, fma(x2, 1.0 / 120.0, -1.0 / 6.0), x);
  const double cx = fma(x2, fma(x2, 1.0 / 24.0, -0.5), 1.0);
  const double2 t = tab[k & (kExpLen - 1)];
  s = fma(t.y, cx, t.x * sx);
  c = fma(t.x, cx, -t.y * sx);
}

// ----------------------------------------------------- interval polynomials
// Cubic Hermite p(s) = c0 + c1 s + c2 s^2 + c3 s^3 on s in [0,1] from values
// y0, y1 and rates r0, r1 over an interval of length h.
__device__ __forceinline__ void hermite(double y0, double d, double r0, double r1, double h, double c[4]) {
  c[0] = y0;
  c[1] = h * r0;
  c[2] = 3.0 * d - h * (2.0 * r0 + r1);
  c[3] = h * (r0 + r1) - 2.0 * d;
}

template <typename T>
__device__ __forceinline__ T poly3(const T c[4], T s) {
  return ((c[3] * s + c[2]) * s + c[1]) * s + c[0];
}

struct IvD {           // FP64 interval data (gm: of 2 gamma~)
  double ph[4], gm[4], al[4], am[4], ec[4];
};

__device__ __forceinline__ double frac0(double hi, double lo) {
  return (hi - floor(hi)) + lo;
}

__device__ __forceinline__ void interval_phase(double ahi, double alo, double ar, double bhi, double blo,
                                               double br, double h, double c[4]) {
  const double d = (bhi - ahi) + (blo - alo);
  hermite(frac0(ahi, alo), d, ar, br, h, c);
}

__device__ void build_iv(const Knot& a, const Knot& b, double h, IvD& o) {
  interval_phase(a.phd_hi, a.phd_lo, a.phd_rate, b.phd_hi, b.phd_lo, b.phd_rate, h, o.ph);
  interval_phase(a.gam_hi, a.gam_lo, a.gam_rate, b.gam_hi, b.gam_lo, b.gam_rate, h, o.gm);
  for (int q = 0; q < 4; ++q) o.gm[q] *= 2.0;   // the kernel uses 2 gamma~ (exact scaling)
  interval_phase(a.alp_hi, a.alp_lo, a.alp_rate, b.alp_hi, b.alp_lo, b.alp_rate, h, o.al);
  hermite(a.amp, b.amp - a.amp, a.amp_rate, b.amp_rate, h, o.am);
  hermite(a.e, b.e - a.e, a.e_rate, b.e_rate, h, o.ec);
}

__device__ __forceinline__ unsigned long long to_q64(double f) {
  f -= floor(f);                                   // [0, 1)
  return (unsigned long long)(f * 18446744073709551616.0);
}

// a per-sample phase increment [cycles] as a signed Q0.64 fraction: the
// phase is kept mod 1, so the increment is reduced to [-1/2, 1/2) first (at
// long sample intervals it exceeds half a cycle)
__device__ __forceinline__ long long to_q64s(double f) {
  f -= rint(f);
  if (f >= 0.5) f -= 1.0;
  return (long long)llrint(f * 18446744073709551616.0);
}

__device__ void build_iv_mixed(const Knot& a, const Knot& b, double h, int ks, IvM& o) {
  double c[4];
  interval_phase(a.phd_hi, a.phd_lo, a.phd_rate, b.phd_hi, b.phd_lo, b.phd_rate, h, c);
  o.ph_base = to_q64(c[0]);
  o.ph_inc = to_q64s(c[1] / ks);
  o.ph_c[0] = (float)c[2];
  o.ph_c[1] = (float)c[3];
  interval_phase(a.gam_hi, a.gam_lo, a.gam_rate, b.gam_hi, b.gam_lo, b.gam_rate, h, c);
  for (int q = 0; q < 4; ++q) c[q] *= 2.0;   // the kernel uses 2 gamma~ (exact scaling)
  o.gm_base = to_q64(c[0]);
  o.gm_inc = to_q64s(c[1] / ks);
  o.gm_c[0] = (float)c[2];
  o.gm_c[1] = (float)c[3];
  interval_phase(a.alp_hi, a.alp_lo, a.alp_rate, b.alp_hi, b.alp_lo, b.alp_rate, h, c);
  o.al_base = to_q64(c[0]);
  o.al_inc = to_q64s(c[1] / ks);
  o.al_c[0] = (float)c[2];
  o.al_c[1] = (float)c[3];
  hermite(a.amp, b.amp - a.amp, a.amp_rate, b.amp_rate, h, c);
  for (int q = 0; q < 4; ++q) o.am[q] = (float)c[q];
  hermite(a.e, b.e - a.e, a.e_rate, b.e_rate, h, c);
  for (int q = 0; q < 4; ++q) o.ec[q] = (float)c[q];
}

// eccentricity on an interval, in the record's precision
__device__ __forceinline__ double iv_e(const IvD& v, double s) { return poly3<double>(v.ec, s); }
__device__ __forceinline__ float iv_e(const IvM& v, float s) { return poly3<float>(v.ec, s); }

static_assert(sizeof(IvM) == kIvMBytes, "interval record size");

// Knots -> mixed interval records, one thread per (interval, walker).
__global__ void k1b_intervals(const Knot* __restrict__ knots, int64_t nk, int ks, double dt, IvM* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int64_t wk = blockIdx.y;
  const Knot* kn = knots + wk * (nk + 1);
  build_iv_mixed(kn[k], kn[k + 1], (double)ks * dt, ks, out[wk * nk + k]);
}

// cos, sin of the LISA orbital phase phibar = 2 pi t / T at the four
// pattern-fit nodes of each 256-sample tile (offsets 0, 256/3, 512/3, 256):
// tab[tile][2q] = cos, tab[tile][2q + 1] = sin.
__global__ void k_lisa_tiles(int64_t ntiles, double t0, double dt, double* __restrict__ tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntiles) return;
  for (int q = 0; q < 4; ++q) {
    double f = (t0 + ((double)(i * 256) + 256.0 * (double)q / 3.0) * dt) / kYear;
    f -= floor(f);
    double sn, cs;
    sincospi(2.0 * f, &sn, &cs);
    tab[i * 8 + 2 * q] = cs;
    tab[i * 8 + 2 * q + 1] = sn;
  }
}

void launch_intervals_mixed(const Knot* knots, int w, int64_t n, int ks, double dt, void* ivs, cudaStream_t s) {
  if (w <= 0) return;
  const int64_t nk = n / ks;
  // walkers on grid y, at most kMaxGridY per launch
  for (int w0 = 0; w0 < w; w0 += kMaxGridY) {
    const int ww = w - w0 < kMaxGridY ? w - w0 : kMaxGridY;
    dim3 g((unsigned)((nk + 127) / 128), (unsigned)ww);
    k1b_intervals<<<g, 128, 0, s>>>(knots + (int64_t)w0 * (nk + 1), nk, ks, dt, (IvM*)ivs + (int64_t)w0 * nk);
  }
}

void launch_lisa_tiles(int64_t n, double t0, double dt, double* tab, cudaStream_t s) {
  const int64_t nt = n / 256;
  k_lisa_tiles<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(nt, t0, dt, tab);
}

// fixed-point phase: (base + tau*inc) mod 1 to 32 bits, plus the FP32
// correction c2 s^2 + c3 s^3; returns the phase in cycles in [-0.5, 0.5)
__device__ __forceinline__ float phase_fx(unsigned long long base, long long inc, const float c[2], int tau,
                                          float s) {
  const unsigned long long p = base + (unsigned long long)tau * (unsigned long long)inc;   // mod 2^64
  const int top = (int)(unsigned)(p >> 32);
  float f = (float)top * 2.3283064365386963e-10f;  // 2^-32
  f += (c[1] * s + c[0]) * s * s;
  return f - rintf(f);
}

// --------------------------------------------------- response + harmonics
template <typename T>
__device__ __forceinline__ T rcp_fast(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ float rcp_fast<float>(float x) { return __fdividef(1.f, x); }

// (x, y) -> (cos 2 atan2(y, x), sin 2 atan2(y, x)); (1, 0) when degenerate
template <typename T>
__device__ __forceinline__ void double_angle(T x, T y, T& c2, T& s2, bool degenerate) {
  const T r2 = x * x + y * y;
  if (degenerate || !(r2 > T(0))) {
    c2 = T(1);
    s2 = T(0);
  } else {
    const T inv = rcp_fast(r2);
    c2 = (x * x - y * y) * inv;
    s2 = T(2) * x * y * inv;
  }
}

// cos(n Phi), sin(n Phi) for n = 1, 2, ...: complex rotation (FP32) or the
// Chebyshev three-term recurrence c_{n+1} = 2 cos(Phi) c_n - c_{n-1} (FP64,
// whose error growth ~n^2 eps is harmless at n <= 32 in double).
template <typename T>
struct HarmStep {
  T cn, sn, cp, sp, c1, s1;
  __device__ __forceinline__ void init(T c, T s) {
    cn = c; sn = s; cp = T(1); sp = T(0); c1 = c; s1 = s;
  }
  __device__ __forceinline__ void next();
};
template <>
__device__ __forceinline__ void HarmStep<double>::next() {
  const double tc = 2.0 * c1 * cn - cp, ts = 2.0 * c1 * sn - sp;
  cp = cn; sp = sn; cn = tc; sn = ts;
}

// a_n, b_n, c_n of harmonic index n at fit time st (FP64 layout: 9 per harmonic)
__device__ __forceinline__ void amps_at(const double* __restrict__ bq, int n, double st, double& an, double& bn,
                                        double& rn) {
  const double* b = bq + 9 * n;
  an = (b[2] * st + b[1]) * st + b[0];
  bn = (b[5] * st + b[4]) * st + b[3];
  rn = (b[8] * st + b[7]) * st + b[6];
}

// Harmonic sums at one sample (FP64): Cs = sum_n a_n cos(n Phi), Ss =
// sum_n b_n sin(n Phi), Rs = sum_n c_n cos(n Phi), with the amplitudes from
// the tile's fit bq at time st in [0, 1]; cph/sph: cos/sin of the Doppler
// orbital phase; (cos, sin)(n Phi) by the Chebyshev recurrence.
__device__ __forceinline__ void harmonic_sums(double cph, double sph, double st, const double* __restrict__ bq,
                                              int n_max, double& Cs, double& Ss, double& Rs) {
  Cs = 0.0;
  Ss = 0.0;
  Rs = 0.0;
  HarmStep<double> hs;
  hs.init(cph, sph);
  for (int n = 0; n < n_max; ++n) {
    double an, bn, rn;
    amps_at(bq, n, st, an, bn, rn);
    Cs += an * hs.cn;
    Ss += bn * hs.sn;
    Rs += rn * hs.cn;
    hs.next();
  }
}

// FP32 amplitude coefficients per harmonic, each stored twice so that the
// paired (f32x2) instructions of harmonic_sums4 take natural register pairs:
// (a0 a0 a1 a1)(a2 a2 b0 b0)(b1 b1 b2 b2)(r0 r0 r1 r1)(r2 r2 - -).
constexpr int kAmpStrideM = 20;

// ----------------------------------------------------------- response
// The LISA response of Sec. 2 (Eq. 2 with the Barack-Cutler antenna
// patterns) contracts the detector tensor with the polarisation tensors, and
// the AK polarisations are the transverse-traceless projection of the
// orbit's quadrupole tensor
//   M = X (u1 u1 - u2 u2) + Y (u1 u2 + u2 u1) + Rs (u1 u1 + u2 u2),
// u1, u2 the orbital-plane basis of Geo (pericentre at angle gamma~ from u1),
// (X, Y) the harmonic sums (Cs, Ss) rotated by 2 gamma~.  The contraction does
// not depend on the polarisation basis, so it is taken in the fixed sky basis
// (P, Q) of Geo: the angle beta and the L-dependent polarisation angle psi
// drop out, and
//   h_I = F+_I H+ + Fx_I Hx,  H+ + i Hx = (Rs + X) z1^2 + (Rs - X) z2^2 + 2 Y z1 z2,
// z_k = P.u_k + i Q.u_k, with F_I, F_II the antenna patterns at the
// polarisation angle psi_P of P (tan psi_P = (z_d.Q)/(z_d.P), z_d the
// detector normal).  The patterns depend on time only through the LISA
// orbital phase phibar, a one-year period, so each tile fits them by a cubic.

// The four patterns (sqrt3/2 F+_I, sqrt3/2 Fx_I, sqrt3/2 F+_II, sqrt3/2 Fx_II)
// times scale at phibar = atan2(sb, cb): detector-frame polar angle
// cos(theta_d) = z_d.N, azimuth phi_d = phibar + atan2(sqrt3 cos thS + sin thS
// cos(phibar - phS), 2 sin thS sin(phibar - phS)), channel II at phi_d - pi/4.
template <typename T>
__device__ __forceinline__ void antenna_fixed(const Geo<T>& g, T cb, T sb, T scale, T F[4]) {
  const T h3 = T(kSqrt3Half);
  const T cdp = cb * g.cos_phs + sb * g.sin_phs;
  const T sdp = sb * g.cos_phs - cb * g.sin_phs;
  const T ct = T(0.5) * g.cos_ths - h3 * g.sin_ths * cdp;
  T c2x, s2x, c2p, s2p;
  double_angle<T>(T(2) * g.sin_ths * sdp, T(1.7320508075688772) * g.cos_ths + g.sin_ths * cdp, c2x, s2x, false);
  double_angle<T>(h3 * sdp, h3 * g.cos_ths * cdp + T(0.5) * g.sin_ths, c2p, s2p, false);
  const T c2b = cb * cb - sb * sb, s2b = T(2) * sb * cb;
  const T c2f = c2b * c2x - s2b * s2x;   // cos, sin of 2 phi_d
  const T s2f = s2b * c2x + c2b * s2x;
  const T q = T(0.5) * (T(1) + ct * ct);
  const T k = h3 * scale;
  F[0] = k * (q * c2f * c2p - ct * s2f * s2p);
  F[1] = k * (q * c2f * s2p + ct * s2f * c2p);
  F[2] = k * (q * s2f * c2p + ct * c2f * s2p);
  F[3] = k * (q * s2f * s2p - ct * c2f * c2p);
}

// Cubic c0 + c1 s + c2 s^2 + c3 s^3 through y0..y3 at s = 0, 1/3, 2/3, 1
// (Newton forward differences in u = 3 s).
template <typename T>
__device__ __forceinline__ void fit_cubic4(T y0, T y1, T y2, T y3, T* c) {
  const T d1 = y1 - y0, d2 = (y2 - y1) - d1, d3 = ((y3 - y2) - (y2 - y1)) - d2;
  c[0] = y0;
  c[1] = T(3) * (d1 - T(0.5) * d2 + d3 * T(1.0 / 3.0));
  c[2] = T(4.5) * (d2 - d3);
  c[3] = T(4.5) * d3;
}

template <typename T>
__device__ __forceinline__ T cubic_at(const T* c, T s) {
  return ((c[3] * s + c[2]) * s + c[1]) * s + c[0];
}

// Channels from the harmonic sums at one sample.  c2gt/s2gt: cos/sin of
// 2 gamma~; ca/sa: of alpha; A = x^(2/3); F: the four patterns at the sample.
template <typename T>
__device__ __forceinline__ void response(const Geo<T>& g, T c2gt, T s2gt, T ca, T sa, T A, T Cs, T Ss, T Rs,
                                         const T F[4], T& hI, T& hII) {
  const T z1r = sa * g.pe1 - ca * g.pe2, z1i = sa * g.qe1 - ca * g.qe2;
  const T z2r = ca * g.cpe1 + sa * g.cpe2 - g.spS, z2i = ca * g.cqe1 + sa * g.cqe2 - g.sqS;
  const T X = Cs * c2gt - Ss * s2gt, Y = Cs * s2gt + Ss * c2gt;
  const T a = A * (Rs + X), b = A * (Rs - X), y = T(2) * A * Y;
  const T Hp = a * (z1r * z1r - z1i * z1i) + b * (z2r * z2r - z2i * z2i) + y * (z1r * z2r - z1i * z2i);
  const T Hx = T(2) * (a * (z1r * z1i) + b * (z2r * z2i)) + y * (z1r * z2i + z1i * z2r);
  hI = F[0] * Hp + F[1] * Hx;
  hII = F[2] * Hp + F[3] * Hx;
}

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// response<float> for two samples at once, every quantity a (sample A,
// sample B) pair and every step one paired FP32 instruction.  gk: the
// walker's geometry constants as duplicated pairs,
//   gk[0] = (pe1 pe1 -pe2 -pe2), gk[1] = (qe1 qe1 -qe2 -qe2),
//   gk[2] = (cpe1 cpe1 cpe2 cpe2), gk[3] = (cqe1 cqe1 cqe2 cqe2),
//   gk[4] = (-spS -spS -sqS -sqS).
__device__ __forceinline__ void response_pair(const float4* gk, float2 c2gt, float2 s2gt, float2 ca, float2 sa,
                                              float2 A, float2 Cs, float2 Ss, float2 Rs, const float2 F[4],
                                              float2& hI, float2& hII) {
  const float4 k0 = gk[0], k1 = gk[1], k2 = gk[2], k3 = gk[3], k4 = gk[4];
  const float2 z1r = __ffma2_rn(sa, lo2(k0), __fmul2_rn(ca, hi2(k0)));
  const float2 z1i = __ffma2_rn(sa, lo2(k1), __fmul2_rn(ca, hi2(k1)));
  const float2 z2r = __ffma2_rn(ca, lo2(k2), __ffma2_rn(sa, hi2(k2), lo2(k4)));
  const float2 z2i = __ffma2_rn(ca, lo2(k3), __ffma2_rn(sa, hi2(k3), hi2(k4)));
  const float2 X = __ffma2_rn(Cs, c2gt, neg2(__fmul2_rn(Ss, s2gt)));
  const float2 Y = __ffma2_rn(Cs, s2gt, __fmul2_rn(Ss, c2gt));
  const float2 a = __fmul2_rn(A, __fadd2_rn(Rs, X));
  const float2 b = __fmul2_rn(A, __fadd2_rn(Rs, neg2(X)));
  const float2 y = __fmul2_rn(__fadd2_rn(A, A), Y);
  const float2 u1 = __ffma2_rn(z1r, z1r, neg2(__fmul2_rn(z1i, z1i)));
  const float2 u2 = __ffma2_rn(z2r, z2r, neg2(__fmul2_rn(z2i, z2i)));
  const float2 u3 = __ffma2_rn(z1r, z2r, neg2(__fmul2_rn(z1i, z2i)));
  const float2 Hp = __ffma2_rn(a, u1, __ffma2_rn(b, u2, __fmul2_rn(y, u3)));
  const float2 v3 = __ffma2_rn(z1r, z2i, __fmul2_rn(z1i, z2r));
  const float2 w = __ffma2_rn(a, __fmul2_rn(z1r, z1i), __fmul2_rn(b, __fmul2_rn(z2r, z2i)));
  const float2 Hx = __ffma2_rn(y, v3, __fadd2_rn(w, w));
  hI = __ffma2_rn(F[0], Hp, __fmul2_rn(F[1], Hx));
  hII = __ffma2_rn(F[2], Hp, __fmul2_rn(F[3], Hx));
}

// Channels at one sample (harmonic sums, then the response).
__device__ __forceinline__ void channels(const Geo<double>& g, double cph, double sph, double c2gt, double s2gt,
                                         double ca, double sa, double A, double st, const double* __restrict__ bq,
                                         int n_max, const double F[4], double& hI, double& hII) {
  double Cs, Ss, Rs;
  harmonic_sums(cph, sph, st, bq, n_max, Cs, Ss, Rs);
  response<double>(g, c2gt, s2gt, ca, sa, A, Cs, Ss, Rs, F, hI, hII);
}


// FP32, four samples at once, as two (A, B) pairs of every quantity --
// cos(n Phi), sin(n Phi), the three amplitudes and the three sums -- so each
// step is one paired (f32x2) instruction on operands that are natural
// register pairs, and the coefficients of a harmonic (five 16-byte loads) are
// loaded once for all four samples.  c1, s1: cos, sin of the Doppler orbital
// phase; st: fit times in [0, 1]; C, S, R: sum_n a_n cos(n Phi),
// sum_n b_n sin(n Phi), sum_n c_n cos(n Phi).
__device__ __forceinline__ void harmonic_sums4(const float2 (&c1)[2], const float2 (&s1)[2], const float2 (&st)[2],
                                               const float* __restrict__ bq, int n_max, bool cheb, float2 (&C)[2],
                                               float2 (&S)[2], float2 (&R)[2]) {
  for (int p = 0; p < 2; ++p) C[p] = S[p] = R[p] = make_float2(0.f, 0.f);
  auto harm = [&](int n, const float2 (&c)[2], const float2 (&sn)[2]) {
    const float4* b = reinterpret_cast<const float4*>(bq + kAmpStrideM * n);
    const float4 x0 = b[0], x1 = b[1], x2 = b[2], x3 = b[3], x4 = b[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 a = __ffma2_rn(__ffma2_rn(make_float2(x1.x, x1.y), st[p], make_float2(x0.z, x0.w)), st[p],
                                  make_float2(x0.x, x0.y));
      const float2 bb = __ffma2_rn(__ffma2_rn(make_float2(x2.z, x2.w), st[p], make_float2(x2.x, x2.y)), st[p],
                                   make_float2(x1.z, x1.w));
      const float2 r = __ffma2_rn(__ffma2_rn(make_float2(x4.x, x4.y), st[p], make_float2(x3.z, x3.w)), st[p],
                                  make_float2(x3.x, x3.y));
      C[p] = __ffma2_rn(a, c[p], C[p]);
      S[p] = __ffma2_rn(bb, sn[p], S[p]);
      R[p] = __ffma2_rn(r, c[p], R[p]);
    }
  };
  float2 cu[2] = {c1[0], c1[1]}, su[2] = {s1[0], s1[1]};
  int n = 0;
  if (cheb) {
    const float2 tc[2] = {make_float2(2.f * c1[0].x, 2.f * c1[0].y), make_float2(2.f * c1[1].x, 2.f * c1[1].y)};
    float2 cv[2] = {make_float2(1.f, 1.f), make_float2(1.f, 1.f)}, sv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (; n + 1 < n_max; n += 2) {
      harm(n, cu, su);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        cv[p] = __ffma2_rn(tc[p], cu[p], make_float2(-cv[p].x, -cv[p].y));
        sv[p] = __ffma2_rn(tc[p], su[p], make_float2(-sv[p].x, -sv[p].y));
      }
      harm(n + 1, cv, sv);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        cu[p] = __ffma2_rn(tc[p], cv[p], make_float2(-cu[p].x, -cu[p].y));
        su[p] = __ffma2_rn(tc[p], sv[p], make_float2(-su[p].x, -su[p].y));
      }
    }
  } else {
    const float2 ns[2] = {make_float2(-s1[0].x, -s1[0].y), make_float2(-s1[1].x, -s1[1].y)};
    for (; n + 1 < n_max; n += 2) {
      harm(n, cu, su);
      float2 cv[2], sv[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        cv[p] = __ffma2_rn(cu[p], c1[p], __fmul2_rn(su[p], ns[p]));
        sv[p] = __ffma2_rn(su[p], c1[p], __fmul2_rn(cu[p], s1[p]));
      }
      harm(n + 1, cv, sv);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        cu[p] = __ffma2_rn(cv[p], c1[p], __fmul2_rn(sv[p], ns[p]));
        su[p] = __ffma2_rn(sv[p], c1[p], __fmul2_rn(cv[p], s1[p]));
      }
    }
  }
  if (n < n_max) harm(n, cu, su);
}

// Per-harmonic amplitude coefficients in shared memory: 9 values (a, b, c
// quadratics) at stride AmpStride<T>; FP32 stores each twice in the layout
// of harmonic_sums4 (five 16-byte loads per harmonic).
template <typename T>
struct AmpStride;
template <>
struct AmpStride<double> {
  static constexpr int v = 9;
};
template <>
struct AmpStride<float> {
  static constexpr int v = kAmpStrideM;
};

// Bessel amplitude fit for the tile: nodes at tile-relative sample offsets
// 0, L/2, L (L = 256, or the last valid offset when the orbit plunges inside
// the tile), quadratic in st = t / L.
template <typename T, typename IV>
__device__ __forceinline__ void tile_harmonics(const IV* iv, int ni, int64_t j0, int64_t kfirst, int ks,
                                               int n_max, int span, T* bnode, T* bq, const T* __restrict__ bc,
                                               const T* __restrict__ ifact) {
  const int t = threadIdx.x;
  if (t < 3 * n_max) {
    // harmonic-major: a warp holds neighbouring n, whose series lengths
    // (growing with x = n e) are alike
    const int node = t % 3, n = t / 3 + 1;
    // node at offset span*node/2: integer arithmetic in half samples, so no
    // FP64 instruction runs here in the FP32 kernel
    const int64_t pos2 = 2 * j0 + (int64_t)span * node;
    int64_t ki = pos2 / (2 * ks) - kfirst;
    if (ki > ni - 1) ki = ni - 1;
    if (ki < 0) ki = 0;
    const int64_t rem2 = pos2 - 2 * (kfirst + ki) * ks;
    const T s = T(rem2) / T(2 * ks);
    const T e = T(iv_e(iv[ki], s));
    T out[3];
    harmonic_amps<T>(n, e, out, bc, ifact);
    bnode[(node * 32 + (n - 1)) * 3 + 0] = out[0];
    bnode[(node * 32 + (n - 1)) * 3 + 1] = out[1];
    bnode[(node * 32 + (n - 1)) * 3 + 2] = out[2];
  }
  __syncthreads();
  if (t < 3 * n_max) {
    const int n = t / 3, f = t % 3;
    const T f0 = bnode[(0 * 32 + n) * 3 + f], fh = bnode[(1 * 32 + n) * 3 + f], f1 = bnode[(2 * 32 + n) * 3 + f];
    const T q0 = f0, q1 = T(-3) * f0 + T(4) * fh - f1, q2 = T(2) * f0 - T(4) * fh + T(2) * f1;
    T* o = bq + AmpStride<T>::v * n;
    if (sizeof(T) == 4) {                // FP32: quantity f, coefficient p at 6 f + 2 p and the next
      o[6 * f + 0] = q0;
      o[6 * f + 1] = q0;
      o[6 * f + 2] = q1;
      o[6 * f + 3] = q1;
      o[6 * f + 4] = q2;
      o[6 * f + 5] = q2;
    } else {
      o[3 * f + 0] = q0;
      o[3 * f + 1] = q1;
      o[3 * f + 2] = q2;
    }
  }
}

// span of the Bessel fit: the L samples from j0, or up to the last sample
// before a plunge
__device__ __forceinline__ int tile_span(int64_t j0, int64_t jp, int L = kTile) {
  if (jp >= j0 + L) return L;
  const int64_t l = jp - 1 - j0;
  return l < 1 ? 1 : (int)l;
}

// ------------------------------------------------------------- kernels
template <typename T>
__device__ __forceinline__ void fit3(T f0, T fh, T f1, T* q) {
  q[0] = f0;
  q[1] = T(-3) * f0 + T(4) * fh - f1;
  q[2] = T(2) * f0 - T(4) * fh + T(2) * f1;
}

// Above these sample intervals the per-tile cubic of the antenna patterns
// (error ~ (256 dt / T)^4) is replaced by their exact value per sample.
constexpr double kPatternFitDtMax64 = 64.0;     // [s]; fit error < 2e-12 below
constexpr double kPatternFitDtMaxM = 1024.0;    // [s]; fit error < 1e-7 below

// FP64 kernel: one CTA per segment of kSegF = 1024 samples (four tiles of
// 256; each thread evaluates its offset in the four tiles in turn), so the
// Bessel amplitude fit is made once per 1024 samples (its error over that
// span is ~1e-14 of the amplitudes) and the set-up's FP64 work, ~6 % of the
// kernel's at one fit per tile, drops four-fold.
constexpr int kSegF = 1024;

__global__ void __launch_bounds__(kTile, 2) k2_wave_f64(const Knot* __restrict__ knots, const WalkerC* __restrict__ wcs,
                                                        int64_t n, double dt, double t0, int ks, int n_max,
                                                        double2* __restrict__ z, int unit_scale, int exact_f,
                                                        const double* __restrict__ bc, const double* __restrict__ ifact,
                                                        const double* __restrict__ lisa) {
  constexpr int kTiles = kSegF / kTile;
  __shared__ IvD iv[kSegF / 64];
  __shared__ double bnode[3 * 32 * 3];
  __shared__ double bq[32 * 9];
  __shared__ double fn[kTiles][4][4];   // the four patterns at the four fit nodes of each tile
  __shared__ double fq[kTiles][4][4];   // their cubics in (t mod 256) / 256
  __shared__ double2 ex[kExpLen];
  __shared__ Geo<double> g;
  const int wk = blockIdx.y;
  const WalkerC& C = wcs[wk];
  const int64_t nk = n / ks;
  const Knot* kn = knots + (int64_t)wk * (nk + 1);
  const int64_t j0 = (int64_t)blockIdx.x * kSegF;
  const int64_t kfirst = j0 / ks;
  const int ni = ks >= kSegF ? 1 : kSegF / ks;
  const int t = threadIdx.x;
  const double h = (double)ks * dt;
  const double scale = unit_scale ? C.gd.amp_scale : 1.0;
  if (t < ni) build_iv(kn[kfirst + t], kn[kfirst + t + 1], h, iv[t]);
  if (t >= 224 && t < 224 + 4 * kTiles && !exact_f) {   // node q of tile tt
    const int i = t - 224, tt = i / 4, q = i % 4;
    const double* L = lisa + ((int64_t)blockIdx.x * kTiles + tt) * 8 + 2 * q;
    antenna_fixed<double>(C.gd, L[0], L[1], scale, fn[tt][q]);
  }
  if (t == 160) g = C.gd;
  for (int i = t; i < kExpLen; i += kTile) ex[i] = g_exp512[i];
  __syncthreads();
  if (t >= 224 && t < 224 + 4 * kTiles && !exact_f) {   // pattern q of tile tt
    const int i = t - 224, tt = i / 4, q = i % 4;
    fit_cubic4<double>(fn[tt][0][q], fn[tt][1][q], fn[tt][2][q], fn[tt][3][q], fq[tt][q]);
  }
  const int64_t jplunge = C.j_plunge;
  const int span = tile_span(j0, jplunge, kSegF);
  tile_harmonics<double, IvD>(iv, ni, j0, kfirst, ks, n_max, span, bnode, bq, bc, ifact);
  __syncthreads();
  const double inv_span = 1.0 / (double)span;
  const int lks = __ffs(ks) - 1;   // ks: a power of two
  const double so = (double)t * (1.0 / kTile);
#pragma unroll 1
  for (int tt = 0; tt < kTiles; ++tt) {
    const int r = tt * kTile + t;   // offset in the segment
    const int64_t j = j0 + r;
    double2 out = make_double2(0.0, 0.0);
    if (j < jplunge) {
      const int ki = ks >= kSegF ? 0 : r >> lks;
      const double s = (double)(j - (kfirst + ki) * ks) * (1.0 / (double)ks);
      const IvD& v = iv[ki];
      // phases in cycles over the knot interval (|f| < 2^20: the table index
      // wraps them, no reduction to one cycle is needed)
      const double fph = poly3<double>(v.ph, s);
      const double fgm = poly3<double>(v.gm, s);
      const double fal = poly3<double>(v.al, s);
      const double A = poly3<double>(v.am, s);
      double F[4];
      if (!exact_f) {
#pragma unroll
        for (int q = 0; q < 4; ++q) F[q] = cubic_at<double>(fq[tt][q], so);
      } else {
        double f = (t0 + (double)j * dt) / kYear;
        f -= floor(f);
        double sb, cb;
        sincospi(2.0 * f, &sb, &cb);
        antenna_fixed<double>(g, cb, sb, scale, F);
      }
      double sph, cph, s2g, c2g, sa, ca;
      sincos2pi_tab(fph, ex, sph, cph);
      sincos2pi_tab(fgm, ex, s2g, c2g);
      sincos2pi_tab(fal, ex, sa, ca);
      double hI, hII;
      channels(g, cph, sph, c2g, s2g, ca, sa, A, (double)r * inv_span, bq, n_max, F, hI, hII);
      out = make_double2(hI, hII);
    }
    z[(int64_t)wk * n + j] = out;
  }
}

// Mixed kernel: one CTA per segment of kSegM = 1024, 2048 or 4096 samples
// (tiles of 256, four per pass of the sample loop: each thread evaluates the
// samples at its offset in four tiles at once, four CTAs per SM at 64
// registers: as fast as three at 78 alone, and one CTA's registers then hold
// a pass-2 CTA of the pipelined schedule), so the Bessel amplitude
// fit -- a quadratic in time per harmonic, from three nodes -- is made once
// per segment.  The eccentricity moves by ~1e-4 relative per 256 samples, and
// the fit's error grows as the cube of the segment: ~5e-14 of the amplitudes
// over 2048 samples, far below FP32 resolution.  Longer segments spend less
// of the kernel in that set-up (its barrier waits); the launch takes the
// length from the series length alone (at least 16 segments per walker).
//
// exact_f: exact patterns per sample (long sample intervals), dphib: the
// LISA orbital phase step per sample [cycles] for them.  No FP64 instruction
// runs per thread: e0 is tested once per CTA.
template <int kSegM, bool kOneIv>
__global__ void __launch_bounds__(kTile, 4) k2_wave_mixed(const Knot* __restrict__ knots, const WalkerC* __restrict__ wcs,
                                                          int64_t n, int exact_f, float dphib, int ks, int n_max,
                                                          float2* __restrict__ z, int unit_scale,
                                                          const float* __restrict__ bc, const float* __restrict__ ifact,
                                                          const double* __restrict__ lisa, const IvM* __restrict__ ivs) {
  __shared__ IvM iv[kSegM / 64];
  __shared__ float bnode[3 * 32 * 3];
  __shared__ __align__(16) float bq[32 * kAmpStrideM];
  constexpr int kTiles = kSegM / kTile;
  static_assert(kTiles % 4 == 0, "tiles are processed in fours");
  __shared__ float fn[kTiles][4][4];   // the four patterns at the fit nodes of each tile
  // their cubics in (t mod 256) / 256, tiles paired: fq2[m][q][k] = (tile 2m, tile 2m + 1)
  __shared__ __align__(16) float2 fq2[kTiles / 2][4][4];
  __shared__ float cs0[kTiles][2];     // cos, sin phibar at each tile's start
  __shared__ Geo<float> g;
  __shared__ float4 gk[5];             // response_pair's duplicated geometry constants
  __shared__ int64_t jplunge;
  __shared__ int cheb_s;
  const int wk = blockIdx.y;
  const WalkerC& C = wcs[wk];
  const int64_t nk = n / ks;
  const int64_t j0 = (int64_t)blockIdx.x * kSegM;
  const int64_t kfirst = j0 / ks;
  const int ni = ks >= kSegM ? 1 : kSegM / ks;
  const int t = threadIdx.x;
  const float scale = unit_scale ? C.gf.amp_scale : 1.f;
  if (t < ni) iv[t] = ivs[(int64_t)wk * nk + kfirst + t];
  if (t >= 128 && t < 128 + 4 * kTiles) {   // node q of tile tt
    const int i = t - 128, tt = i / 4, q = i % 4;
    const double* L = lisa + (blockIdx.x * kTiles + tt) * 8 + 2 * q;
    const float cb = (float)L[0], sb = (float)L[1];
    antenna_fixed<float>(C.gf, cb, sb, scale, fn[tt][q]);
    if (q == 0) {
      cs0[tt][0] = cb;
      cs0[tt][1] = sb;
    }
  }
  if (t == 224) {
    const Geo<float>& G = C.gf;
    g = G;
    gk[0] = make_float4(G.pe1, G.pe1, -G.pe2, -G.pe2);
    gk[1] = make_float4(G.qe1, G.qe1, -G.qe2, -G.qe2);
    gk[2] = make_float4(G.cpe1, G.cpe1, G.cpe2, G.cpe2);
    gk[3] = make_float4(G.cqe1, G.cqe1, G.cqe2, G.cqe2);
    gk[4] = make_float4(-G.spS, -G.spS, -G.sqS, -G.sqS);
    jplunge = C.j_plunge;
    cheb_s = C.e0 < 0.5;
  }
  __syncthreads();
  if (t >= 128 && t < 128 + 4 * kTiles) {   // pattern q of tile tt
    const int i = t - 128, tt = i / 4, q = i % 4;
    float cf[4];
    fit_cubic4<float>(fn[tt][0][q], fn[tt][1][q], fn[tt][2][q], fn[tt][3][q], cf);
    float* o = reinterpret_cast<float*>(&fq2[tt >> 1][q][0]) + (tt & 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) o[2 * k] = cf[k];
  }
  const int span = tile_span(j0, jplunge, kSegM);
  const bool cheb = cheb_s != 0;   // per walker (uniform in the CTA)
  tile_harmonics<float, IvM>(iv, ni, j0, kfirst, ks, n_max, span, bnode, bq, bc, ifact);
  __syncthreads();
  const float inv_span = 1.f / (float)span;
  const float inv_ks = 1.f / (float)ks;
  const int lks = __ffs(ks) - 1;   // ks is a power of two: the interval index by a shift
  constexpr float kTwoPiF = 6.283185307179586f;
  // per-sample inputs: the orbital phase (for the harmonic sums) first, the
  // response's angles and amplitude after the sums (fewer registers live
  // across the harmonic loop)
  // knot interval ki and offset tau in it of sample r; with K_s >= four
  // tiles (kOneIv) the four samples of a pass share the interval of the
  // first, so its record is read once for the four
  auto interval = [&](const int (&r)[4], int i, int& ki, int& tau) {
    ki = ks >= kSegM ? 0 : (kOneIv ? r[0] : r[i]) >> lks;
    tau = r[i] - ki * ks;
  };
  auto orb = [&](int ki, int tau, float& cph, float& sph) {
    const float s = (float)tau * inv_ks;
    const IvM& v = iv[ki];
    const float fph = phase_fx(v.ph_base, v.ph_inc, v.ph_c, tau, s);
    __sincosf(kTwoPiF * fph, &sph, &cph);
  };
  auto resp_in = [&](int ki, int tau, float& c2g, float& s2g, float& ca, float& sa, float& A) {
    const float s = (float)tau * inv_ks;
    const IvM& v = iv[ki];
    const float fgm = phase_fx(v.gm_base, v.gm_inc, v.gm_c, tau, s);   // 2 gamma~
    const float fal = phase_fx(v.al_base, v.al_inc, v.al_c, tau, s);
    A = poly3<float>(v.am, s);
    __sincosf(kTwoPiF * fgm, &s2g, &c2g);
    __sincosf(kTwoPiF * fal, &sa, &ca);
  };
  // the four patterns at offset t of tiles tt (even) and tt + 1, paired
  const float so = (float)t * (1.f / kTile);
  const float2 so2 = make_float2(so, so);
  auto patterns2 = [&](int tt, float2 F[4]) {
    if (!exact_f) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2* c = fq2[tt >> 1][q];
        F[q] = __ffma2_rn(__ffma2_rn(__ffma2_rn(c[3], so2, c[2]), so2, c[1]), so2, c[0]);
      }
    } else {
      float sd, cd, FA[4], FB[4];
      __sincosf(kTwoPiF * dphib * (float)t, &sd, &cd);
      antenna_fixed<float>(g, cs0[tt][0] * cd - cs0[tt][1] * sd, cs0[tt][1] * cd + cs0[tt][0] * sd, scale, FA);
      antenna_fixed<float>(g, cs0[tt + 1][0] * cd - cs0[tt + 1][1] * sd, cs0[tt + 1][1] * cd + cs0[tt + 1][0] * sd,
                           scale, FB);
#pragma unroll
      for (int q = 0; q < 4; ++q) F[q] = make_float2(FA[q], FB[q]);
    }
  };
  // four samples per thread (tiles tt..tt+3, offset t): the amplitude
  // coefficients of each harmonic are loaded once for all four
#pragma unroll 1
  for (int tt = 0; tt < kTiles; tt += 4) {
    int r[4], ki[4], tau[4];
    float2 c1[2], s1[2], st[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = (tt + i) * kTile + t;
#pragma unroll
    for (int i = 0; i < 4; ++i) interval(r, i, ki[i], tau[i]);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float ca_, sa_, cb_, sb_;
      orb(ki[2 * p], tau[2 * p], ca_, sa_);
      orb(ki[2 * p + 1], tau[2 * p + 1], cb_, sb_);
      c1[p] = make_float2(ca_, cb_);
      s1[p] = make_float2(sa_, sb_);
      st[p] = make_float2((float)r[2 * p] * inv_span, (float)r[2 * p + 1] * inv_span);
    }
    float2 Cs[2], Ss[2], Rs[2];
    harmonic_sums4(c1, s1, st, bq, n_max, cheb, Cs, Ss, Rs);
#pragma unroll
    for (int p = 0; p < 2; ++p) {   // samples r[2p] (x) and r[2p + 1] (y)
      float2 c2g, s2g, ca, sa, A, F[4], hI, hII;
      resp_in(ki[2 * p], tau[2 * p], c2g.x, s2g.x, ca.x, sa.x, A.x);
      resp_in(ki[2 * p + 1], tau[2 * p + 1], c2g.y, s2g.y, ca.y, sa.y, A.y);
      patterns2(tt + 2 * p, F);
      response_pair(gk, c2g, s2g, ca, sa, A, Cs[p], Ss[p], Rs[p], F, hI, hII);
      const int64_t ja = j0 + r[2 * p], jb = j0 + r[2 * p + 1];
      z[(int64_t)wk * n + ja] = ja < jplunge ? make_float2(hI.x, hII.x) : make_float2(0.f, 0.f);
      z[(int64_t)wk * n + jb] = jb < jplunge ? make_float2(hI.y, hII.y) : make_float2(0.f, 0.f);
    }
  }
}

void launch_wave(const Knot* knots, const WalkerC* wc, int w, int64_t n, double dt, double t0,
                 const OptsN& o, void* z, bool unit_scale, const BesselTab& bt, const double* lisa, const void* ivs,
                 cudaStream_t s) {
  if (w <= 0) return;
  const int64_t nk = n / o.ks;
  // walkers on grid y, at most kMaxGridY per launch
  for (int w0 = 0; w0 < w; w0 += kMaxGridY) {
    const int ww = w - w0 < kMaxGridY ? w - w0 : kMaxGridY;
    const Knot* kn = knots + (int64_t)w0 * (nk + 1);
    if (o.precision == 0) {
      dim3 grid((unsigned)(n / kSegF), (unsigned)ww);
      k2_wave_f64<<<grid, kTile, 0, s>>>(kn, wc + w0, n, dt, t0, o.ks, o.n_max, (double2*)z + (int64_t)w0 * n,
                                         unit_scale ? 1 : 0, dt > kPatternFitDtMax64 ? 1 : 0, bt.c64, bt.f64, lisa);
    } else {
      // segment length from the series length alone (so a walker's result
      // does not depend on the batch it is in): at least 16 segments per
      // walker, 1024 to 4096 samples
      const int seg = n >= (1 << 16) ? 4096 : n >= (1 << 15) ? 2048 : 1024;
      dim3 grid((unsigned)(n / seg), (unsigned)ww);
      const int ef = dt > kPatternFitDtMaxM ? 1 : 0;
      const float dpb = (float)(dt / kYear);
      float2* zz = (float2*)z + (int64_t)w0 * n;
      const IvM* iv = (const IvM*)ivs + (int64_t)w0 * nk;
      const int us = unit_scale ? 1 : 0;
#define EMRI_WAVE_MIXED(SEG, ONE) \
  k2_wave_mixed<SEG, ONE><<<grid, kTile, 0, s>>>(kn, wc + w0, n, ef, dpb, o.ks, o.n_max, zz, us, bt.c32, bt.f32, lisa, iv)
      const bool one = o.ks >= 4 * kTile;   // one knot interval per pass of four samples
      if (seg == 4096) {
        if (one) EMRI_WAVE_MIXED(4096, true); else EMRI_WAVE_MIXED(4096, false);
      } else if (seg == 2048) {
        if (one) EMRI_WAVE_MIXED(2048, true); else EMRI_WAVE_MIXED(2048, false);
      } else {
        if (one) EMRI_WAVE_MIXED(1024, true); else EMRI_WAVE_MIXED(1024, false);
      }
#undef EMRI_WAVE_MIXED
    }
  }
}

}  // namespace emri
