// emri_common.cuh -- device-side constants, per-walker records and
// double-double arithmetic shared by the libemri kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace emri {

// ----------------------------------------------------------------- constants
// cgs units (paper Sec. 2); standard values, written as their doubles.
constexpr double kGMsun = 1.32712440018e26;   // G M_sun [cm^3 s^-2]
constexpr double kC = 2.99792458e10;          // speed of light [cm/s]
constexpr double kMpc = 3.0856775814913673e24;// megaparsec [cm]
constexpr double kAUc = 499.004783836;        // 1 AU / c [s]
constexpr double kYear = 31557600.0;          // LISA orbital period [s]
constexpr double kPi = 3.141592653589793;
constexpr double kTwoPiHi = 6.283185307179586;        // 2 pi = hi + lo
constexpr double kTwoPiLo = 2.4492935982947064e-16;
constexpr double kSqrt3Half = 0.8660254037844386;

constexpr int kNParam = 16;
enum { P_M = 0, P_MU, P_SPIN, P_E0, P_NU0, P_PHI0, P_GAM0, P_ALP0, P_THS, P_PHS, P_THK, P_PHK,
       P_LAM, P_Z, P_XI0, P_ALPT };

enum : uint32_t { ST_PLUNGE = 1u, ST_BADPARAM = 2u, ST_NONFINITE = 4u };

// Orbit knot: the AK state at t_k = t0 + k*K_s*dt and its time derivative.
// Angles in cycles as compensated (hi, lo) pairs; phd is the Doppler-shifted
// orbital phase Phi/2pi + nu * (R/c) sin(theta_S) cos(phibar - phi_S).
// amp = x^(2/3) = (2 pi M nu)^(2/3).  128 bytes.
struct __align__(16) Knot {
  double phd_hi, phd_lo, phd_rate;
  double gam_hi, gam_lo, gam_rate;
  double alp_hi, alp_lo, alp_rate;
  double amp, amp_rate;
  double e, e_rate;
  double pad0, pad1, pad2;
};
static_assert(sizeof(Knot) == 128, "knot size");

// Walker geometry of the channel response in the precision of a kernel.
// The response is evaluated in a fixed polarisation basis of the sky plane,
// P = phi^ and Q = theta^ at the source direction N.  With p = e1 cos(alpha)
// + e2 sin(alpha) and L = S cos(lam) + p sin(lam), the orbital-plane vectors
// u1 = p x S = sin(alpha) e1 - cos(alpha) e2 (the direction of L x S) and
// u2 = L x u1 = cos(lam) p - sin(lam) S enter only through their components
// along P and Q, which need the projections below.
template <typename T>
struct Geo {
  T pe1, pe2, qe1, qe2;       // P.e1, P.e2, Q.e1, Q.e2
  T cpe1, cpe2, cqe1, cqe2;   // cos(lam) P.e1, cos(lam) P.e2, cos(lam) Q.e1, cos(lam) Q.e2
  T spS, sqS;                 // sin(lam) P.S, sin(lam) Q.S
  T sin_ths, cos_ths, sin_phs, cos_phs;
  T amp_scale;
};

// Per-walker constants written by the prologue kernel and read by the rest.
struct __align__(16) WalkerC {
  // orbit
  double m_s, mu_s;          // G M/c^3, G mu/c^3 [s]
  double spin, coslam, sinlam;
  double kv, ke, inv2pim;    // dv/dt prefactor (32/5) mu/M^2, de/dt prefactor mu/M^2, 1/(2 pi M)
  double v0_hi, v0_lo;       // v = (2 pi M nu)^(1/3) at t0
  double e0, phi0c, gam0c, alp0c;   // initial e and angles [cycles]
  double amp_scale;          // mu_s c [cm]: strain at 1 cm per unit x^(2/3)
  // propagation
  double d_l, xi, d_gw;      // [cm]
  double dt_gw;              // [s]
  double r_hi, r_lo;         // frac(dt_gw / T)
  double cn_re, cn_im;       // exp(+2 pi i frac(N r))
  // geometry (ecliptic frame)
  double nx, ny, nz;         // source direction N
  double sx, sy, sz;         // spin direction S
  double e1x, e1y, e1z;      // e1 = (z - S cos thK)/sin thK
  double e2x, e2y, e2z;      // e2 = S x e1
  double sin_ths, cos_ths, sin_phs, cos_phs;
  double dop;                // (R/c) sin(theta_S) [s]
  double pad[3];
  Geo<double> gd;            // response geometry (FP64 kernels)
  Geo<float> gf;             // the same rounded to FP32 (mixed kernels)
  float cnf[2];              // (cn_re, cn_im) rounded to FP32
  int64_t j_plunge;          // first zeroed sample (n if none); written by the orbit kernel
  uint32_t status;           // status bits (prologue | orbit)
  uint32_t pad_u;
};

// Frequency-dependent propagation of one walker (Sec. 2, alpha_M(f),
// alpha_T(f) as power series in f/f_*): bin k (|k_s| = a) gets the amplitude
// exp(nlz_half * sum_m a_m (a xs)^m) and the extra phase (cycles, mod 1)
// sgn(k_s) * sum_m beta_m a^(m+1), beta_m as 128-bit fixed-point fractions.
struct FdW {
  double nlz_half;                  // -ln(1+z)/2
  double xs;                        // df / f_*
  double a[3];                      // alpha_M coefficients a_1..a_3
  unsigned long long bhi[3], blo[3];// beta_1..beta_3, value = (hi 2^64 + lo) / 2^128
  int qm, qt;
};


// Mixed-precision interval record of one knot interval: the three phases
// (Doppler orbital phase, 2 gamma~, alpha; cycles) as 64-bit fixed point
// base + inc * tau plus FP32 s^2, s^3 corrections (s = tau / K_s), and the
// amplitude x^(2/3) and eccentricity cubics in FP32.
struct IvM {
  unsigned long long ph_base, gm_base, al_base;
  long long ph_inc, gm_inc, al_inc;   // cycles per sample, Q0.64
  float ph_c[2], gm_c[2], al_c[2];
  float am[4];
  float ec[4];
};

// ------------------------------------------------------ double-double (dd)
// Unevaluated sums hi + lo with |lo| <= ulp(hi)/2, after Dekker (1971) and
// Knuth's TwoSum; the QD-library formulation of Hida, Li and Bailey (2001).
struct dd {
  double hi, lo;
};

__host__ __device__ __forceinline__ dd dd_make(double a) { return dd{a, 0.0}; }

__host__ __device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

__host__ __device__ __forceinline__ dd quick_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd{s, e};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd{p, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.hi, b);
  s.lo += a.lo;
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add_d(q, q3);
}

__device__ __forceinline__ dd dd_sqrt(dd a) {
  // one Newton step from the double square root: s + (a - s^2) / (2 s)
  if (a.hi <= 0.0) return dd{0.0, 0.0};
  double s = sqrt(a.hi);
  dd r = dd_sub(a, two_prod(s, s));
  return dd_add_d(dd{s, 0.0}, r.hi / (2.0 * s));
}

// exp of a dd argument: x = k ln2 + r, r reduced by 2^-9, Taylor series to
// order 14 in dd, then 9 squarings and the 2^k scale.
__device__ inline dd dd_exp(dd x) {
  const dd ln2{0.6931471805599453, 2.3190468138462996e-17};
  double k = rint(x.hi / ln2.hi);
  dd r = dd_sub(x, dd_mul_d(ln2, k));
  r = dd{ldexp(r.hi, -9), ldexp(r.lo, -9)};
  dd term = r, sum = r;
  for (int i = 2; i <= 14; ++i) {
    term = dd_div(dd_mul(term, r), dd_make((double)i));
    sum = dd_add(sum, term);
  }
  // exp(r) - 1 = sum; square 9 times: (1 + s)^2 - 1 = 2 s + s^2
  for (int i = 0; i < 9; ++i) sum = dd_add(dd_mul_d(sum, 2.0), dd_mul(sum, sum));
  dd e = dd_add_d(sum, 1.0);
  return dd{ldexp(e.hi, (int)k), ldexp(e.lo, (int)k)};
}

// log of a positive dd: y0 = log(hi), then one Newton step y0 + (a e^-y0 - 1)
// with the second-order term, accurate to dd precision.
__device__ inline dd dd_log(dd a) {
  double y0 = log(a.hi);
  dd t = dd_mul(a, dd_exp(dd{-y0, 0.0}));   // ~ 1 + eps
  dd u = dd_add_d(t, -1.0);
  dd corr = dd_sub(u, dd_mul_d(dd_mul(u, u), 0.5));
  return dd_add(dd{y0, 0.0}, corr);
}

// asinh(a) = log(a + sqrt(a^2 + 1)) for a >= 0
__device__ inline dd dd_asinh(dd a) {
  dd s = dd_sqrt(dd_add_d(dd_mul(a, a), 1.0));
  return dd_log(dd_add(a, s));
}

// fractional part in [0, 1) of a dd value
__device__ inline dd dd_frac(dd a) {
  double f = floor(a.hi);
  dd r = dd_add_d(dd{a.hi - f, 0.0}, a.lo);   // a.hi - f is exact
  if (r.hi < 0.0) r = dd_add_d(r, 1.0);
  if (r.hi >= 1.0) r = dd_add_d(r, -1.0);
  return r;
}

// Compensated accumulation of x into the unevaluated sum hi + lo.
// comp_add: exact TwoSum of hi and (x + lo), any magnitudes.
__device__ __forceinline__ void comp_add(double& hi, double& lo, double x) {
  dd s = two_sum(hi, x + lo);
  hi = s.hi;
  lo = s.lo;
}
// comp_add_small: Fast2Sum variant, valid when |x + lo| <= |hi|.
__device__ __forceinline__ void comp_add_small(double& hi, double& lo, double x) {
  double y = x + lo;
  double t = hi + y;
  lo = y - (t - hi);
  hi = t;
}

}  // namespace emri
