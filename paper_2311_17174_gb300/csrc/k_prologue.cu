// k_prologue.cu -- step S0: per-walker constants.
//
// One thread per walker computes, from the structure-of-arrays parameters:
//  * the orbit constants G M/c^3, G mu/c^3 and the right-hand-side
//    prefactors, all formed in double-double and rounded once;
//  * the starting PN velocity v0 = (2 pi G M nu0 / c^3)^(1/3) to dd accuracy
//    (one Newton step on the cube), because a rounding of v0 is a systematic
//    frequency offset that the phase integrates over ~1e4-1e5 cycles;
//  * the LISA geometry vectors of the source and spin directions;
//  * the propagation factors of the paper's Sec. 2: d_L(z) (32-point
//    Gauss-Legendre quadrature of the flat Lambda-CDM comoving integral),
//    Xi(z) of Eq. (6), d_GW = Xi d_L, and the GW-speed delay of Eqs. (4)-(5)
//    for constant alpha_T, dt_GW = -(alpha_T/2) t_lookback(z), with the
//    lookback time in closed form evaluated in double-double.  The delay is
//    ~1e15 s; the per-bin phase needs frac(dt_GW / T) to ~1e-16 absolute, so
//    it is formed and reduced in dd.
#include "emri_common.cuh"
#include "emri_internal.h"

namespace emri {

__device__ __forceinline__ bool finite_all(const double* th, int64_t ld, int i) {
  for (int p = 0; p < kNParam; ++p)
    if (!isfinite(th[p * ld + i])) return false;
  return true;
}

// lookback time (flat Lambda-CDM, closed form) in dd:
//   t_LB = (1/H0) (2/(3 sqrt(OL))) [asinh(s) - asinh(s (1+z)^(-3/2))], s = sqrt(OL/Om)
__device__ dd lookback_dd(double zz, double omega_m, double h0) {
  dd om = dd_make(omega_m);
  dd ol = dd_add_d(dd_neg(om), 1.0);
  dd s = dd_sqrt(dd_div(ol, om));
  dd zp = two_sum(1.0, zz);
  dd u = dd_div(dd_make(1.0), dd_mul(zp, dd_sqrt(zp)));
  dd hinv_dd = dd_div(dd_make(kMpc), two_prod(h0, 1e5));
  dd diff = dd_sub(dd_asinh(s), dd_asinh(dd_mul(s, u)));
  return dd_mul(dd_div(dd_mul_d(hinv_dd, 2.0), dd_mul_d(dd_sqrt(ol), 3.0)), diff);
}

__global__ void k0_prologue(const double* __restrict__ theta, int64_t ld, int w, int64_t n, double dt,
                            int mode, double n_xi, double omega_m, double h0,
                            const double* __restrict__ gl, WalkerC* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w) return;
  WalkerC c;
  const double M = theta[P_M * ld + i], mu = theta[P_MU * ld + i], spin = theta[P_SPIN * ld + i];
  const double e0 = theta[P_E0 * ld + i], nu0 = theta[P_NU0 * ld + i];
  const double z = theta[P_Z * ld + i];
  uint32_t st = 0;
  const bool fin = finite_all(theta, ld, i);
  if (!fin || !(M > 0) || !(mu > 0) || !(spin >= 0 && spin <= 1) || !(e0 >= 0 && e0 < 1) ||
      !(z >= 0) || (mode == 0 && !(nu0 > 0)))
    st |= ST_BADPARAM;

  // G M_sun / c^3 in dd
  dd c3 = dd_mul_d(two_prod(kC, kC), kC);
  dd tsun = dd_div(dd_make(kGMsun), c3);
  dd ms = dd_mul_d(tsun, st ? 1.0 : M);
  dd mus = dd_mul_d(tsun, st ? 1.0 : mu);
  dd ms2 = dd_mul(ms, ms);
  c.m_s = ms.hi;
  c.mu_s = mus.hi;
  c.spin = st ? 0.0 : spin;
  double lam = theta[P_LAM * ld + i];
  sincos(lam, &c.sinlam, &c.coslam);
  c.kv = dd_div(dd_mul_d(mus, 32.0), dd_mul_d(ms2, 5.0)).hi;   // (32/5) mu/M^2
  c.ke = dd_div(mus, ms2).hi;                                  // mu/M^2
  dd twopi{kTwoPiHi, kTwoPiLo};
  dd twopim = dd_mul(twopi, ms);
  c.inv2pim = dd_div(dd_make(1.0), twopim).hi;

  // starting velocity v0 = x0^(1/3), x0 = 2 pi M nu0 (forward) or the LSO value
  dd x0;
  if (mode == 0) {
    x0 = dd_mul_d(twopim, st ? 1e-3 : nu0);
  } else {
    // nu_LSO: x_LSO = ((1 - e^2)/(6 + 2 e))^(3/2)
    dd p = dd_div(dd_add_d(dd_neg(two_prod(e0, e0)), 1.0), dd_add_d(dd_make(2.0 * e0), 6.0));
    x0 = dd_mul(p, dd_sqrt(p));
  }
  double v = cbrt(x0.hi);
  dd v3 = dd_mul_d(two_prod(v, v), v);
  dd resid = dd_sub(v3, x0);
  dd vd = dd_add_d(dd_make(v), -resid.hi / (3.0 * v * v));
  c.v0_hi = vd.hi;
  c.v0_lo = vd.lo;
  c.e0 = st ? 0.0 : e0;
  c.phi0c = theta[P_PHI0 * ld + i] / kTwoPiHi;
  c.gam0c = theta[P_GAM0 * ld + i] / kTwoPiHi;
  c.alp0c = theta[P_ALP0 * ld + i] / kTwoPiHi;
  c.amp_scale = mus.hi * kC;

  // geometry
  double ths = theta[P_THS * ld + i], phs = theta[P_PHS * ld + i];
  double thk = theta[P_THK * ld + i], phk = theta[P_PHK * ld + i];
  double sts, cts, sps, cps, stk, ctk, spk, cpk;
  sincos(ths, &sts, &cts);
  sincos(phs, &sps, &cps);
  sincos(thk, &stk, &ctk);
  sincos(phk, &spk, &cpk);
  c.nx = sts * cps; c.ny = sts * sps; c.nz = cts;
  c.sx = stk * cpk; c.sy = stk * spk; c.sz = ctk;
  if (fabs(stk) > 1e-12) {
    // e1 = (z - S cos thK)/sin thK, written out
    c.e1x = (0.0 - c.sx * ctk) / stk; c.e1y = (0.0 - c.sy * ctk) / stk; c.e1z = (1.0 - c.sz * ctk) / stk;
  } else {
    c.e1x = 1.0; c.e1y = 0.0; c.e1z = 0.0;
  }
  c.e2x = c.sy * c.e1z - c.sz * c.e1y;
  c.e2y = c.sz * c.e1x - c.sx * c.e1z;
  c.e2z = c.sx * c.e1y - c.sy * c.e1x;
  c.sin_ths = sts; c.cos_ths = cts; c.sin_phs = sps; c.cos_phs = cps;
  c.dop = kAUc * sts;

  // d_L(z) = (1+z)(c/H0) int_0^z dz'/E(z'), E = sqrt(Om (1+z)^3 + 1 - Om)
  const double zz = st ? 0.0 : z;
  double acc = 0.0;
  for (int q = 0; q < 32; ++q) {
    double zq = 0.5 * zz * (gl[q] + 1.0);
    double a = 1.0 + zq;
    acc += gl[32 + q] / sqrt(omega_m * a * a * a + (1.0 - omega_m));
  }
  const double hinv = kMpc / (h0 * 1e5);   // 1/H0 [s]
  c.d_l = (1.0 + zz) * kC * hinv * 0.5 * zz * acc;
  const double xi0 = theta[P_XI0 * ld + i];
  c.xi = xi0 + (1.0 - xi0) / pow(1.0 + zz, n_xi);
  c.d_gw = c.xi * c.d_l;
  if (!(c.d_gw > 0)) st |= ST_BADPARAM;

  // lookback time (flat Lambda-CDM, closed form) in dd:
  //   t_LB = (1/H0) (2/(3 sqrt(OL))) [asinh(s) - asinh(s (1+z)^(-3/2))], s = sqrt(OL/Om)
  const double alpt = st ? 0.0 : theta[P_ALPT * ld + i];
  if (alpt != 0.0 && zz > 0.0) {
    dd tlb = lookback_dd(zz, omega_m, h0);
    dd dtgw = dd_mul_d(tlb, -0.5 * alpt);
    dd tobs = two_prod((double)n, dt);
    dd r = dd_frac(dd_div(dtgw, tobs));
    c.dt_gw = dtgw.hi;
    c.r_hi = r.hi;
    c.r_lo = r.lo;
    // exp(+2 pi i frac(N r))
    dd nr = dd_add_d(two_prod((double)n, r.hi), (double)n * r.lo);
    dd f = dd_frac(nr);
    double sn, cn;
    sincospi(2.0 * f.hi, &sn, &cn);
    c.cn_re = cn;
    c.cn_im = sn;
  } else {
    c.dt_gw = 0.0; c.r_hi = 0.0; c.r_lo = 0.0; c.cn_re = 1.0; c.cn_im = 0.0;
  }
  c.pad[0] = c.pad[1] = c.pad[2] = 0.0;
  c.cnf[0] = (float)c.cn_re;
  c.cnf[1] = (float)c.cn_im;
  {
    // projections on the fixed sky basis P = (-sin phS, cos phS, 0),
    // Q = P x N = (cos phS cos thS, sin phS cos thS, -sin thS)
    const double P[3] = {-sps, cps, 0.0}, Q[3] = {cps * cts, sps * cts, -sts};
    const double e1[3] = {c.e1x, c.e1y, c.e1z}, e2[3] = {c.e2x, c.e2y, c.e2z}, S[3] = {c.sx, c.sy, c.sz};
    auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    Geo<double>& g = c.gd;
    g.pe1 = dot(P, e1); g.pe2 = dot(P, e2); g.qe1 = dot(Q, e1); g.qe2 = dot(Q, e2);
    g.cpe1 = c.coslam * g.pe1; g.cpe2 = c.coslam * g.pe2;
    g.cqe1 = c.coslam * g.qe1; g.cqe2 = c.coslam * g.qe2;
    g.spS = c.sinlam * dot(P, S); g.sqS = c.sinlam * dot(Q, S);
    g.sin_ths = sts; g.cos_ths = cts; g.sin_phs = sps; g.cos_phs = cps;
    g.amp_scale = c.amp_scale;
    Geo<float>& f = c.gf;
    f.pe1 = (float)g.pe1; f.pe2 = (float)g.pe2; f.qe1 = (float)g.qe1; f.qe2 = (float)g.qe2;
    f.cpe1 = (float)g.cpe1; f.cpe2 = (float)g.cpe2; f.cqe1 = (float)g.cqe1; f.cqe2 = (float)g.cqe2;
    f.spS = (float)g.spS; f.sqS = (float)g.sqS;
    f.sin_ths = (float)sts; f.cos_ths = (float)cts; f.sin_phs = (float)sps; f.cos_phs = (float)cps;
    f.amp_scale = (float)g.amp_scale;
  }
  c.j_plunge = n;
  c.status = st;
  c.pad_u = 0;
  out[i] = c;
}

// Per-walker delay tables for the factorisation
// exp(-2 pi i k r) = exp(-2 pi i k2 r) exp(-2 pi i n2 k1 r) of bin k = k2 + n2 k1:
// tab[k] = exp(-2 pi i frac(mult k r)), k < count (mult = n2 over k1 < n1, and
// mult = 1 over k2 < n2).  fold_neg: the entries with 2 k > count also carry
// exp(+2 pi i frac(N r)), the factor of the signed index k - N (negative
// frequencies).
// The FP32 tables take the fraction in fixed point: r as a 128-bit fraction,
// m r mod 1 from two 64-bit integer products (exact), its top 32 bits as the
// phase in [-1/2, 1/2) cycles, then the FP32 sincospif; no FP64 operation
// per entry.  The FP64 tables take it in double-double and FP64 sincospi.
__device__ void dd_to_fx128(dd x, unsigned long long& hi, unsigned long long& lo);

template <typename C2>
__global__ void k0_delay_table(const WalkerC* __restrict__ wc, int count, int mult, int fold_neg,
                               C2* __restrict__ tab) {
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int wk = blockIdx.y;
  if (k1 >= count) return;
  const double rh = wc[wk].r_hi, rl = wc[wk].r_lo;
  if constexpr (sizeof(C2) == 8) {
    unsigned long long Rh, Rl;
    dd_to_fx128(dd{rh, rl}, Rh, Rl);
    const unsigned long long m = (unsigned long long)mult * (unsigned long long)k1;   // < 2^22
    const unsigned long long ph = m * Rh + __umul64hi(m, Rl);                          // m r mod 1, Q0.64
    const float f = (float)(int)(unsigned)(ph >> 32) * 2.3283064365386963e-10f;        // [-1/2, 1/2)
    float sf, cf;
    sincospif(2.f * f, &sf, &cf);
    float vx = cf, vy = -sf;
    if (fold_neg && 2 * k1 > count) {
      const float cr = wc[wk].cnf[0], ci = wc[wk].cnf[1];
      const float x = vx * cr - vy * ci;
      vy = vx * ci + vy * cr;
      vx = x;
    }
    tab[(int64_t)wk * count + k1] = make_float2(vx, vy);
    return;
  }
  double m = (double)mult * (double)k1;
  dd p = dd_add_d(two_prod(m, rh), m * rl);
  dd f = dd_frac(p);
  double s, c;
  sincospi(2.0 * f.hi, &s, &c);
  double vx = c, vy = -s;
  if (fold_neg && 2 * k1 > count) {
    const double cr = wc[wk].cn_re, ci = wc[wk].cn_im;
    const double x = vx * cr - vy * ci;
    vy = vx * ci + vy * cr;
    vx = x;
  }
  C2 v;
  v.x = (decltype(v.x))vx;
  v.y = (decltype(v.y))vy;
  tab[(int64_t)wk * count + k1] = v;
}

__global__ void k0_export(const WalkerC* __restrict__ wc, int w, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w) return;
  const WalkerC& c = wc[i];
  out[0 * (int64_t)w + i] = c.d_l;
  out[1 * (int64_t)w + i] = c.xi;
  out[2 * (int64_t)w + i] = c.d_gw;
  out[3 * (int64_t)w + i] = c.dt_gw;
  out[4 * (int64_t)w + i] = c.r_hi;
  out[5 * (int64_t)w + i] = c.r_lo;
}

void launch_prologue(const double* theta, int64_t ld, int w, int64_t n, double dt, const OptsN& o,
                     const double* gl, WalkerC* out, cudaStream_t s) {
  if (w <= 0) return;
  k0_prologue<<<(w + 63) / 64, 64, 0, s>>>(theta, ld, w, n, dt, o.mode, o.n_xi, o.omega_m, o.h0, gl, out);
}

void launch_delay_table(const WalkerC* wc, int w, int n1, int n2, bool fp32, void* tab, void* rtab, cudaStream_t s) {
  // walkers on grid y, at most kMaxGridY per launch
  for (int w0 = 0; w0 < w; w0 += kMaxGridY) {
    const int ww = w - w0 < kMaxGridY ? w - w0 : kMaxGridY;
    dim3 g1((n1 + 255) / 256, ww), g2((n2 + 255) / 256, ww);
    if (fp32) {
      k0_delay_table<float2><<<g1, 256, 0, s>>>(wc + w0, n1, n2, 1, (float2*)tab + (int64_t)w0 * n1);
      k0_delay_table<float2><<<g2, 256, 0, s>>>(wc + w0, n2, 1, 0, (float2*)rtab + (int64_t)w0 * n2);
    } else {
      k0_delay_table<double2><<<g1, 256, 0, s>>>(wc + w0, n1, n2, 1, (double2*)tab + (int64_t)w0 * n1);
      k0_delay_table<double2><<<g2, 256, 0, s>>>(wc + w0, n2, 1, 0, (double2*)rtab + (int64_t)w0 * n2);
    }
  }
}

void launch_prologue_export(const WalkerC* wc, int w, double* out, cudaStream_t s) {
  if (w <= 0) return;
  k0_export<<<(w + 127) / 128, 128, 0, s>>>(wc, w, out);
}

// ----------------------------------------- frequency-dependent propagation
// dd fraction x in [0, 1) -> 128-bit fixed point (hi, lo) = x 2^128, mod 2^128.
// x.hi 2^64 is exact but carries only 53 bits; the low bits of the 64-bit
// integer part come from x.lo 2^64, which can reach ~2^11 in magnitude, so
// its integer part is carried into hi and only its fraction goes to lo.
__device__ void dd_to_fx128(dd x, unsigned long long& hi, unsigned long long& lo) {
  const double two64 = 18446744073709551616.0;
  const double t = x.hi * two64;            // exact scaling, 0 <= t < 2^64
  const double H = floor(t);                // exact
  const double r = (t - H) + x.lo * two64;  // t - H and x.lo 2^64 exact; |r| < ~2^12
  const double F = floor(r);                // exact integer
  const double rem = r - F;                 // exact, [0, 1)
  hi = (unsigned long long)H + (unsigned long long)(long long)F;   // mod 2^64
  lo = (unsigned long long)(rem * two64);
}

// beta_m = -(t_LB/2) b_m df^(m+1) / f_*^m (cycles per |k|^(m+1)), reduced mod 1
// in dd before the conversion to fixed point.
__global__ void k0_fdprop(const double* __restrict__ theta, int64_t ld, int w, int64_t n, double dt, double omega_m,
                          double h0, int qm, int qt, double fstar, const double* __restrict__ coef, int64_t ldc,
                          FdW* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w) return;
  FdW f{};
  f.qm = qm;
  f.qt = qt;
  double z = theta[P_Z * ld + i];
  if (!(z >= 0.0) || !isfinite(z)) z = 0.0;   // such a walker is flagged by the prologue
  f.nlz_half = -0.5 * log1p(z);
  const dd tobs = two_prod((double)n, dt);
  const dd df = dd_div(dd_make(1.0), tobs);
  f.xs = dd_div(df, dd_make(fstar)).hi;
  for (int m = 0; m < qm; ++m) f.a[m] = coef[(int64_t)m * ldc + i];
  if (qt > 0) {
    const dd tlb = z > 0.0 ? lookback_dd(z, omega_m, h0) : dd_make(0.0);
    const dd q = dd_div(df, dd_make(fstar));
    dd base = dd_mul(dd_mul_d(tlb, -0.5), df);   // -(t_LB/2) df
    for (int m = 0; m < qt; ++m) {
      base = dd_mul(base, q);                     // -(t_LB/2) df (df/f_*)^(m+1)
      const dd beta = dd_frac(dd_mul_d(base, coef[(int64_t)(qm + m) * ldc + i]));
      dd_to_fx128(beta, f.bhi[m], f.blo[m]);
    }
  }
  out[i] = f;
}

void launch_fdprop(const double* theta, int64_t ld, int w, int64_t n, double dt, const OptsN& o, int qm, int qt,
                   double fstar, const double* coef, int64_t ldc, FdW* fd, cudaStream_t s) {
  if (w <= 0) return;
  k0_fdprop<<<(w + 127) / 128, 128, 0, s>>>(theta, ld, w, n, dt, o.omega_m, o.h0, qm, qt, fstar, coef, ldc, fd);
}

}  // namespace emri
