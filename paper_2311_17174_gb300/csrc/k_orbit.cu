// k_orbit.cu -- step S1: the AK orbit of Eq. (1), FP64.
//
// The paper integrates Y = {Phi, nu, e, gamma~, alpha} with a standard
// Runge-Kutta solver on the time grid (Sec. 3, "Waveform computation"; the
// right-hand side is the AK system of Barack & Cutler 2004 that the paper
// cites).  Here each walker is one thread that integrates the same system
// with classical RK4 at macro steps of K_s samples, in the variable
// v = x^(1/3) = (2 pi G M nu / c^3)^(1/3) instead of nu: then x^(2/3) = v^2,
// x^(11/3) = v^11 and (1-e^2)^(-k/2) = s^k with one s = 1/sqrt(1-e^2), so the
// right-hand side is polynomial apart from one reciprocal square root and the
// FP64 dependency chain is short (FP64 latency dominates this kernel).
// With v = x^(1/3):
//   dv/dt      = (32/5)(mu/M^2) v^9 s^9 B_nu(v, e)
//   de/dt      = -(e/15)(mu/M^2) s^7 v^8 B_e(v, e) + e (mu/M^2) a cos(lam) v^11 s^8 C_e(e)
//   dPhi/dt/2pi = nu = v^3 / (2 pi M)
//   dgamma~/dt/2pi = 3 nu v^2 s^2 [1 + v^2 s^2 (26 - 15 e^2)/4] - 6 nu cos(lam) a v^3 s^3
//   dalpha/dt/2pi  = 2 nu a v^3 s^3
// which is dnu/dt = 3 nu v^-1 dv/dt applied to the paper's equations.
// All five states are compensated (hi + lo) sums, so 1e4 steps add no
// rounding drift to the phase.  Each knot stores the state and its rates;
// the Doppler delay nu (R/c) sin(theta_S) cos(phibar - phi_S) is folded into
// the stored phase, and the sample at which nu reaches nu_LSO(e) (paper
// Sec. 3) is located by re-integrating the crossing interval at step dt.
#include "emri_common.cuh"
#include "emri_internal.h"

namespace emri {

struct OrbSrc {
  double kv, ke, inv2pim, spin, cl;
  int pn;
};

__device__ __forceinline__ void ak_rhs_v(const OrbSrc& s, double v, double e, double& dv, double& de,
                                         double& dph, double& dg, double& da) {
  const double e2 = e * e, e4 = e2 * e2, e6 = e4 * e2;
  const double om = 1.0 - e2;
  const double sq = rsqrt(om);
  const double s2 = sq * sq, s3 = s2 * sq, s4 = s2 * s2, s7 = s4 * s3, s8 = s4 * s4, s9 = s8 * sq;
  const double v2 = v * v, v3 = v2 * v, v4 = v2 * v2, v8 = v4 * v4, v9 = v8 * v, v11 = v9 * v2;
  const double a = s.spin, cl = s.cl;
  double br = (1.0 + (73.0 / 24.0) * e2 + (37.0 / 96.0) * e4) * om;
  double eb = (304.0 + 121.0 * e2) * om;
  if (s.pn) {
    br += v2 * (1273.0 / 336.0 - (2561.0 / 224.0) * e2 - (3885.0 / 128.0) * e4 - (13147.0 / 5376.0) * e6);
    br -= v3 * a * cl * sq * (73.0 / 12.0 + (1211.0 / 24.0) * e2 + (3143.0 / 96.0) * e4 + (65.0 / 64.0) * e6);
    eb = eb * (1.0 + 12.0 * v2) - (1.0 / 56.0) * v2 * (8.0 * 16705.0 + 12.0 * 9082.0 * e2 - 25211.0 * e4);
  }
  dv = s.kv * v9 * s9 * br;
  de = -(e / 15.0) * s.ke * s7 * v8 * eb;
  if (s.pn) de += e * s.ke * a * cl * v11 * s8 * (1364.0 / 5.0 + (5032.0 / 15.0) * e2 + (263.0 / 10.0) * e4);
  const double nu = v3 * s.inv2pim;
  dph = nu;
  double g1 = 3.0 * nu * v2 * s2;
  if (s.pn) g1 *= 1.0 + 0.25 * v2 * s2 * (26.0 - 15.0 * e2);
  dg = g1 - 6.0 * nu * cl * a * v3 * s3;
  da = 2.0 * nu * a * v3 * s3;
}

struct OrbState {
  double v_hi, v_lo, e_hi, e_lo, p_hi, p_lo, g_hi, g_lo, a_hi, a_lo;
};

__device__ __forceinline__ bool plunged(double v, double e) {
  // nu >= nu_LSO(e)  <=>  x^(2/3) = v^2 >= (1 - e^2)/(6 + 2 e)
  return v * v >= (1.0 - e * e) / (6.0 + 2.0 * e);
}

__device__ __forceinline__ bool state_finite(const OrbState& y) {
  return isfinite(y.v_hi) && isfinite(y.e_hi) && isfinite(y.p_hi) && isfinite(y.g_hi) && isfinite(y.a_hi);
}

// One RK4 step of size h; k1 holds the rates at the current state.
__device__ __forceinline__ void rk4_step(const OrbSrc& s, OrbState& y, double h, const double k1[5]) {
  double k2[5], k3[5], k4[5];
  const double hh = 0.5 * h;
  ak_rhs_v(s, y.v_hi + hh * k1[0], y.e_hi + hh * k1[1], k2[0], k2[1], k2[2], k2[3], k2[4]);
  ak_rhs_v(s, y.v_hi + hh * k2[0], y.e_hi + hh * k2[1], k3[0], k3[1], k3[2], k3[3], k3[4]);
  ak_rhs_v(s, y.v_hi + h * k3[0], y.e_hi + h * k3[1], k4[0], k4[1], k4[2], k4[3], k4[4]);
  const double h6 = h / 6.0;
  double d[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) d[q] = h6 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
  comp_add_small(y.v_hi, y.v_lo, d[0]);
  comp_add(y.e_hi, y.e_lo, d[1]);
  comp_add(y.p_hi, y.p_lo, d[2]);
  comp_add(y.g_hi, y.g_lo, d[3]);
  comp_add(y.a_hi, y.a_lo, d[4]);
}

__device__ __forceinline__ void write_knot(Knot* kn, const OrbState& y, const double r[5], const WalkerC& c,
                                           double tk, int doppler) {
  Knot k;
  const double v = y.v_hi, nu = v * v * v * c.inv2pim;
  const double nudot = 3.0 * v * v * r[0] * c.inv2pim;
  double dsh = 0.0, dshdot = 0.0;
  if (doppler) {
    double fb = tk / kYear;
    fb -= floor(fb);
    double sb, cb;
    sincospi(2.0 * fb, &sb, &cb);
    const double cdp = cb * c.cos_phs + sb * c.sin_phs;
    const double sdp = sb * c.cos_phs - cb * c.sin_phs;
    dsh = c.dop * cdp;                                 // (R/c) sin thS cos(phibar - phiS) [s]
    dshdot = -c.dop * sdp * (kTwoPiHi / kYear);
  }
  dd ph = two_sum(y.p_hi, nu * dsh);
  ph = quick_two_sum(ph.hi, ph.lo + y.p_lo);
  k.phd_hi = ph.hi;
  k.phd_lo = ph.lo;
  k.phd_rate = r[2] + nudot * dsh + nu * dshdot;
  k.gam_hi = y.g_hi; k.gam_lo = y.g_lo; k.gam_rate = r[3];
  k.alp_hi = y.a_hi; k.alp_lo = y.a_lo; k.alp_rate = r[4];
  k.amp = v * v;
  k.amp_rate = 2.0 * v * r[0];
  k.e = y.e_hi;
  k.e_rate = r[1];
  k.pad0 = k.pad1 = k.pad2 = 0.0;
  *kn = k;
}

__global__ void k1_orbit(WalkerC* __restrict__ wcs, int w, int64_t n, double dt, double t0, int ks, int pn,
                         int doppler, Knot* __restrict__ knots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w) return;
  const WalkerC c = wcs[i];
  const int64_t nk = n / ks;
  Knot* kn = knots + (int64_t)i * (nk + 1);
  if (c.status & ST_BADPARAM) {
    Knot zk = {};
    for (int64_t k = 0; k <= nk; ++k) kn[k] = zk;
    wcs[i].j_plunge = 0;
    return;
  }
  OrbSrc s{c.kv, c.ke, c.inv2pim, c.spin, c.coslam, pn};
  OrbState y{c.v0_hi, c.v0_lo, c.e0, 0.0, c.phi0c, 0.0, c.gam0c, 0.0, c.alp0c, 0.0};
  const double h = (double)ks * dt;
  int64_t jp = n;
  uint32_t st = 0;
  double r[5];
  ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
  write_knot(kn, y, r, c, t0, doppler);
  int64_t last = 0;   // last knot written
  if (plunged(y.v_hi, y.e_hi)) {
    jp = 0;
    st |= ST_PLUNGE;
  } else {
    for (int64_t k = 0; k < nk; ++k) {
      OrbState y0 = y;
      rk4_step(s, y, h, r);
      if (!state_finite(y) || plunged(y.v_hi, y.e_hi)) {
        // locate the first sample of (k ks, (k+1) ks] at or past the LSO by
        // re-integrating the interval at the sampling step
        OrbState f = y0;
        int64_t j = (k + 1) * ks;
        bool found = false;
        for (int q = 1; q <= ks; ++q) {
          double rr[5];
          ak_rhs_v(s, f.v_hi, f.e_hi, rr[0], rr[1], rr[2], rr[3], rr[4]);
          rk4_step(s, f, dt, rr);
          if (!state_finite(f) || plunged(f.v_hi, f.e_hi)) {
            j = k * ks + q;
            found = true;
            st |= state_finite(f) ? ST_PLUNGE : ST_NONFINITE;
            break;
          }
        }
        if (!found) st |= state_finite(y) ? ST_PLUNGE : ST_NONFINITE;
        jp = j < n ? j : n;
        if (jp == n) st &= ~(uint32_t)ST_PLUNGE;
        if (state_finite(y)) {
          ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
          write_knot(kn + k + 1, y, r, c, t0 + (double)((k + 1) * ks) * dt, doppler);
        } else {
          kn[k + 1] = kn[k];
        }
        last = k + 1;
        break;
      }
      ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
      write_knot(kn + k + 1, y, r, c, t0 + (double)((k + 1) * ks) * dt, doppler);
      last = k + 1;
    }
  }
  // knots past a plunge repeat the last one written (their samples are zeroed)
  for (int64_t q = last + 1; q <= nk; ++q) kn[q] = kn[last];
  wcs[i].j_plunge = jp;
  wcs[i].status = c.status | st;
}

void launch_orbit(WalkerC* wc, int w, int64_t n, double dt, double t0, const OptsN& o, Knot* knots,
                  cudaStream_t s) {
  if (w <= 0) return;
  k1_orbit<<<(w + 31) / 32, 32, 0, s>>>(wc, w, n, dt, t0, o.ks, o.pn_terms, o.doppler, knots);
}

}  // namespace emri
