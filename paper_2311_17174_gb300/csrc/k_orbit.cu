// k_orbit.cu -- step S1: the AK orbit of Eq. (1), FP64.
//
// The paper integrates Y = {Phi, nu, e, gamma~, alpha} with a standard
// solver on the time grid (Sec. 3, "Waveform computation"; the right-hand
// side is the AK system of Barack & Cutler 2004 that the paper cites).
// A step-by-step integrator is a serial FP64 dependency chain per walker, and
// on this GPU one FP64 warp instruction occupies its SM sub-partition for ~64
// cycles; so the orbit is integrated in parallel in time instead: one warp
// per walker, segments of up to 65536 samples (at most 128 knot intervals:
// 16384 samples at K_s = 128), the solution on each segment represented by
// its values at the 32 Chebyshev-Gauss-Lobatto nodes (one per lane) and found
// by Picard iteration y(t) = y(t_a) + int f(y) with the spectral integration
// matrix (Chebyshev-Picard iteration; a segment is ~1e-2..1e-1 of the
// radiation-reaction time, and each segment's sweeps start from the previous
// segment's node increments).  The knots every K_s samples are read off the
// segment's polynomial (integral weights at the knot positions).  The same system is written in the
// variable
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

// Serial compensated RK4 at the knot step from knot k0 (state y, already
// written) over knots k0+1..k1.  Returns true if the orbit stayed inside the
// LSO; otherwise locates the plunge sample jp by re-integrating the crossing
// interval at the sampling step, writes the first knot past the crossing
// (the right end of the interval holding the last valid samples) and sets
// last to it.
__device__ bool rk4_span(const OrbSrc& s, const WalkerC& c, OrbState& y, int64_t k0, int64_t k1, int ks, double dt,
                         double t0, int doppler, int64_t n, Knot* kn, int64_t& jp, uint32_t& st, int64_t& last) {
  const double h = (double)ks * dt;
  double r[5];
  ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
  for (int64_t k = k0; k < k1; ++k) {
    OrbState y0 = y;
    rk4_step(s, y, h, r);
    if (!state_finite(y) || plunged(y.v_hi, y.e_hi)) {
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
      return false;
    }
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    write_knot(kn + k + 1, y, r, c, t0 + (double)((k + 1) * ks) * dt, doppler);
    last = k + 1;
  }
  return true;
}

// ------------------------------------------------------ Chebyshev-Picard
// qn[j*32 + i] = int_0^{tau_i} l_j(tau) dtau (transposed, nodes tau_i =
// (1 - cos(pi i/31))/2 on the unit segment); qk[q*32 + j] = int_0^{q/128} l_j,
// q = 0..128 (knot positions of the finest knot grid).  Built on the host.
constexpr int kSeg = 65536;        // samples per segment (n if smaller; at most 128 knots)

// samples per Chebyshev-Picard segment: kSeg, but no more than n and than 128
// knot intervals (the knot-weight table has 129 rows)
__host__ __device__ __forceinline__ int64_t mcpi_segment(int64_t n, int ks) {
  int64_t seg = n < kSeg ? n : kSeg;
  if (seg > 128 * (int64_t)ks) seg = 128 * (int64_t)ks;
  return seg;
}
constexpr int kOrbitWarps = 1;     // walkers per CTA (one warp each: balances FP64 work over the SMs)

__device__ __forceinline__ void ak_rate_ve(const OrbSrc& s, double v, double e, double& dv, double& de) {
  double d0, d1, d2;
  ak_rhs_v(s, v, e, dv, de, d0, d1, d2);
}

// Start values of (v, e) at this lane's node for the Picard sweeps.  The first
// segment (or one after a serial fallback) starts from the Euler step; later
// ones repeat the previous segment's converged increment at the same node,
// scaled by the ratio of the start rates -- the rates change by ~H/tau_rr
// (~1e-3) per segment, so the start error drops from ~(H/tau)^2 to ~(H/tau)^3
// of the increment and the iteration needs about two sweeps fewer.  The
// fixed point reached is the same.
__device__ __forceinline__ void warm_start(bool warm, const OrbState& y, double H, double taui, double f0v,
                                           double f0e, double dv_prev, double de_prev, double f0v_prev,
                                           double f0e_prev, double& v, double& e) {
  const bool wv = warm && f0v_prev != 0.0;
  const bool we = warm && f0e_prev != 0.0;
  v = y.v_hi + (y.v_lo + (wv ? dv_prev * (f0v / f0v_prev) : H * taui * f0v));
  e = y.e_hi + (y.e_lo + (we ? de_prev * (f0e / f0e_prev) : H * taui * f0e));
}

__global__ void __launch_bounds__(32 * kOrbitWarps) k1_orbit_mcpi(WalkerC* __restrict__ wcs, int w, int64_t n, double dt,
                                                                   double t0, int ks, int pn, int doppler,
                                                                   const double* __restrict__ qn_g,
                                                                   const double* __restrict__ qk_g,
                                                                   Knot* __restrict__ knots) {
  extern __shared__ double osm[];          // qn[32*32], qk[(K+1)*32], fs[warps][5][32]
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int seg = (int)mcpi_segment(n, ks);
  const int K = seg / ks;                   // knots per segment
  const int qstride = 128 / K;
  double* qn = osm;
  double* qk = osm + 32 * 32;
  double* fs = qk + (K + 1) * 32;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) qn[i] = qn_g[i];
  for (int q = 0; q <= K; ++q)
    for (int i = threadIdx.x; i < 32; i += blockDim.x) qk[q * 32 + i] = qk_g[(q * qstride) * 32 + i];
  __syncthreads();
  const int wk = blockIdx.x * kOrbitWarps + wq;
  if (wk >= w) return;
  const WalkerC c = wcs[wk];
  const int64_t nk = n / ks;
  Knot* kn = knots + (int64_t)wk * (nk + 1);
  if (c.status & ST_BADPARAM) {
    Knot zk = {};
    for (int64_t k = lane; k <= nk; k += 32) kn[k] = zk;
    if (lane == 0) wcs[wk].j_plunge = 0;
    return;
  }
  const OrbSrc s{c.kv, c.ke, c.inv2pim, c.spin, c.coslam, pn};
  // segment-start state (identical in every lane), compensated
  OrbState y{c.v0_hi, c.v0_lo, c.e0, 0.0, c.phi0c, 0.0, c.gam0c, 0.0, c.alp0c, 0.0};
  const double H = (double)seg * dt;
  const double taui = 0.5 * (1.0 - cospi((double)lane / 31.0));
  double* f = fs + wq * 5 * 32;
  int64_t jp = n;
  uint32_t st = 0;
  int64_t last = -1;   // last knot written
  if (plunged(y.v_hi, y.e_hi)) {
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    if (lane == 0) write_knot(kn, y, r, c, t0, doppler);
    jp = 0;
    st |= ST_PLUNGE;
    last = 0;
  } else {
    // knot 0 from the start state; each segment then writes its knots 1..K
    // (knot K, its end state, is the next segment's first)
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    if (lane == 0) write_knot(kn, y, r, c, t0, doppler);
  }
  const int64_t nseg = n / seg;
  bool warm = false;
  double dv_prev = 0.0, de_prev = 0.0, f0v_prev = 0.0, f0e_prev = 0.0;
  for (int64_t g = 0; g < nseg && jp == n; ++g) {
    const OrbState ys = y;   // segment start
    const int64_t kbase = g * (int64_t)K;
    // start values at the nodes, then Picard sweeps on (v, e)
    double f0v, f0e;
    ak_rate_ve(s, y.v_hi, y.e_hi, f0v, f0e);
    double v, e;
    warm_start(warm, y, H, taui, f0v, f0e, dv_prev, de_prev, f0v_prev, f0e_prev, v, e);
    bool convw = false;
    for (int it = 0; it < 30; ++it) {
      double fv, fe;
      ak_rate_ve(s, v, e, fv, fe);
      __syncwarp();
      f[0 * 32 + lane] = fv;
      f[1 * 32 + lane] = fe;
      __syncwarp();
      double sv = 0.0, se = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const double q = qn[j * 32 + lane];
        sv = fma(q, f[0 * 32 + j], sv);
        se = fma(q, f[1 * 32 + j], se);
      }
      const double vn = y.v_hi + (y.v_lo + H * sv);
      const double en = y.e_hi + (y.e_lo + H * se);
      // settled to within about two ulps (iterates can cycle at rounding level)
      const bool conv = fabs(vn - v) <= 4e-16 * fabs(y.v_hi) && fabs(en - e) <= 2e-16;
      v = vn;
      e = en;
      const bool ok = isfinite(v) && isfinite(e);
      if (__all_sync(0xffffffffu, conv || !ok)) {
        convw = __all_sync(0xffffffffu, conv && ok);
        break;
      }
    }
    // a segment that reaches the LSO, or on which the iteration does not
    // settle, is integrated serially instead (fallback below)
    bool serial = !convw;
    // this segment's node increments seed the next segment's start values
    warm = convw;
    dv_prev = v - (ys.v_hi + ys.v_lo);
    de_prev = e - (ys.e_hi + ys.e_lo);
    f0v_prev = f0v;
    f0e_prev = f0e;
    if (!serial) {
      // all five rates at the nodes
      double r[5];
      ak_rhs_v(s, v, e, r[0], r[1], r[2], r[3], r[4]);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 5; ++q) f[q * 32 + lane] = r[q];
      __syncwarp();
      // knots q = 1..K of this segment (the start, q = 0, is already
      // written); the end state (q = K) is every lane's next start
      bool anybad = false;
      for (int q0 = 1; q0 <= K; q0 += 32) {
        const int q = q0 + lane;
        bool bad = false;
        OrbState yk = y;
        if (q <= K) {
          double sm[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
          for (int j = 0; j < 32; ++j) {
            const double wq_ = qk[q * 32 + j];
#pragma unroll
            for (int cc = 0; cc < 5; ++cc) sm[cc] = fma(wq_, f[cc * 32 + j], sm[cc]);
          }
          comp_add_small(yk.v_hi, yk.v_lo, H * sm[0]);
          comp_add(yk.e_hi, yk.e_lo, H * sm[1]);
          comp_add(yk.p_hi, yk.p_lo, H * sm[2]);
          comp_add(yk.g_hi, yk.g_lo, H * sm[3]);
          comp_add(yk.a_hi, yk.a_lo, H * sm[4]);
          bad = !state_finite(yk) || plunged(yk.v_hi, yk.e_hi);
          if (!bad) {
            double rk[5];
            ak_rhs_v(s, yk.v_hi, yk.e_hi, rk[0], rk[1], rk[2], rk[3], rk[4]);
            write_knot(kn + kbase + q, yk, rk, c, t0 + (double)((kbase + q) * ks) * dt, doppler);
          }
        }
        anybad |= __any_sync(0xffffffffu, bad);
        const int src = K - q0;
        if (src >= 0 && src < 32) {
          y.v_hi = __shfl_sync(0xffffffffu, yk.v_hi, src); y.v_lo = __shfl_sync(0xffffffffu, yk.v_lo, src);
          y.e_hi = __shfl_sync(0xffffffffu, yk.e_hi, src); y.e_lo = __shfl_sync(0xffffffffu, yk.e_lo, src);
          y.p_hi = __shfl_sync(0xffffffffu, yk.p_hi, src); y.p_lo = __shfl_sync(0xffffffffu, yk.p_lo, src);
          y.g_hi = __shfl_sync(0xffffffffu, yk.g_hi, src); y.g_lo = __shfl_sync(0xffffffffu, yk.g_lo, src);
          y.a_hi = __shfl_sync(0xffffffffu, yk.a_hi, src); y.a_lo = __shfl_sync(0xffffffffu, yk.a_lo, src);
        }
      }
      serial = anybad;
    }
    if (serial) {
      // lane 0 redoes the segment with knot-step RK4 (rk4_span) from
      // the segment start; its knots replace any written above
      warm = false;
      __syncwarp();
      int valid = 1;
      if (lane == 0) {
        OrbState yy = ys;
        double r0[5];
        ak_rhs_v(s, yy.v_hi, yy.e_hi, r0[0], r0[1], r0[2], r0[3], r0[4]);
        write_knot(kn + kbase, yy, r0, c, t0 + (double)(kbase * ks) * dt, doppler);
        valid = rk4_span(s, c, yy, kbase, kbase + K, ks, dt, t0, doppler, n, kn, jp, st, last) ? 1 : 0;
        y = yy;
      }
      valid = __shfl_sync(0xffffffffu, valid, 0);
      jp = __shfl_sync(0xffffffffu, jp, 0);
      st = __shfl_sync(0xffffffffu, st, 0);
      last = __shfl_sync(0xffffffffu, last, 0);
      y.v_hi = __shfl_sync(0xffffffffu, y.v_hi, 0); y.v_lo = __shfl_sync(0xffffffffu, y.v_lo, 0);
      y.e_hi = __shfl_sync(0xffffffffu, y.e_hi, 0); y.e_lo = __shfl_sync(0xffffffffu, y.e_lo, 0);
      y.p_hi = __shfl_sync(0xffffffffu, y.p_hi, 0); y.p_lo = __shfl_sync(0xffffffffu, y.p_lo, 0);
      y.g_hi = __shfl_sync(0xffffffffu, y.g_hi, 0); y.g_lo = __shfl_sync(0xffffffffu, y.g_lo, 0);
      y.a_hi = __shfl_sync(0xffffffffu, y.a_hi, 0); y.a_lo = __shfl_sync(0xffffffffu, y.a_lo, 0);
      if (!valid) break;
    }
    last = kbase + K - 1;
  }
  if (jp == n && last == nk - 1) {
    // the end knot (sample n) from the final state
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    if (lane == 0) write_knot(kn + nk, y, r, c, t0 + (double)(nk * ks) * dt, doppler);
    last = nk;
  }
  __syncwarp();
  // knots past a plunge repeat the last one written (their samples are zeroed)
  for (int64_t q = last + 1 + lane; q <= nk; q += 32) kn[q] = kn[last];
  if (lane == 0) {
    wcs[wk].j_plunge = jp;
    wcs[wk].status = c.status | st;
  }
}

// Backward mode (paper Sec. 3: initial conditions at the LSO, integrated back
// in time): the LSO state (v_LSO(e0), e0, Phi0, gamma~0, alpha0) sits at the
// last sample t0 + (n-1) dt.  One RK4 step of +dt carries it to the last knot
// (sample n), from where the segments are integrated with negative step,
// knots written from the end; the AK system is regular at the LSO, so the
// short step past it is harmless.  A segment whose iteration does not settle
// is redone serially (knot-step RK4 backwards).  No plunge check applies; an
// orbit that becomes non-finite gives a zero waveform and ST_NONFINITE.
__device__ bool rk4_span_back(const OrbSrc& s, const WalkerC& c, OrbState& y, int64_t k0, int64_t k1, int ks,
                              double dt, double t0, int doppler, Knot* kn) {
  const double h = -(double)ks * dt;
  double r[5];
  ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
  for (int64_t k = k0; k > k1; --k) {
    rk4_step(s, y, h, r);
    if (!state_finite(y)) return false;
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    write_knot(kn + k - 1, y, r, c, t0 + (double)((k - 1) * ks) * dt, doppler);
  }
  return true;
}

__global__ void __launch_bounds__(32 * kOrbitWarps) k1_orbit_mcpi_back(WalkerC* __restrict__ wcs, int w, int64_t n,
                                                                        double dt, double t0, int ks, int pn,
                                                                        int doppler, const double* __restrict__ qn_g,
                                                                        const double* __restrict__ qk_g,
                                                                        Knot* __restrict__ knots) {
  extern __shared__ double osm[];          // qn[32*32], qk[(K+1)*32], fs[warps][5][32]
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int seg = (int)mcpi_segment(n, ks);
  const int K = seg / ks;                   // knots per segment
  const int qstride = 128 / K;
  double* qn = osm;
  double* qk = osm + 32 * 32;
  double* fs = qk + (K + 1) * 32;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) qn[i] = qn_g[i];
  for (int q = 0; q <= K; ++q)
    for (int i = threadIdx.x; i < 32; i += blockDim.x) qk[q * 32 + i] = qk_g[(q * qstride) * 32 + i];
  __syncthreads();
  const int wk = blockIdx.x * kOrbitWarps + wq;
  if (wk >= w) return;
  const WalkerC c = wcs[wk];
  const int64_t nk = n / ks;
  Knot* kn = knots + (int64_t)wk * (nk + 1);
  if (c.status & ST_BADPARAM) {
    Knot zk = {};
    for (int64_t k = lane; k <= nk; k += 32) kn[k] = zk;
    if (lane == 0) wcs[wk].j_plunge = 0;
    return;
  }
  const OrbSrc s{c.kv, c.ke, c.inv2pim, c.spin, c.coslam, pn};
  OrbState y{c.v0_hi, c.v0_lo, c.e0, 0.0, c.phi0c, 0.0, c.gam0c, 0.0, c.alp0c, 0.0};
  {
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    rk4_step(s, y, dt, r);
  }
  const double H = -(double)seg * dt;
  const double taui = 0.5 * (1.0 - cospi((double)lane / 31.0));
  double* f = fs + wq * 5 * 32;
  bool fail = !state_finite(y);
  if (!fail) {
    // knot nk from the start state; each segment then writes its knots
    // kend - 1 .. kend - K (the last is the next segment's start)
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    if (lane == 0) write_knot(kn + nk, y, r, c, t0 + (double)(nk * ks) * dt, doppler);
  }
  const int64_t nseg = n / seg;
  bool warm = false;
  double dv_prev = 0.0, de_prev = 0.0, f0v_prev = 0.0, f0e_prev = 0.0;
  for (int64_t g = nseg - 1; g >= 0 && !fail; --g) {
    const OrbState ys = y;
    const int64_t kend = (g + 1) * (int64_t)K;   // knot at the segment's start (its latest time)
    double f0v, f0e;
    ak_rate_ve(s, y.v_hi, y.e_hi, f0v, f0e);
    double v, e;
    warm_start(warm, y, H, taui, f0v, f0e, dv_prev, de_prev, f0v_prev, f0e_prev, v, e);
    bool convw = false;
    for (int it = 0; it < 30; ++it) {
      double fv, fe;
      ak_rate_ve(s, v, e, fv, fe);
      __syncwarp();
      f[0 * 32 + lane] = fv;
      f[1 * 32 + lane] = fe;
      __syncwarp();
      double sv = 0.0, se = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const double q = qn[j * 32 + lane];
        sv = fma(q, f[0 * 32 + j], sv);
        se = fma(q, f[1 * 32 + j], se);
      }
      const double vn = y.v_hi + (y.v_lo + H * sv);
      const double en = y.e_hi + (y.e_lo + H * se);
      const bool conv = fabs(vn - v) <= 4e-16 * fabs(y.v_hi) && fabs(en - e) <= 2e-16;
      v = vn;
      e = en;
      const bool ok = isfinite(v) && isfinite(e);
      if (__all_sync(0xffffffffu, conv || !ok)) {
        convw = __all_sync(0xffffffffu, conv && ok);
        break;
      }
    }
    bool serial = !convw;
    // this segment's node increments seed the next segment's start values
    warm = convw;
    dv_prev = v - (ys.v_hi + ys.v_lo);
    de_prev = e - (ys.e_hi + ys.e_lo);
    f0v_prev = f0v;
    f0e_prev = f0e;
    if (!serial) {
      double r[5];
      ak_rhs_v(s, v, e, r[0], r[1], r[2], r[3], r[4]);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 5; ++q) f[q * 32 + lane] = r[q];
      __syncwarp();
      bool anybad = false;
      for (int q0 = 1; q0 <= K; q0 += 32) {
        const int q = q0 + lane;
        bool bad = false;
        OrbState yk = y;
        if (q <= K) {
          double sm[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
          for (int j = 0; j < 32; ++j) {
            const double wq_ = qk[q * 32 + j];
#pragma unroll
            for (int cc = 0; cc < 5; ++cc) sm[cc] = fma(wq_, f[cc * 32 + j], sm[cc]);
          }
          comp_add_small(yk.v_hi, yk.v_lo, H * sm[0]);
          comp_add(yk.e_hi, yk.e_lo, H * sm[1]);
          comp_add(yk.p_hi, yk.p_lo, H * sm[2]);
          comp_add(yk.g_hi, yk.g_lo, H * sm[3]);
          comp_add(yk.a_hi, yk.a_lo, H * sm[4]);
          bad = !state_finite(yk);
          if (!bad) {
            double rk[5];
            ak_rhs_v(s, yk.v_hi, yk.e_hi, rk[0], rk[1], rk[2], rk[3], rk[4]);
            write_knot(kn + kend - q, yk, rk, c, t0 + (double)((kend - q) * ks) * dt, doppler);
          }
        }
        anybad |= __any_sync(0xffffffffu, bad);
        const int src = K - q0;
        if (src >= 0 && src < 32) {
          y.v_hi = __shfl_sync(0xffffffffu, yk.v_hi, src); y.v_lo = __shfl_sync(0xffffffffu, yk.v_lo, src);
          y.e_hi = __shfl_sync(0xffffffffu, yk.e_hi, src); y.e_lo = __shfl_sync(0xffffffffu, yk.e_lo, src);
          y.p_hi = __shfl_sync(0xffffffffu, yk.p_hi, src); y.p_lo = __shfl_sync(0xffffffffu, yk.p_lo, src);
          y.g_hi = __shfl_sync(0xffffffffu, yk.g_hi, src); y.g_lo = __shfl_sync(0xffffffffu, yk.g_lo, src);
          y.a_hi = __shfl_sync(0xffffffffu, yk.a_hi, src); y.a_lo = __shfl_sync(0xffffffffu, yk.a_lo, src);
        }
      }
      serial = anybad;
    }
    if (serial) {
      warm = false;
      __syncwarp();
      int valid = 1;
      if (lane == 0) {
        OrbState yy = ys;
        double r0[5];
        ak_rhs_v(s, yy.v_hi, yy.e_hi, r0[0], r0[1], r0[2], r0[3], r0[4]);
        write_knot(kn + kend, yy, r0, c, t0 + (double)(kend * ks) * dt, doppler);
        valid = rk4_span_back(s, c, yy, kend, kend - K, ks, dt, t0, doppler, kn) ? 1 : 0;
        y = yy;
      }
      valid = __shfl_sync(0xffffffffu, valid, 0);
      y.v_hi = __shfl_sync(0xffffffffu, y.v_hi, 0); y.v_lo = __shfl_sync(0xffffffffu, y.v_lo, 0);
      y.e_hi = __shfl_sync(0xffffffffu, y.e_hi, 0); y.e_lo = __shfl_sync(0xffffffffu, y.e_lo, 0);
      y.p_hi = __shfl_sync(0xffffffffu, y.p_hi, 0); y.p_lo = __shfl_sync(0xffffffffu, y.p_lo, 0);
      y.g_hi = __shfl_sync(0xffffffffu, y.g_hi, 0); y.g_lo = __shfl_sync(0xffffffffu, y.g_lo, 0);
      y.a_hi = __shfl_sync(0xffffffffu, y.a_hi, 0); y.a_lo = __shfl_sync(0xffffffffu, y.a_lo, 0);
      fail = !valid;
    }
  }
  if (!fail && lane == 0) {
    double r[5];
    ak_rhs_v(s, y.v_hi, y.e_hi, r[0], r[1], r[2], r[3], r[4]);
    write_knot(kn, y, r, c, t0, doppler);   // knot 0 (sample 0)
  }
  if (lane == 0) {
    wcs[wk].j_plunge = fail ? 0 : n;
    wcs[wk].status = c.status | (fail ? (uint32_t)ST_NONFINITE : 0u);
  }
}

void launch_orbit(WalkerC* wc, int w, int64_t n, double dt, double t0, const OptsN& o, Knot* knots,
                  const double* mcpi_tab, cudaStream_t s) {
  if (w <= 0) return;
  const int64_t seg = mcpi_segment(n, o.ks);
  const int K = (int)(seg / o.ks);
  const size_t smem = sizeof(double) * (32 * 32 + (size_t)(K + 1) * 32 + kOrbitWarps * 5 * 32);
  if (o.mode == 1) {   // backward from the LSO (the integration tables are always present)
    k1_orbit_mcpi_back<<<(w + kOrbitWarps - 1) / kOrbitWarps, 32 * kOrbitWarps, smem, s>>>(
        wc, w, n, dt, t0, o.ks, o.pn_terms, o.doppler, mcpi_tab, mcpi_tab + 32 * 32, knots);
  } else {
    k1_orbit_mcpi<<<(w + kOrbitWarps - 1) / kOrbitWarps, 32 * kOrbitWarps, smem, s>>>(
        wc, w, n, dt, t0, o.ks, o.pn_terms, o.doppler, mcpi_tab, mcpi_tab + 32 * 32, knots);
  }
}

}  // namespace emri
