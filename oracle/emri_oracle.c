/*
 * emri_oracle.c -- plain, slow CPU oracle for the batched Analytic-Kludge (AK)
 * log-likelihood of Saltas & Oliveri, "emri_mc: A GPU-based Python code for
 * Bayesian inference of EMRI waveforms" (arXiv:2311.17174).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load, call or link
 * this file: only the test-suite, the package smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes, step by step, in the paper's order:
 *   1. per-walker propagation constants: EM luminosity distance d_L(z), the
 *      damping Xi(z) of Eq. (6), d_GW = Xi d_L, and the GW-speed delay
 *      (paper Sec. 2, Eqs. (4)-(6));
 *   2. the AK orbit Y = {Phi, nu, e, gamma~, alpha} of Eq. (1), integrated with
 *      fixed-step classical RK4 at the sampling step dt (paper Sec. 3,
 *      "Waveform computation"; the AK right-hand side is the one of
 *      Barack & Cutler 2004, Phys. Rev. D 69, 082005, which the paper cites for
 *      its equations);
 *   3. the Peters-Mathews harmonic sum of Eq. (2) with the LISA beam pattern and
 *      the Doppler phase of Barack & Cutler 2004, giving the two detector
 *      channels h_I, h_II at unit distance (1 cm); the distance is applied in
 *      the likelihood, as the paper's Sec. 3 module description says;
 *   4. the FFT (own recursive radix-2, no library) with h~_k = dt * DFT;
 *   5. the noise-weighted inner product and lnL of Eq. (8).
 *
 * Precision.  The orbit state, all phase bookkeeping and the reduction of
 * n*Phi modulo 2 pi run in long double (x87 80-bit on x86-64, IEEE binary128
 * on AArch64).  The GW-speed delay fraction is computed in _Float128 on every
 * platform, because the delay is ~1e15 s and the per-bin phase needs it to
 * ~1e-25 relative.  Amplitude arithmetic (Bessel functions, antenna patterns)
 * is double.  Physical constants are the double values of their decimal
 * strings, widened exactly, so every implementation starting from the same
 * decimals starts from the same binary constants.
 *
 * Parity status (what pins each function; see tests/test_oracle_pins.py):
 *   bessel series            pinned: scipy.special.jv, Neumann sum rule
 *   Peters-Mathews brackets  pinned: e=0 closed form (only n=2 survives),
 *                            Peters-Mathews power sum rule
 *   nu_LSO                   pinned: Schwarzschild ISCO frequency, separatrix
 *   AK RHS, Newtonian parts  pinned: quadrupole chirp closed form (e=0),
 *                            Peters a(e) invariant (e>0)
 *   AK RHS, precession       pinned: periastron advance leading term (x->0),
 *                            Lense-Thirring rate, spin/LT identity
 *   AK RHS, 1PN dnu/dt at e=0 pinned: textbook test-mass circular chirp
 *                            (743/336) converted to the radial frequency by
 *                            the 1PN periastron advance
 *   AK RHS, 2PN periastron term at e=0
 *                            pinned: exact circular-orbit Schwarzschild
 *                            periastron advance expanded in the radial frequency
 *   AK RHS, the e-dependent 1PN and 2PN terms and the spin-orbit
 *   radiation-reaction coefficients:
 *                            PARITY UNPINNED (the coefficients come from
 *                            Barack & Cutler 2004, not printed in the paper)
 *   RK4 integrator           pinned: chirp closed form, step halving
 *   antenna patterns         pinned: F+^2+Fx^2 independent of psi,
 *                            F_II(phi) = F_I(phi - pi/4)
 *   FFT                      pinned: brute-force DFT, Parseval, impulse
 *   inner product            pinned: time-domain sum (Parseval) for a white
 *                            all-bin weight, one-sided textbook form
 *   d_L, lookback time       pinned: Einstein-de Sitter closed form,
 *                            numerical quadrature (scipy)
 *   lnL                      pinned: noise-free data at the injection gives
 *                            lnL - <d|d>/2 = 0; GR limit; pure delay leaves
 *                            <h|h> unchanged
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double R;
typedef _Float128 Q;

/* ---------------------------------------------------------------- constants
 * cgs units (paper Sec. 2: "we work in cgs units").  The paper does not print
 * the values; these are the standard ones, written as doubles and widened. */
#define CONST(x) ((R)(double)(x))
static const R GM_SUN = CONST(1.32712440018e26);   /* G*M_sun  [cm^3 s^-2]      */
static const R C_CGS = CONST(2.99792458e10);       /* speed of light [cm s^-1] */
static const R MPC_CM = CONST(3.0856775814913673e24); /* megaparsec [cm]       */
static const R AU_OVER_C = CONST(499.004783836);   /* 1 AU / c [s]              */
static const R YEAR_S = CONST(31557600.0);         /* LISA orbital period [s]   */
static const R PI_R = 3.141592653589793238462643383279502884L;

/* parameter order of one walker (16 doubles) */
enum {
  P_M = 0, P_MU, P_SPIN, P_E0, P_NU0, P_PHI0, P_GAM0, P_ALP0,
  P_THS, P_PHS, P_THK, P_PHK, P_LAM, P_Z, P_XI0, P_ALPT, P_COUNT
};

typedef struct {
  int n_max;       /* harmonic cutoff n_max of Eq. (2)                          */
  int pn_terms;    /* 1: full AK right-hand side; 0: Newtonian radiation reaction */
  int doppler;     /* 1: Doppler phase modulation on                            */
  int backward;    /* 1: start at the LSO and integrate backwards (Sec. 3)      */
  double n_xi;     /* exponent n of Eq. (6)                                     */
  double omega_m;  /* flat Lambda-CDM matter density                            */
  double h0;       /* Hubble constant [km s^-1 Mpc^-1]                          */
} orc_opts;

enum { ST_PLUNGE = 1u, ST_BADPARAM = 2u };

/* ------------------------------------------------------------ Bessel J_m(x)
 * Defining power series J_m(x) = sum_k (-1)^k (x/2)^(2k+m) / (k! (m+k)!),
 * negative orders from J_{-m} = (-1)^m J_m.  Used at x = n e <= n, order
 * >= n - 2, where the series has no harmful cancellation. */
static double bessel_series(int m, double x) {
  double half = 0.5 * x, term = 1.0, sum;
  for (int i = 1; i <= m; ++i) term *= half / i;
  sum = term;
  double q = -half * half;
  for (int k = 1; k < 400; ++k) {
    term *= q / ((double)k * (double)(m + k));
    sum += term;
    if (fabs(term) <= 1e-18 * fabs(sum)) break;
  }
  return sum;
}

double orc_bessel_j(int n, double x) {
  int m = n < 0 ? -n : n;
  double v = bessel_series(m, x);
  return (n < 0 && (m & 1)) ? -v : v;
}

/* Peters-Mathews brackets of the harmonic amplitudes (Eq. (2) with the
 * coefficients of Peters & Mathews 1963 as used by Barack & Cutler 2004):
 *   pa = J_{n-2} - 2e J_{n-1} + (2/n) J_n + 2e J_{n+1} - J_{n+2}
 *   pb = J_{n-2} - 2 J_n + J_{n+2}
 *   pc = J_n                                   (all at argument n e)
 * so that a_n = -n A pa cos(n Phi), b_n = -n A sqrt(1-e^2) pb sin(n Phi),
 * c_n = 2 A pc cos(n Phi). */
void orc_pm_brackets(int n, double e, double out[3]) {
  double x = n * e;
  double jm2 = orc_bessel_j(n - 2, x), jm1 = orc_bessel_j(n - 1, x);
  double j0 = orc_bessel_j(n, x), jp1 = orc_bessel_j(n + 1, x), jp2 = orc_bessel_j(n + 2, x);
  out[0] = jm2 - 2.0 * e * jm1 + (2.0 / n) * j0 + 2.0 * e * jp1 - jp2;
  out[1] = jm2 - 2.0 * j0 + jp2;
  out[2] = j0;
}

/* ------------------------------------------------------------- orbit (Eq. 1)
 * Last-stable-orbit frequency (paper Sec. 3, "Waveform computation"):
 * nu_LSO = c^3/(2 pi G M) * ((1 - e^2)/(6 + 2 e))^(3/2). */
static R nu_lso_r(R m_s, R e) {
  R p = (1 - e * e) / (6 + 2 * e);
  return powl(p, 1.5L) / (2 * PI_R * m_s);
}

double orc_nu_lso(double m_sun, double e) {
  R m_s = GM_SUN * (R)m_sun / (C_CGS * C_CGS * C_CGS);
  return (double)nu_lso_r(m_s, (R)e);
}

typedef struct {
  R m_s, mu_s;      /* G M / c^3, G mu / c^3 [s] */
  R spin, coslam;   /* S/M^2, cos(lambda)        */
  int pn;
} orbit_src;

/* Right-hand side f(Y; theta) of Eq. (1); Y = {Phi, nu, e, gamma~, alpha} in
 * radians / Hz.  Coefficients from Barack & Cutler 2004 (the paper's
 * reference for the AK equations); x = 2 pi nu G M / c^3 (paper Sec. 2). */
static void ak_rhs(const orbit_src* s, const R y[5], R dy[5]) {
  const R nu = y[1], e = y[2];
  const R twopinu = 2 * PI_R * nu;
  const R x = twopinu * s->m_s;
  const R x13 = cbrtl(x), x23 = x13 * x13, x83 = x * x * x23;   /* x^(1/3), x^(2/3), x^(8/3) */
  const R x113 = x83 * x;
  const R e2 = e * e, e4 = e2 * e2, e6 = e4 * e2;
  const R om = 1 - e2;             /* 1 - e^2 */
  const R som = sqrtl(om);         /* (1 - e^2)^(1/2) */
  const R a = s->spin, cl = s->coslam;
  const R mu_m3 = s->mu_s / (s->m_s * s->m_s * s->m_s);
  const R mu_m2 = s->mu_s / (s->m_s * s->m_s);

  /* dPhi/dt */
  dy[0] = twopinu;

  /* dnu/dt */
  R br = (1 + (73.0L / 24) * e2 + (37.0L / 96) * e4) * om;
  if (s->pn) {
    br += x23 * (1273.0L / 336 - (2561.0L / 224) * e2 - (3885.0L / 128) * e4 - (13147.0L / 5376) * e6);
    br -= x * a * cl / som * (73.0L / 12 + (1211.0L / 24) * e2 + (3143.0L / 96) * e4 + (65.0L / 64) * e6);
  }
  dy[1] = (96.0L / (10 * PI_R)) * mu_m3 * x113 / (om * om * om * om * som) * br;

  /* de/dt */
  R eb;
  if (s->pn) {
    eb = (304 + 121 * e2) * om * (1 + 12 * x23)
       - (1.0L / 56) * x23 * (8 * 16705.0L + 12 * 9082.0L * e2 - 25211.0L * e4);
  } else {
    eb = (304 + 121 * e2) * om;
  }
  R de = -(e / 15) * mu_m2 / (om * om * om * som) * x83 * eb;
  if (s->pn)
    de += e * mu_m2 * a * cl * x113 / (om * om * om * om) * (1364.0L / 5 + (5032.0L / 15) * e2 + (263.0L / 10) * e4);
  dy[2] = de;

  /* dgamma~/dt: periastron advance (1PN, 2PN) and its spin-orbit part */
  R dg = 3 * twopinu * x23 / om;
  if (s->pn) dg *= 1 + 0.25L * x23 / om * (26 - 15 * e2);
  dg -= 6 * twopinu * cl * a * x / (om * som);
  dy[3] = dg;

  /* dalpha/dt: Lense-Thirring precession of L about S */
  dy[4] = 2 * twopinu * a * x / (om * som);
}

/* exposed for the pins: the right-hand side at (nu, e) for one walker */
void orc_rhs_eval(const double* theta, double nu, double e, int pn_terms, double out[5]) {
  orbit_src s;
  R c3 = C_CGS * C_CGS * C_CGS;
  s.m_s = GM_SUN * (R)theta[P_M] / c3;
  s.mu_s = GM_SUN * (R)theta[P_MU] / c3;
  s.spin = theta[P_SPIN];
  s.coslam = cosl((R)theta[P_LAM]);
  s.pn = pn_terms;
  R y[5] = {0, nu, e, 0, 0}, dy[5];
  ak_rhs(&s, y, dy);
  for (int i = 0; i < 5; ++i) out[i] = (double)dy[i];
}

static void rk4_step(const orbit_src* s, R y[5], R h) {
  R k1[5], k2[5], k3[5], k4[5], t[5];
  ak_rhs(s, y, k1);
  for (int i = 0; i < 5; ++i) t[i] = y[i] + 0.5L * h * k1[i];
  ak_rhs(s, t, k2);
  for (int i = 0; i < 5; ++i) t[i] = y[i] + 0.5L * h * k2[i];
  ak_rhs(s, t, k3);
  for (int i = 0; i < 5; ++i) t[i] = y[i] + h * k3[i];
  ak_rhs(s, t, k4);
  for (int i = 0; i < 5; ++i) y[i] += h / 6 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
}

static void make_src(const double* th, const orc_opts* o, orbit_src* s) {
  R c3 = C_CGS * C_CGS * C_CGS;
  s->m_s = GM_SUN * (R)th[P_M] / c3;
  s->mu_s = GM_SUN * (R)th[P_MU] / c3;
  s->spin = th[P_SPIN];
  s->coslam = cosl((R)th[P_LAM]);
  s->pn = o->pn_terms;
}

static int bad_params(const double* th) {
  return !(th[P_M] > 0 && th[P_MU] > 0 && th[P_SPIN] >= 0 && th[P_SPIN] <= 1 &&
           th[P_E0] >= 0 && th[P_E0] < 1 && th[P_Z] >= 0);
}

/* Orbit at every sample t_j = t0 + j dt.  Forward mode starts from
 * (Phi0, nu0, e0, gamma0, alpha0) at t0; backward mode puts the last sample at
 * the LSO with e = e0 (paper Sec. 3) and integrates with step -dt.  The state
 * is stored per sample in long double (the caller's arrays, 5*N entries).
 * A forward orbit that reaches nu >= nu_LSO(e) is marked plunged from that
 * sample on.  Returns the first plunged sample index (N if none). */
static int64_t orbit_all(const double* th, const orc_opts* o, int64_t n, double dt, R* ys) {
  orbit_src s;
  make_src(th, o, &s);
  R y[5];
  if (!o->backward) {
    y[0] = th[P_PHI0]; y[1] = th[P_NU0]; y[2] = th[P_E0]; y[3] = th[P_GAM0]; y[4] = th[P_ALP0];
    for (int64_t j = 0; j < n; ++j) {
      if (y[1] >= nu_lso_r(s.m_s, y[2]) || !isfinite((double)y[1])) return j;
      for (int i = 0; i < 5; ++i) ys[5 * j + i] = y[i];
      if (j + 1 < n) rk4_step(&s, y, (R)dt);
    }
    return n;
  }
  y[0] = th[P_PHI0]; y[2] = th[P_E0]; y[1] = nu_lso_r(s.m_s, y[2]); y[3] = th[P_GAM0]; y[4] = th[P_ALP0];
  for (int64_t j = n - 1; j >= 0; --j) {
    for (int i = 0; i < 5; ++i) ys[5 * j + i] = y[i];
    if (j > 0) rk4_step(&s, y, -(R)dt);
  }
  return n;
}

/* exposed: orbit per sample as doubles (Phi, gamma~, alpha in radians) */
int64_t orc_orbit(const double* th, const orc_opts* o, int64_t n, double dt,
                  double* phi, double* nu, double* e, double* gam, double* alp) {
  R* ys = (R*)malloc(sizeof(R) * 5 * (size_t)n);
  if (!ys) return -1;
  int64_t np = orbit_all(th, o, n, dt, ys);
  for (int64_t j = 0; j < n; ++j) {
    int ok = j < np;
    phi[j] = ok ? (double)ys[5 * j] : 0; nu[j] = ok ? (double)ys[5 * j + 1] : 0;
    e[j] = ok ? (double)ys[5 * j + 2] : 0; gam[j] = ok ? (double)ys[5 * j + 3] : 0;
    alp[j] = ok ? (double)ys[5 * j + 4] : 0;
  }
  free(ys);
  return np;
}

/* ------------------------------------------------------ response (Eq. 2)
 * Fractional part of an angle in cycles, from radians in long double. */
static double frac_cycles(R rad) {
  R c = rad / (2 * PI_R);
  return (double)(c - floorl(c));
}

typedef struct {
  double nx, ny, nz;        /* N: direction to the source            */
  double sx, sy, sz;        /* S: spin direction                     */
  double e1x, e1y, e1z;     /* basis of the plane normal to S        */
  double e2x, e2y, e2z;
  double sinlam, coslam, sin_ths, cos_ths, phs;
} geom;

static void make_geom(const double* th, geom* g) {
  double ths = th[P_THS], phs = th[P_PHS], thk = th[P_THK], phk = th[P_PHK];
  g->nx = sin(ths) * cos(phs); g->ny = sin(ths) * sin(phs); g->nz = cos(ths);
  g->sx = sin(thk) * cos(phk); g->sy = sin(thk) * sin(phk); g->sz = cos(thk);
  /* e1 = (z - S cos thK)/sin thK, e2 = S x e1 (orientation of L about S,
   * Barack & Cutler 2004).  For S along z any orthonormal pair is used. */
  double st = sin(thk);
  if (fabs(st) > 1e-12) {
    g->e1x = (0 - g->sx * cos(thk)) / st; g->e1y = (0 - g->sy * cos(thk)) / st; g->e1z = (1 - g->sz * cos(thk)) / st;
  } else {
    g->e1x = 1; g->e1y = 0; g->e1z = 0;
  }
  g->e2x = g->sy * g->e1z - g->sz * g->e1y;
  g->e2y = g->sz * g->e1x - g->sx * g->e1z;
  g->e2z = g->sx * g->e1y - g->sy * g->e1x;
  g->sinlam = sin(th[P_LAM]); g->coslam = cos(th[P_LAM]);
  g->sin_ths = sin(ths); g->cos_ths = cos(ths); g->phs = phs;
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Antenna patterns of one Michelson channel (Barack & Cutler 2004), from
 * the detector-frame angles theta, phi and the polarisation angle psi. */
void orc_antenna(double theta, double phi, double psi, double out[2]) {
  double ct = cos(theta);
  out[0] = 0.5 * (1 + ct * ct) * cos(2 * phi) * cos(2 * psi) - ct * sin(2 * phi) * sin(2 * psi);
  out[1] = 0.5 * (1 + ct * ct) * cos(2 * phi) * sin(2 * psi) + ct * sin(2 * phi) * cos(2 * psi);
}

/* Geometry of the LISA response at time t (Barack & Cutler 2004): with
 * alpha the Lense-Thirring angle of L about S, returns
 * out = {c = L.N, psi, beta, theta_d, phi_d, doppler} where psi is the
 * polarisation angle, beta the angle in the orbital plane from L x N to
 * L x S (gamma = gamma~ + beta), (theta_d, phi_d) the source direction in the
 * rotating detector frame and doppler = (R/c) sin(theta_S) cos(phibar - phi_S)
 * [s], the light-travel delay across the LISA orbit.  Computed with explicit
 * 3-vectors and atan2. */
static void geometry_at(const geom* g, double t, R alpha, double out[6]) {
  const double phib = (double)(2 * PI_R * (R)t / YEAR_S);   /* phibar(t), phibar_0 = 0 */
  const double cdp = cos(phib - g->phs), sdp = sin(phib - g->phs);
  double fa = frac_cycles(alpha);
  double ca = cos(2 * M_PI * fa), sa = sin(2 * M_PI * fa);
  double L[3] = {g->sx * g->coslam + g->sinlam * (g->e1x * ca + g->e2x * sa),
                 g->sy * g->coslam + g->sinlam * (g->e1y * ca + g->e2y * sa),
                 g->sz * g->coslam + g->sinlam * (g->e1z * ca + g->e2z * sa)};
  double N[3] = {g->nx, g->ny, g->nz}, S[3] = {g->sx, g->sy, g->sz};
  double c = dot3(L, N);
  /* detector normal z_d(t) = z/2 - (sqrt3/2)(cos phibar x + sin phibar y) */
  double zd[3] = {-0.5 * sqrt(3.0) * cos(phib), -0.5 * sqrt(3.0) * sin(phib), 0.5};
  /* tan psi = [L.z_d - (L.N)(z_d.N)] / [N.(L x z_d)] */
  double lxz[3];
  cross3(L, zd, lxz);
  double py = dot3(L, zd) - c * dot3(zd, N), px = dot3(N, lxz);
  double psi = (fabs(px) + fabs(py) > 1e-300) ? atan2(py, px) : 0.0;
  /* beta: angle about L from L x N to L x S.  L x S = sin(lam) (p x S) with
   * p = e1 cos a + e2 sin a, so the direction p x S is used: the same angle
   * for sin(lam) > 0, and well conditioned as lam -> 0. */
  double pv[3] = {g->e1x * ca + g->e2x * sa, g->e1y * ca + g->e2y * sa, g->e1z * ca + g->e2z * sa};
  double u[3], v[3], uv[3];
  cross3(L, N, u);
  cross3(pv, S, v);
  double nu_ = sqrt(dot3(u, u)), beta = 0.0;
  if (nu_ > 1e-12) {
    cross3(u, v, uv);
    beta = atan2(dot3(L, uv), dot3(u, v));
  }
  double cth = 0.5 * g->cos_ths - 0.5 * sqrt(3.0) * g->sin_ths * cdp;
  out[0] = c;
  out[1] = psi;
  out[2] = beta;
  out[3] = acos(fmax(-1.0, fmin(1.0, cth)));
  out[4] = phib + atan2(sqrt(3.0) * g->cos_ths + g->sin_ths * cdp, 2 * g->sin_ths * sdp);
  out[5] = (double)AU_OVER_C * g->sin_ths * cdp;
}

/* Harmonic sum of Eq. (2): plus and cross polarisations
 *   A+_n = -(1 + c^2)[a_n cos 2g - b_n sin 2g] + (1 - c^2) c_n,
 *   Ax_n = 2 c [b_n cos 2g + a_n sin 2g],   h = sum_{n=1}^{n_max} A_n,
 * with a_n, b_n, c_n from the Peters-Mathews brackets, amplitude amp,
 * orbital phase phi_c in cycles (reduced exactly per harmonic), 2g in radians. */
static void polarizations(int n_max, double e, double amp, R phi_c, double two_gamma, double c,
                          double* hp_out, double* hx_out) {
  const double som = sqrt(1 - e * e);
  const double c2g = cos(two_gamma), s2g = sin(two_gamma);
  double hp = 0, hx = 0;
  for (int n = 1; n <= n_max; ++n) {
    R nc = (R)n * phi_c;
    double fr = (double)(nc - floorl(nc));
    double cn = cos(2 * M_PI * fr), sn = sin(2 * M_PI * fr);
    double br[3];
    orc_pm_brackets(n, e, br);
    double an = -n * amp * br[0] * cn;
    double bn = -n * amp * som * br[1] * sn;
    double cc = 2 * amp * br[2] * cn;
    hp += -(1 + c * c) * (an * c2g - bn * s2g) + (1 - c * c) * cc;
    hx += 2 * c * (bn * c2g + an * s2g);
  }
  *hp_out = hp;
  *hx_out = hx;
}

/* exposed for the pins */
void orc_polarizations(int n_max, double e, double amp, double phi_cycles, double two_gamma,
                       double c, double out[2]) {
  polarizations(n_max, e, amp, (R)phi_cycles, two_gamma, c, out, out + 1);
}

void orc_geometry(const double* theta, double t, double alpha_rad, double out[6]) {
  geom g;
  make_geom(theta, &g);
  geometry_at(&g, t, (R)alpha_rad, out);
}

/* One time sample of the two detector channels at unit distance (1 cm):
 * h_{I,II} = (sqrt3/2)[F+_{I,II} h+ + Fx_{I,II} hx], channel II with
 * phi -> phi - pi/4; the Doppler phase is added to Phi only. */
static void sample_channels(const orc_opts* o, const geom* g, const orbit_src* s,
                            const R* y, double t, double* hI, double* hII) {
  const R nu = y[1];
  const double e = (double)y[2];
  double geo[6];
  geometry_at(g, t, y[4], geo);
  const double c = geo[0], psi = geo[1], beta = geo[2];
  double fI[2], fII[2];
  orc_antenna(geo[3], geo[4], psi, fI);
  orc_antenna(geo[3], geo[4] - M_PI / 4, psi, fII);
  R phi_d = y[0];
  if (o->doppler) phi_d += 2 * PI_R * nu * (R)geo[5];
  /* amplitude A = x^(2/3) mu at unit distance: mu_s c in cm */
  const double x = (double)(2 * PI_R * nu * s->m_s);
  const double amp = pow(x, 2.0 / 3.0) * (double)(s->mu_s * C_CGS);
  /* 2 gamma = 2 gamma~ + 2 beta */
  const double two_gamma = 2 * M_PI * frac_cycles(2 * y[3]) + 2 * beta;
  double hp, hx;
  polarizations(o->n_max, e, amp, phi_d / (2 * PI_R), two_gamma, c, &hp, &hx);
  const double h3 = 0.5 * sqrt(3.0);
  *hI = h3 * (fI[0] * hp + fI[1] * hx);
  *hII = h3 * (fII[0] * hp + fII[1] * hx);
}

/* Waveform of one walker at the samples idx[0..m) (ascending); all samples
 * when idx is NULL (then m = n).  Returns status bits. */
static uint32_t waveform_one(const double* th, const orc_opts* o, int64_t n, double dt, double t0,
                             const int64_t* idx, int64_t m, double* hI, double* hII) {
  if (bad_params(th)) {
    for (int64_t i = 0; i < m; ++i) hI[i] = hII[i] = 0;
    return ST_BADPARAM;
  }
  orbit_src s;
  make_src(th, o, &s);
  geom g;
  make_geom(th, &g);
  R* ys = (R*)malloc(sizeof(R) * 5 * (size_t)n);
  if (!ys) return ST_BADPARAM;
  int64_t np = orbit_all(th, o, n, dt, ys);
  for (int64_t i = 0; i < m; ++i) {
    int64_t j = idx ? idx[i] : i;
    if (j >= np) { hI[i] = hII[i] = 0; continue; }
    sample_channels(o, &g, &s, ys + 5 * j, t0 + (double)j * dt, hI + i, hII + i);
  }
  free(ys);
  return np < n ? ST_PLUNGE : 0u;
}

/* exposed: W walkers (theta AoS [W][16]), full waveform [W][N] per channel */
void orc_waveform(const double* theta, int w, const orc_opts* o, int64_t n, double dt, double t0,
                  double* hI, double* hII, uint32_t* status, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < w; ++k) {
    uint32_t st = waveform_one(theta + (size_t)k * P_COUNT, o, n, dt, t0, NULL, n,
                               hI + (size_t)k * n, hII + (size_t)k * n);
    if (status) status[k] = st;
  }
}

/* exposed: waveform at sampled indices idx[0..m) for W walkers */
void orc_waveform_sampled(const double* theta, int w, const orc_opts* o, int64_t n, double dt, double t0,
                          const int64_t* idx, int64_t m, double* hI, double* hII, uint32_t* status,
                          int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < w; ++k) {
    uint32_t st = waveform_one(theta + (size_t)k * P_COUNT, o, n, dt, t0, idx, m,
                               hI + (size_t)k * m, hII + (size_t)k * m);
    if (status) status[k] = st;
  }
}

/* ------------------------------------------------------------------ FFT
 * Z_k = sum_j z_j exp(sign * 2 pi i j k / N), recursive radix-2 decimation in
 * time, N a power of two.  tw[m] = exp(sign 2 pi i m / N), m < N/2. */
typedef struct { R re, im; } cplx;

static void fft_rec(const cplx* in, size_t stride, cplx* out, size_t n, const cplx* tw, size_t tw_step) {
  if (n == 1) { out[0] = in[0]; return; }
  size_t h = n / 2;
  fft_rec(in, 2 * stride, out, h, tw, 2 * tw_step);
  fft_rec(in + stride, 2 * stride, out + h, h, tw, 2 * tw_step);
  for (size_t k = 0; k < h; ++k) {
    cplx w = tw[k * tw_step], o = out[k + h], e = out[k];
    R tr = w.re * o.re - w.im * o.im, ti = w.re * o.im + w.im * o.re;
    out[k].re = e.re + tr; out[k].im = e.im + ti;
    out[k + h].re = e.re - tr; out[k + h].im = e.im - ti;
  }
}

static int fft_ld(const cplx* in, cplx* out, size_t n, int sign) {
  if (n == 0 || (n & (n - 1))) return -1;
  if (n == 1) { out[0] = in[0]; return 0; }
  cplx* tw = (cplx*)malloc(sizeof(cplx) * (n / 2));
  if (!tw) return -1;
  for (size_t m = 0; m < n / 2; ++m) {
    R a = 2 * PI_R * (R)m / (R)n;
    tw[m].re = cosl(a); tw[m].im = sign * sinl(a);
  }
  fft_rec(in, 1, out, n, tw, 1);
  free(tw);
  return 0;
}

/* exposed: batch FFT of double (re, im) arrays, computed in long double */
int orc_fft(const double* re, const double* im, int64_t n, int batch, int sign, double* ore, double* oim) {
  cplx* a = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cplx* b = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  int rc = 0;
  if (!a || !b) { free(a); free(b); return -1; }
  for (int k = 0; k < batch && rc == 0; ++k) {
    for (int64_t j = 0; j < n; ++j) { a[j].re = re[(size_t)k * n + j]; a[j].im = im[(size_t)k * n + j]; }
    rc = fft_ld(a, b, (size_t)n, sign);
    for (int64_t j = 0; j < n; ++j) { ore[(size_t)k * n + j] = (double)b[j].re; oim[(size_t)k * n + j] = (double)b[j].im; }
  }
  free(a); free(b);
  return rc;
}

/* exposed: brute-force DFT (definition), exact reduction of j k mod N */
void orc_dft(const double* re, const double* im, int64_t n, int sign, double* ore, double* oim) {
  for (int64_t k = 0; k < n; ++k) {
    R sr = 0, si = 0;
    for (int64_t j = 0; j < n; ++j) {
      R a = 2 * PI_R * (R)((j * k) % n) / (R)n;
      R c = cosl(a), s = sign * sinl(a);
      sr += re[j] * c - im[j] * s;
      si += re[j] * s + im[j] * c;
    }
    ore[k] = (double)sr; oim[k] = (double)si;
  }
}

/* --------------------------------------------------------- cosmology (Eqs. 4-6)
 * E(z) = H(z)/H0 for flat Lambda-CDM. */
static R e_of_z(R z, R om) { R a = 1 + z; return sqrtl(om * a * a * a + (1 - om)); }

static R hubble_inv_s(const orc_opts* o) {   /* 1/H0 [s] */
  return MPC_CM / ((R)o->h0 * (R)1e5);
}

/* EM luminosity distance d_L(z) = (1+z) (c/H0) int_0^z dz'/E(z')  [cm],
 * composite Simpson rule with 2^16 panels. */
double orc_dl_cm(double z, const orc_opts* o) {
  const int n = 1 << 16;
  R h = (R)z / n, sum = 0, om = (R)o->omega_m;
  for (int i = 0; i <= n; ++i) {
    R f = 1 / e_of_z(h * i, om);
    sum += (i == 0 || i == n) ? f : ((i & 1) ? 4 * f : 2 * f);
  }
  return (double)((1 + (R)z) * C_CGS * hubble_inv_s(o) * sum * h / 3);
}

/* Damping Xi(z) = Xi0 + (1 - Xi0)/(1+z)^n, Eq. (6). */
double orc_xi(double z, double xi0, double n_xi) {
  return (double)((R)xi0 + (1 - (R)xi0) / powl(1 + (R)z, (R)n_xi));
}

/* Lookback time t_LB(z) = int_0^z dz' / ((1+z') H(z')) for flat Lambda-CDM,
 * in closed form: (2/(3 H0 sqrt(OL))) [asinh(s) - asinh(s (1+z)^(-3/2))],
 * s = sqrt(OL/Om).  Computed in _Float128. */
static Q lookback_q(double z, const orc_opts* o) {
  Q om = (Q)o->omega_m, ol = 1 - om, s = sqrtf128(ol / om);
  Q zp = 1 + (Q)z;
  Q u = 1 / (zp * sqrtf128(zp));
  Q hinv = (Q)(double)3.0856775814913673e24 / ((Q)o->h0 * (Q)100000);
  return hinv * 2 / (3 * sqrtf128(ol)) * (asinhf128(s) - asinhf128(s * u));
}

double orc_lookback_s(double z, const orc_opts* o) { return (double)lookback_q(z, o); }

/* GW-speed delay (reading of Eqs. (4)-(5) for constant alpha_T):
 * dt_GW = -(alpha_T/2) t_LB(z); the frequency-domain factor is
 * exp(-2 pi i f_k dt_GW) with signed f_k = k_s / T.  Returns
 * r = frac(dt_GW / T) split into two doubles. */
static Q delay_frac_q(double alpha_t, double z, const orc_opts* o, double t_obs_n, double dt) {
  Q dtgw = -(Q)alpha_t / 2 * lookback_q(z, o);
  Q tobs = (Q)t_obs_n * (Q)dt;
  Q q = dtgw / tobs;
  return q - floorf128(q);
}

void orc_delay(double alpha_t, double z, const orc_opts* o, int64_t n, double dt, double out[3]) {
  Q dtgw = -(Q)alpha_t / 2 * lookback_q(z, o);
  Q r = delay_frac_q(alpha_t, z, o, (double)n, dt);
  out[0] = (double)dtgw;
  out[1] = (double)r;
  out[2] = (double)(r - (Q)out[1]);
}

/* ------------------------------------------------------- inner product (Eq. 8)
 * Per-bin weights w_k = 2 dt^2 df / S_n(|f_k|) for 0 < k < N/2 and
 * fmin <= |f_k| <= fmax, zero elsewhere (DC and Nyquist excluded), so that
 * sum_k w_k Re(conj(A_k) B_k) over all k equals the one-sided
 * 4 Re sum_{k>0} a~*_k b~_k / S_n df with a~ = dt A. psd has N/2+1 entries. */
void orc_weights(const double* psd, int64_t n, double dt, double fmin, double fmax, double* w) {
  R df = 1 / ((R)n * (R)dt);
  for (int64_t k = 0; k < n; ++k) {
    int64_t kk = k <= n / 2 ? k : n - k;
    R f = kk * df;
    int in = kk > 0 && 2 * kk < n && f >= fmin && f <= fmax;
    w[k] = in ? (double)(2 * (R)dt * (R)dt * df / (R)psd[kk]) : 0.0;
  }
}

/* exposed: sum_k w_k Re(conj(A_k) B_k) */
double orc_inner(const double* ar, const double* ai, const double* br, const double* bi, const double* w, int64_t n) {
  R s = 0;
  for (int64_t k = 0; k < n; ++k) s += (R)w[k] * ((R)ar[k] * br[k] + (R)ai[k] * bi[k]);
  return (double)s;
}

/* exposed: X_k * exp(-2 pi i frac(k_s r)) for a natural-order spectrum, with
 * r = r_hi + r_lo and signed k_s (the delay factor of the likelihood) */
void orc_delay_apply(const double* re, const double* im, int64_t n, double r_hi, double r_lo,
                     double* ore, double* oim) {
  Q r = (Q)r_hi + (Q)r_lo;
  for (int64_t j = 0; j < n; ++j) {
    int64_t ks = (2 * j <= n) ? j : j - n;
    Q ph = (Q)ks * r;
    ph -= floorf128(ph);
    R a = 2 * PI_R * (R)ph;
    R fr = cosl(a), fi = -sinl(a);
    ore[j] = (double)(re[j] * fr - im[j] * fi);
    oim[j] = (double)(re[j] * fi + im[j] * fr);
  }
}

/* Per-walker propagation constants: out = {d_L [cm], Xi, d_GW [cm], dt_GW [s],
 * r_hi, r_lo} with r = frac(dt_GW / T), T = N dt. */
void orc_prologue(const double* th, const orc_opts* o, int64_t n, double dt, double out[6]) {
  double dl = orc_dl_cm(th[P_Z], o);
  double xi = orc_xi(th[P_Z], th[P_XI0], o->n_xi);
  double d3[3];
  orc_delay(th[P_ALPT], th[P_Z], o, n, dt, d3);
  out[0] = dl; out[1] = xi; out[2] = (double)((R)xi * (R)dl);
  out[3] = d3[0]; out[4] = d3[1]; out[5] = d3[2];
}

/* Frequency-dependent propagation (paper Sec. 2: alpha_M = F(z, f),
 * alpha_T = G(z, f), e.g. a power series in f/f_*, acting on the waveform in
 * frequency space).  Reading: coefficients constant in z,
 *   alpha_M(f) = sum_{m=1..qm} a_m (f/f_*)^m   (its constant part is Xi of Eq. (6)),
 *   alpha_T(f) = alpha_T + sum_{m=1..qt} b_m (f/f_*)^m.
 * With the z-independent alpha_M the damping integral of Sec. 2 is
 * (1/2) alpha_M ln(1+z), so each bin is scaled by (1+z)^(-alpha_M(|f|)/2); the
 * delay of G3 becomes dt_GW(f) = -(alpha_T(|f|)/2) t_LB(z), i.e. the extra
 * phase in cycles -(t_LB/2) sum_m b_m f (|f|/f_*)^m at the signed f = k_s/T. */
typedef struct {
  int qm, qt;
  double fstar;
  const double* coef;   /* a_1..a_qm, b_1..b_qt of this walker */
} fd_walker;

/* Log-likelihood of W walkers against packed data spectrum D_k
 * (D = DFT(d_I + i d_II), natural order, N complex) and weights w (N):
 *   <d|h> = sum_k w_k Re(conj(D_k) H_k F_k exp(-2 pi i k_s r)) / d_GW,
 *   <h|h> = sum_k w_k |H_k F_k|^2 / d_GW^2,
 *   lnL   = <d|h> - <h|h>/2     (the constant -<d|d>/2 is left out),
 * H = DFT(h_I + i h_II) of the unit-distance channels, F_k = 1 or the
 * frequency-dependent factor above.  Also returns the unit-distance sums
 * dh_u = sum w Re(conj D H F e^{..}), hh_u = sum w |H F|^2. */
static void loglike_impl(const double* theta, int w, const orc_opts* o, int64_t n, double dt, double t0,
                         const double* d_re, const double* d_im, const double* wt, int qm, int qt,
                         double fstar, const double* coef, double* lnl, double* dh_u, double* hh_u,
                         uint32_t* status, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < w; ++k) {
    const double* th = theta + (size_t)k * P_COUNT;
    const fd_walker fd = {qm, qt, fstar, coef ? coef + (size_t)k * (qm + qt) : NULL};
    double* hI = (double*)malloc(sizeof(double) * (size_t)n);
    double* hII = (double*)malloc(sizeof(double) * (size_t)n);
    cplx* z = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* Z = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    uint32_t st = ST_BADPARAM;
    double l = NAN, dh = NAN, hh = NAN;
    if (hI && hII && z && Z) {
      st = waveform_one(th, o, n, dt, t0, NULL, n, hI, hII);
      for (int64_t j = 0; j < n; ++j) { z[j].re = hI[j]; z[j].im = hII[j]; }
      fft_ld(z, Z, (size_t)n, -1);
      double pro[6];
      orc_prologue(th, o, n, dt, pro);
      Q r = (Q)pro[4] + (Q)pro[5];
      const int use_fd = fd.coef && (fd.qm > 0 || fd.qt > 0);
      Q tlb = 0, df = 1 / ((Q)n * (Q)dt);
      R l1z = 0;
      if (use_fd) {
        tlb = lookback_q(th[P_Z], o);
        l1z = log1pl((R)th[P_Z]);
      }
      R sdh = 0, shh = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (wt[j] == 0) continue;
        int64_t ks = (2 * j <= n) ? j : j - n;   /* signed frequency index */
        Q ph = (Q)ks * r;
        R amp = 1;
        if (use_fd) {
          Q f = (Q)ks * df;
          Q x = (f < 0 ? -f : f) / (Q)fd.fstar;
          Q xm = 1, am = 0, bt = 0;
          for (int m = 1; m <= (fd.qm > fd.qt ? fd.qm : fd.qt); ++m) {
            xm *= x;
            if (m <= fd.qm) am += (Q)fd.coef[m - 1] * xm;
            if (m <= fd.qt) bt += (Q)fd.coef[fd.qm + m - 1] * xm;
          }
          ph += -tlb / 2 * bt * f;                /* f * dt_GW extra, cycles */
          amp = expl(-0.5L * l1z * (R)am);        /* (1+z)^(-alpha_M(|f|)/2) */
        }
        ph -= floorf128(ph);
        R a = 2 * PI_R * (R)ph;
        R fr = amp * cosl(a), fi = -amp * sinl(a);  /* F_k exp(-2 pi i k_s r) */
        R hr = Z[j].re * fr - Z[j].im * fi, hi = Z[j].re * fi + Z[j].im * fr;
        sdh += (R)wt[j] * ((R)d_re[j] * hr + (R)d_im[j] * hi);
        shh += (R)wt[j] * (Z[j].re * Z[j].re + Z[j].im * Z[j].im) * (amp * amp);
      }
      R dgw = (R)pro[2];
      dh = (double)sdh; hh = (double)shh;
      l = (double)(sdh / dgw - 0.5L * shh / (dgw * dgw));
    }
    free(hI); free(hII); free(z); free(Z);
    lnl[k] = l;
    if (dh_u) dh_u[k] = dh;
    if (hh_u) hh_u[k] = hh;
    if (status) status[k] = st;
  }
}

void orc_loglike(const double* theta, int w, const orc_opts* o, int64_t n, double dt, double t0,
                 const double* d_re, const double* d_im, const double* wt,
                 double* lnl, double* dh_u, double* hh_u, uint32_t* status, int nthreads) {
  loglike_impl(theta, w, o, n, dt, t0, d_re, d_im, wt, 0, 0, 1.0, NULL, lnl, dh_u, hh_u, status, nthreads);
}

/* exposed: the same with frequency-dependent propagation; coef [W][qm+qt]
 * (a_1..a_qm, b_1..b_qt per walker), f_* = fstar [Hz] */
void orc_loglike_fd(const double* theta, int w, const orc_opts* o, int64_t n, double dt, double t0,
                    const double* d_re, const double* d_im, const double* wt, int qm, int qt, double fstar,
                    const double* coef, double* lnl, double* dh_u, double* hh_u, uint32_t* status,
                    int nthreads) {
  loglike_impl(theta, w, o, n, dt, t0, d_re, d_im, wt, qm, qt, fstar, coef, lnl, dh_u, hh_u, status, nthreads);
}
