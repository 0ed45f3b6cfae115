"""Seeded synthetic inputs for the batched AK log-likelihood.

This module only draws numbers: walker parameters, noise realisations and the
analytic noise curve sampled on the frequency grid.  It holds none of the
likelihood's arithmetic (no orbit, waveform, FFT or inner product) and imports
neither the CUDA library nor the oracle, so both sides can be fed the same
inputs from it.  Everything is deterministic given the seed (numpy PCG64).

Parameter order of one walker (16 doubles), following the paper's parameter
set theta = {M, mu, S/M^2, ...} (Sec. 2; the first three are the ones the
orbit solver needs, Sec. 3 "Extending the parameters"):

    0 M [M_sun]      1 mu [M_sun]     2 spin S/M^2     3 e0
    4 nu0 [Hz]       5 Phi0 [rad]     6 gamma0 [rad]   7 alpha0 [rad]
    8 theta_S        9 phi_S         10 theta_K       11 phi_K
   12 lambda        13 z             14 Xi0           15 alpha_T

The library takes them structure-of-arrays, ``theta[16][W]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

P = 16
(I_M, I_MU, I_SPIN, I_E0, I_NU0, I_PHI0, I_GAM0, I_ALP0, I_THS, I_PHS, I_THK, I_PHK,
 I_LAM, I_Z, I_XI0, I_ALPT) = range(P)
#: components perturbed by an absolute (radian) offset rather than a relative one
ANGLE_IDX = (I_PHI0, I_GAM0, I_ALP0, I_THS, I_PHS, I_THK, I_PHK, I_LAM)

DT = 15.0  # sampling step of every configuration [s]
#: G*M_sun / c^3 [s] for the input recipe only (the library and the oracle
#: carry their own constants)
_TSUN = 1.32712440018e26 / 2.99792458e10 ** 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def start_frequency(m_sun: float, mu_sun: float, e0: float, t_to_lso: float) -> float:
    """Input recipe for nu0: the circular quadrupole time from nu0 to the LSO
    frequency of the starting eccentricity equals ``t_to_lso``:
    u0^(-8/3) = uL^(-8/3) + (256/5)(mu/M^2) t,  u = 2 pi (G M/c^3) nu,
    uL = ((1-e0^2)/(6+2 e0))^(3/2).  This only places the start of the orbit so
    that the plunge falls after the observation; the likelihood path does its
    own plunge check on the full equations."""
    m_s, mu_s = m_sun * _TSUN, mu_sun * _TSUN
    u_l = ((1.0 - e0 * e0) / (6.0 + 2.0 * e0)) ** 1.5
    u0 = (u_l ** (-8.0 / 3.0) + (256.0 / 5.0) * (mu_s / m_s ** 2) * t_to_lso) ** (-3.0 / 8.0)
    return u0 / (2.0 * np.pi * m_s)


def draw_sources(seed: int, count: int, n: int, dt: float = DT,
                 t_margin=(1.5, 3.0)) -> np.ndarray:
    """``count`` independent sources [count, 16] with the distributions of the
    configurations: M ~ U[5e5, 5e6], mu ~ U[5, 20], spin ~ U[0, 0.9],
    e0 ~ U[0.1, 0.4], nu0 from ``start_frequency`` with the time to the LSO
    ~ T U[t_margin], cos(theta_S), cos(theta_K), cos(lambda) ~ U[-1, 1],
    phi_S, phi_K, Phi0, gamma0, alpha0 ~ U[0, 2 pi), z ~ U[0.1, 1],
    Xi0 ~ N(1, 0.05), alpha_T ~ N(0, 0.05)."""
    g = _rng(seed)
    t_obs = n * dt
    out = np.zeros((count, P))
    for k in range(count):
        m = g.uniform(5e5, 5e6)
        mu = g.uniform(5.0, 20.0)
        spin = g.uniform(0.0, 0.9)
        e0 = g.uniform(0.1, 0.4)
        tp = t_obs * g.uniform(*t_margin)
        out[k, I_M], out[k, I_MU], out[k, I_SPIN], out[k, I_E0] = m, mu, spin, e0
        out[k, I_NU0] = start_frequency(m, mu, e0, tp)
        out[k, I_PHI0], out[k, I_GAM0], out[k, I_ALP0] = g.uniform(0, 2 * np.pi, 3)
        out[k, I_THS] = np.arccos(g.uniform(-1, 1))
        out[k, I_PHS] = g.uniform(0, 2 * np.pi)
        out[k, I_THK] = np.arccos(g.uniform(-1, 1))
        out[k, I_PHK] = g.uniform(0, 2 * np.pi)
        out[k, I_LAM] = np.arccos(g.uniform(-1, 1))
        out[k, I_Z] = g.uniform(0.1, 1.0)
        out[k, I_XI0] = g.normal(1.0, 0.05)
        out[k, I_ALPT] = g.normal(0.0, 0.05)
    return out


def scatter_walkers(seed: int, center: np.ndarray, count: int, rel: float = 1e-4) -> np.ndarray:
    """``count`` walkers [count, 16] scattered about ``center``: relative
    N(0, rel) for physical components, absolute N(0, rel) radians for angles.
    Walker 0 is the centre itself."""
    g = _rng(seed)
    c = np.asarray(center, dtype=np.float64)
    eps = g.normal(0.0, rel, size=(count, P))
    out = c[None, :] * (1.0 + eps)
    for i in ANGLE_IDX:
        out[:, i] = c[i] + eps[:, i]
    out[0] = c
    # keep physical ranges valid
    out[:, I_SPIN] = np.clip(out[:, I_SPIN], 0.0, 1.0)
    out[:, I_E0] = np.clip(out[:, I_E0], 0.0, 0.95)
    return out


def psd_bc04(n: int, dt: float = DT) -> np.ndarray:
    """One-sided instrumental noise curve of Barack & Cutler 2004 (the noise
    model of the paper's example, Sec. 3) sampled at f_k = k / (N dt), k = 0..N/2:
    S(f) = 9.18e-52 f^-4 + 1.59e-41 + 9.18e-38 f^2  [1/Hz].  The DC entry
    repeats the k=1 value (DC carries no weight)."""
    f = np.arange(n // 2 + 1) / (n * dt)
    f[0] = f[1]
    return 9.18e-52 * f ** -4 + 1.59e-41 + 9.18e-38 * f ** 2


# Galactic-confusion fit parameters (alpha, beta, kappa, gamma, f_k) of the
# Cornish-Robson LISA sensitivity for observation times of 0.5, 1, 2, 4 yr.
_CR_CONFUSION = {0.5: (0.133, 243.0, 482.0, 917.0, 2.58e-3), 1.0: (0.171, 292.0, 1020.0, 1680.0, 2.15e-3),
                 2.0: (0.165, 299.0, 611.0, 1340.0, 1.73e-3), 4.0: (0.138, -221.0, 521.0, 1680.0, 1.13e-3)}


def psd_cornish_robson(n: int, dt: float = DT, t_obs_yr: float | None = 1.0) -> np.ndarray:
    """The second noise model the paper's code implements (Sec. 3): the LISA
    sensitivity of Robson, Cornish & Liu (2019), sampled at f_k = k/(N dt),
    k = 0..N/2 (DC repeats k = 1):
      S_n = 10/(3 L^2) [P_oms + 2 (1 + cos^2(f/f*)) P_acc / (2 pi f)^4] (1 + 0.6 (f/f*)^2) + S_c,
      P_oms = (1.5e-11 m)^2 (1 + (2 mHz/f)^4),
      P_acc = (3e-15 m/s^2)^2 (1 + (0.4 mHz/f)^2) (1 + (f/8 mHz)^4),
    L = 2.5e9 m, f* = c/(2 pi L), plus the galactic confusion
      S_c = 9e-45 f^(-7/3) exp(-f^a + b f sin(k f)) (1 + tanh(g (f_k - f)))
    for the observation time t_obs_yr (0.5, 1, 2 or 4; None: instrument only).
    It is an input array: both the oracle and the kernels take it as given."""
    f = np.arange(n // 2 + 1) / (n * dt)
    f[0] = f[1]
    L = 2.5e9
    fstar = 2.99792458e8 / (2.0 * np.pi * L)
    p_oms = (1.5e-11) ** 2 * (1.0 + (2e-3 / f) ** 4)
    p_acc = (3e-15) ** 2 * (1.0 + (0.4e-3 / f) ** 2) * (1.0 + (f / 8e-3) ** 4)
    s = 10.0 / (3.0 * L * L) * (p_oms + 2.0 * (1.0 + np.cos(f / fstar) ** 2) * p_acc / (2.0 * np.pi * f) ** 4) \
        * (1.0 + 0.6 * (f / fstar) ** 2)
    if t_obs_yr is not None:
        a, b, k, g, fk = _CR_CONFUSION[t_obs_yr]
        s = s + 9e-45 * f ** (-7.0 / 3.0) * np.exp(-f ** a + b * f * np.sin(k * f)) * (1.0 + np.tanh(g * (fk - f)))
    return s


def noise_spectrum(seed: int, psd: np.ndarray, n: int, dt: float = DT) -> np.ndarray:
    """Packed DFT N_k = X_I,k + i X_II,k (natural order, length N) of two
    independent real Gaussian noise channels with one-sided PSD ``psd``:
    for 0 < k < N/2, X_c,k = sqrt(S_k / (2 df dt^2)) (g1 + i g2)/sqrt(2),
    X_c,N-k = conj(X_c,k); DC and Nyquist set to zero (they carry no weight)."""
    g = _rng(seed)
    df = 1.0 / (n * dt)
    k = np.arange(1, n // 2)
    sig = np.sqrt(psd[k] / (2.0 * df * dt * dt) / 2.0)
    x = np.zeros((2, n), dtype=np.complex128)
    for c in range(2):
        z = sig * (g.standard_normal(k.size) + 1j * g.standard_normal(k.size))
        x[c, k] = z
        x[c, n - k] = np.conj(z)
    return x[0] + 1j * x[1]


def solve_distance(target_cm: float, dgw_of_z, lo: float = 1e-4, hi: float = 10.0) -> float:
    """Redshift z with dgw_of_z(z) = target_cm, by bisection (dgw increasing in z).
    The distance function is supplied by the caller."""
    a, b = lo, hi
    for _ in range(200):
        m = 0.5 * (a + b)
        if dgw_of_z(m) < target_cm:
            a = m
        else:
            b = m
        if b - a < 1e-15 * max(1.0, m):
            break
    return 0.5 * (a + b)


@dataclass
class Workload:
    """One configuration: walkers, grid, harmonic cutoff and data recipe."""
    name: str
    theta: np.ndarray            # [W, 16]
    n: int
    dt: float
    n_max: int
    injection: np.ndarray        # [16]
    noise_seed: int
    snr: float | None            # target SNR of the injection (None: drawn z)
    fmin: float = 1e-4
    extra: dict = field(default_factory=dict)

    @property
    def w(self) -> int:
        return self.theta.shape[0]

    def theta_soa(self) -> np.ndarray:
        return np.ascontiguousarray(self.theta.T)


def config_c1() -> Workload:
    """16 independent sources, 2^16 samples, n <= 10; data = source 0 + noise."""
    n = 1 << 16
    th = draw_sources(1, 16, n)
    return Workload("c1-16src-2^16-n10-fp64", th, n, DT, 10, th[0].copy(), 101, None)


def config_c2(walkers: int = 1024, n: int = 1 << 21, n_max: int = 20) -> Workload:
    """One ensemble step: 1024 walkers N(0, 1e-4) about an injection,
    2^21 samples (~1 yr), n <= 20, SNR 50."""
    inj = draw_sources(2, 1, n)[0]
    th = scatter_walkers(1002, inj, walkers)
    lg = int(np.log2(n))
    name = "c2-1024w-2^21-n20" if (walkers, n, n_max) == (1024, 1 << 21, 20) else \
        f"c2-recipe-{walkers}w-2^{lg}-n{n_max}"
    return Workload(name, th, n, DT, n_max, inj, 102, 50.0)


def config_c3(walkers: int = 4096, n: int = 1 << 20, snr: float = 50.0) -> Workload:
    """Precision sweep: 4096 walkers, 2^20 samples, n <= 20, SNR 20/50/100;
    the oracle runs on 32 walkers whose indices come from seed 33."""
    inj = draw_sources(3, 1, n)[0]
    th = scatter_walkers(1003, inj, walkers)
    idx = np.sort(_rng(33).choice(walkers, 32, replace=False))
    return Workload(f"c3-4096w-2^20-n20-snr{snr:g}", th, n, DT, 20, inj, 103, snr,
                    extra={"oracle_idx": idx})


def config_paper(walkers: int = 8, n: int = 1 << 21, n_max: int = 10, seed: int = 6,
                 rel: float = 1e-4) -> Workload:
    """The paper's example run (Sec. 3 and its corner-plot example): initial
    conditions at the LSO with e_LSO = 0.3 and Phi, gamma~, alpha = 0 there,
    theta_S = pi/4, phi_S = 0, theta_K = pi/8, phi_K = 0, lambda = pi/6, fixed;
    the four free parameters M = 1e6, mu = 10, S/M^2 = 0.1, Xi_0 = 1 scattered
    by N(0, rel) relative; GW speed as in GR; a one-year window (n dt);
    noise-free data (the paper's choice).  The source sits at 1 Gpc: z is a
    placeholder that the caller sets from ``extra['d_gpc']`` with its own
    distance function."""
    inj = np.zeros(P)
    inj[[I_M, I_MU, I_SPIN, I_E0, I_NU0]] = [1e6, 10.0, 0.1, 0.3, 0.0]
    inj[[I_THS, I_PHS, I_THK, I_PHK, I_LAM]] = [np.pi / 4, 0.0, np.pi / 8, 0.0, np.pi / 6]
    inj[[I_Z, I_XI0, I_ALPT]] = [0.2, 1.0, 0.0]
    g = _rng(seed)
    th = np.repeat(inj[None, :], walkers, axis=0)
    for p_ in (I_M, I_MU, I_SPIN, I_XI0):
        th[:, p_] *= 1.0 + rel * g.standard_normal(walkers)
    return Workload(f"paper-lso-{walkers}w-2^{int(np.log2(n))}-n{n_max}", th, n, DT, n_max, inj, -1, None,
                    extra={"d_gpc": 1.0, "free": (I_M, I_MU, I_SPIN, I_XI0), "mode": "backward_from_lso"})


def config_c4(chains: int = 64):
    """Uneven batching: ``chains`` independent chains, W_c ~ U{32..512},
    N_c = 2^U{16..22}, n_max_c ~ U{5..30}; own injection, noise and PSD each."""
    g = _rng(4)
    out = []
    for c in range(chains):
        w = int(g.integers(32, 513))
        n = 1 << int(g.integers(16, 23))
        nm = int(g.integers(5, 31))
        inj = draw_sources(4000 + c, 1, n)[0]
        th = scatter_walkers(5000 + c, inj, w)
        out.append(Workload(f"c4-chain{c}", th, n, DT, nm, inj, 6000 + c, 50.0))
    return out


def config_c5(rate: float, duration_s: float, seed: int = 5):
    """Serving: Poisson arrivals at ``rate`` per second over ``duration_s``;
    each request has W ~ U{8..512} walkers and N = 2^U{16..22} samples and
    picks one of 16 resident datasets of its length.  Returns a list of
    (arrival_s, dataset_index, walkers, n)."""
    g = _rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t > duration_s:
            break
        out.append((t, int(g.integers(0, 16)), int(g.integers(8, 513)), 1 << int(g.integers(16, 23))))
    return out
