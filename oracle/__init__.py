"""ctypes front end of the plain CPU oracle (``oracle/emri_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct reference
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module; the product
package never does, and the oracle never imports the product package.

The library is compiled on first use with gcc (``build()``), into this
directory, for the machine it runs on.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emri_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

#: number of parameters of one walker, in the order of ``PARAM_NAMES``
P = 16
PARAM_NAMES = ("M", "mu", "spin", "e0", "nu0", "Phi0", "gamma0", "alpha0",
               "thetaS", "phiS", "thetaK", "phiK", "lambda", "z", "Xi0", "alphaT")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [("n_max", C.c_int), ("pn_terms", C.c_int), ("doppler", C.c_int),
                ("backward", C.c_int), ("n_xi", C.c_double), ("omega_m", C.c_double),
                ("h0", C.c_double)]


@dataclass
class Opts:
    """Oracle options (same meaning as the library's ``emri_opts``)."""
    n_max: int = 10
    pn_terms: int = 1
    doppler: int = 1
    backward: int = 0
    n_xi: float = 2.0
    omega_m: float = 0.315
    h0: float = 67.4

    def c(self) -> _Opts:
        return _Opts(self.n_max, self.pn_terms, self.doppler, self.backward,
                     self.n_xi, self.omega_m, self.h0)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i64, i32, u32 = C.POINTER(C.c_double), C.c_int64, C.c_int, C.POINTER(C.c_uint32)
            po = C.POINTER(_Opts)
            sig = {
                "orc_bessel_j": (C.c_double, [i32, C.c_double]),
                "orc_pm_brackets": (None, [i32, C.c_double, d]),
                "orc_nu_lso": (C.c_double, [C.c_double, C.c_double]),
                "orc_rhs_eval": (None, [d, C.c_double, C.c_double, i32, d]),
                "orc_orbit": (i64, [d, po, i64, C.c_double, d, d, d, d, d]),
                "orc_antenna": (None, [C.c_double, C.c_double, C.c_double, d]),
                "orc_polarizations": (None, [i32, C.c_double, C.c_double, C.c_double, C.c_double,
                                             C.c_double, d]),
                "orc_geometry": (None, [d, C.c_double, C.c_double, d]),
                "orc_waveform": (None, [d, i32, po, i64, C.c_double, C.c_double, d, d, u32, i32]),
                "orc_waveform_sampled": (None, [d, i32, po, i64, C.c_double, C.c_double,
                                                C.POINTER(C.c_int64), i64, d, d, u32, i32]),
                "orc_fft": (i32, [d, d, i64, i32, i32, d, d]),
                "orc_dft": (None, [d, d, i64, i32, d, d]),
                "orc_dl_cm": (C.c_double, [C.c_double, po]),
                "orc_xi": (C.c_double, [C.c_double, C.c_double, C.c_double]),
                "orc_lookback_s": (C.c_double, [C.c_double, po]),
                "orc_delay": (None, [C.c_double, C.c_double, po, i64, C.c_double, d]),
                "orc_weights": (None, [d, i64, C.c_double, C.c_double, C.c_double, d]),
                "orc_inner": (C.c_double, [d, d, d, d, d, i64]),
                "orc_prologue": (None, [d, po, i64, C.c_double, d]),
                "orc_delay_apply": (None, [d, d, i64, C.c_double, C.c_double, d, d]),
                "orc_loglike": (None, [d, i32, po, i64, C.c_double, C.c_double, d, d, d,
                                       d, d, d, u32, i32]),
                "orc_loglike_fd": (None, [d, i32, po, i64, C.c_double, C.c_double, d, d, d, i32, i32,
                                          C.c_double, d, d, d, d, u32, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _theta_aos(theta) -> np.ndarray:
    """Accept [W,16] (AoS) or [16,W] (SoA, as the library takes it)."""
    t = np.asarray(theta, dtype=np.float64)
    if t.ndim == 1:
        t = t[None, :]
    if t.shape[-1] != P and t.shape[0] == P:
        t = t.T
    return np.ascontiguousarray(t)


def _nthreads(n):
    return int(n) if n else int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


# ----------------------------------------------------------------- special
def bessel_j(n: int, x: float) -> float:
    return lib().orc_bessel_j(int(n), float(x))


def pm_brackets(n: int, e: float) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_pm_brackets(int(n), float(e), _dp(out))
    return out


def nu_lso(m_sun: float, e: float) -> float:
    return lib().orc_nu_lso(float(m_sun), float(e))


def rhs(theta, nu: float, e: float, pn_terms: int = 1) -> np.ndarray:
    """Right-hand side (dPhi, dnu, de, dgamma, dalpha)/dt of one walker."""
    t = _f64(_theta_aos(theta)[0])
    out = np.zeros(5)
    lib().orc_rhs_eval(_dp(t), float(nu), float(e), int(pn_terms), _dp(out))
    return out


def antenna(theta_d: float, phi_d: float, psi: float) -> np.ndarray:
    out = np.zeros(2)
    lib().orc_antenna(float(theta_d), float(phi_d), float(psi), _dp(out))
    return out


def polarizations(n_max: int, e: float, amp: float, phi_cycles: float, two_gamma: float,
                  c: float) -> np.ndarray:
    """(h+, hx) of the harmonic sum for one sample."""
    out = np.zeros(2)
    lib().orc_polarizations(int(n_max), float(e), float(amp), float(phi_cycles),
                            float(two_gamma), float(c), _dp(out))
    return out


def geometry(theta, t: float, alpha_rad: float) -> np.ndarray:
    """{L.N, psi, beta, theta_d, phi_d, doppler delay [s]} at time t."""
    tt = _f64(_theta_aos(theta)[0])
    out = np.zeros(6)
    lib().orc_geometry(_dp(tt), float(t), float(alpha_rad), _dp(out))
    return out


# ------------------------------------------------------------------- orbit
def orbit(theta, n: int, dt: float, opts: Opts | None = None):
    """Orbit of one walker at every sample: dict of arrays and the plunge index."""
    o = (opts or Opts()).c()
    t = _f64(_theta_aos(theta)[0])
    arrs = [np.zeros(n) for _ in range(5)]
    np_ = lib().orc_orbit(_dp(t), C.byref(o), int(n), float(dt), *[_dp(a) for a in arrs])
    return dict(phi=arrs[0], nu=arrs[1], e=arrs[2], gamma=arrs[3], alpha=arrs[4], n_valid=int(np_))


def waveform(theta, n: int, dt: float, opts: Opts | None = None, t0: float = 0.0, nthreads=None):
    """Channels (h_I, h_II) [W,N] at unit distance (1 cm) and status bits [W]."""
    o = (opts or Opts()).c()
    t = _theta_aos(theta)
    w = t.shape[0]
    hI = np.zeros((w, n))
    hII = np.zeros((w, n))
    st = np.zeros(w, dtype=np.uint32)
    lib().orc_waveform(_dp(t), w, C.byref(o), int(n), float(dt), float(t0), _dp(hI), _dp(hII),
                       st.ctypes.data_as(C.POINTER(C.c_uint32)), _nthreads(nthreads))
    return hI, hII, st


def waveform_sampled(theta, n: int, dt: float, idx, opts: Opts | None = None, t0: float = 0.0,
                     nthreads=None):
    """Channels at the sample indices ``idx`` (sorted ascending) of an N-sample grid."""
    o = (opts or Opts()).c()
    t = _theta_aos(theta)
    w = t.shape[0]
    ix = np.ascontiguousarray(np.sort(np.asarray(idx, dtype=np.int64)))
    m = ix.size
    hI = np.zeros((w, m))
    hII = np.zeros((w, m))
    st = np.zeros(w, dtype=np.uint32)
    lib().orc_waveform_sampled(_dp(t), w, C.byref(o), int(n), float(dt), float(t0),
                               ix.ctypes.data_as(C.POINTER(C.c_int64)), m, _dp(hI), _dp(hII),
                               st.ctypes.data_as(C.POINTER(C.c_uint32)), _nthreads(nthreads))
    return hI, hII, st


# --------------------------------------------------------------------- FFT
def fft(x, sign: int = -1) -> np.ndarray:
    """sum_j x_j exp(sign 2 pi i j k / N) along the last axis (long double inside)."""
    a = np.asarray(x, dtype=np.complex128)
    shp = a.shape
    a2 = a.reshape(-1, shp[-1])
    re, im = _f64(a2.real), _f64(a2.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(im)
    rc = lib().orc_fft(_dp(re), _dp(im), shp[-1], a2.shape[0], int(sign), _dp(ore), _dp(oim))
    if rc != 0:
        raise ValueError("oracle FFT needs a power-of-two length")
    return (ore + 1j * oim).reshape(shp)


def dft(x, sign: int = -1) -> np.ndarray:
    """Brute-force DFT by definition (O(N^2), long double)."""
    a = np.asarray(x, dtype=np.complex128)
    re, im = _f64(a.real), _f64(a.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(im)
    lib().orc_dft(_dp(re), _dp(im), a.size, int(sign), _dp(ore), _dp(oim))
    return ore + 1j * oim


# -------------------------------------------------------------- cosmology
def dl_cm(z: float, opts: Opts | None = None) -> float:
    o = (opts or Opts()).c()
    return lib().orc_dl_cm(float(z), C.byref(o))


def xi(z: float, xi0: float, n_xi: float = 2.0) -> float:
    return lib().orc_xi(float(z), float(xi0), float(n_xi))


def lookback_s(z: float, opts: Opts | None = None) -> float:
    o = (opts or Opts()).c()
    return lib().orc_lookback_s(float(z), C.byref(o))


def delay(alpha_t: float, z: float, n: int, dt: float, opts: Opts | None = None):
    """(dt_GW [s], r_hi, r_lo) with r = frac(dt_GW / (N dt))."""
    o = (opts or Opts()).c()
    out = np.zeros(3)
    lib().orc_delay(float(alpha_t), float(z), C.byref(o), int(n), float(dt), _dp(out))
    return out


def prologue(theta, n: int, dt: float, opts: Opts | None = None) -> np.ndarray:
    """{d_L [cm], Xi, d_GW [cm], dt_GW [s], r_hi, r_lo} of one walker."""
    o = (opts or Opts()).c()
    t = _f64(_theta_aos(theta)[0])
    out = np.zeros(6)
    lib().orc_prologue(_dp(t), C.byref(o), int(n), float(dt), _dp(out))
    return out


def delay_apply(x, r_hi: float, r_lo: float) -> np.ndarray:
    """x_k exp(-2 pi i frac(k_s r)) (natural order, signed k_s)."""
    a = np.asarray(x, dtype=np.complex128)
    re, im = _f64(a.real), _f64(a.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(im)
    lib().orc_delay_apply(_dp(re), _dp(im), a.size, float(r_hi), float(r_lo), _dp(ore), _dp(oim))
    return ore + 1j * oim


def injection_data(theta_inj, n: int, dt: float, psd, noise_seed: int | None, opts: Opts | None = None,
                   snr: float | None = None, fmin: float = 1e-4, nthreads=None):
    """Data spectrum d = DFT(h(theta_inj)) + noise, built by the oracle.

    h is the unit-distance waveform delayed by the injection's GW-speed delay
    and divided by its d_GW.  With ``snr`` set, the injection's redshift is
    first solved so that sqrt(<h|h>) equals it (the returned theta carries
    that z).  Returns (data, theta_inj, weights, rho_unit)."""
    from paper_2311_17174_gb300 import inputs as _in
    o = opts or Opts()
    th = np.array(theta_inj, dtype=np.float64).copy()
    hI, hII, _ = waveform(th, n, dt, o, nthreads=nthreads)
    H = packed_spectrum(hI[0], hII[0])
    w = weights(psd, n, dt, fmin, 1.0 / (2 * dt))
    rho_u = float(np.sqrt(inner(H, H, w)))
    if snr is not None:
        target = rho_u / snr
        f = lambda z: prologue(np.concatenate([th[:13], [z], th[14:]]), n, dt, o)[2]
        th[13] = _in.solve_distance(target, f)
    pro = prologue(th, n, dt, o)
    d = delay_apply(H, pro[4], pro[5]) / pro[2]
    if noise_seed is not None:
        d = d + _in.noise_spectrum(noise_seed, psd, n, dt)
    return d, th, w, rho_u


# --------------------------------------------------------- inner product
def weights(psd, n: int, dt: float, fmin: float, fmax: float) -> np.ndarray:
    """Per-bin weights w_k (natural DFT order, length N) from a one-sided PSD [N/2+1]."""
    p = _f64(psd)
    assert p.size == n // 2 + 1
    w = np.zeros(n)
    lib().orc_weights(_dp(p), int(n), float(dt), float(fmin), float(fmax), _dp(w))
    return w


def inner(a, b, w) -> float:
    """sum_k w_k Re(conj(a_k) b_k)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ar, ai, br, bi, ww = _f64(a.real), _f64(a.imag), _f64(b.real), _f64(b.imag), _f64(w)
    return lib().orc_inner(_dp(ar), _dp(ai), _dp(br), _dp(bi), _dp(ww), a.size)


def loglike(theta, n: int, dt: float, data_fd, w, opts: Opts | None = None, t0: float = 0.0,
            nthreads=None):
    """lnL, unit-distance <d|h_u>, <h_u|h_u> and status for W walkers.

    ``data_fd`` is the packed data spectrum DFT(d_I + i d_II) in natural order.
    """
    o = (opts or Opts()).c()
    t = _theta_aos(theta)
    nw = t.shape[0]
    d = np.asarray(data_fd, dtype=np.complex128)
    dr, di, ww = _f64(d.real), _f64(d.imag), _f64(w)
    lnl, dh, hh = np.zeros(nw), np.zeros(nw), np.zeros(nw)
    st = np.zeros(nw, dtype=np.uint32)
    lib().orc_loglike(_dp(t), nw, C.byref(o), int(n), float(dt), float(t0), _dp(dr), _dp(di),
                      _dp(ww), _dp(lnl), _dp(dh), _dp(hh),
                      st.ctypes.data_as(C.POINTER(C.c_uint32)), _nthreads(nthreads))
    return lnl, dh, hh, st


def loglike_fd(theta, n: int, dt: float, data_fd, w, qm: int, qt: int, fstar: float, coef,
               opts: Opts | None = None, t0: float = 0.0, nthreads=None):
    """``loglike`` with frequency-dependent propagation: coef [W][qm+qt] holds
    a_1..a_qm (alpha_M) and b_1..b_qt (extra alpha_T terms) per walker, in
    powers of f/fstar."""
    o = (opts or Opts()).c()
    t = _theta_aos(theta)
    nw = t.shape[0]
    d = np.asarray(data_fd, dtype=np.complex128)
    dr, di, ww = _f64(d.real), _f64(d.imag), _f64(w)
    cf = _f64(np.asarray(coef, dtype=np.float64).reshape(nw, qm + qt))
    lnl, dh, hh = np.zeros(nw), np.zeros(nw), np.zeros(nw)
    st = np.zeros(nw, dtype=np.uint32)
    lib().orc_loglike_fd(_dp(t), nw, C.byref(o), int(n), float(dt), float(t0), _dp(dr), _dp(di), _dp(ww),
                         int(qm), int(qt), float(fstar), _dp(cf), _dp(lnl), _dp(dh), _dp(hh),
                         st.ctypes.data_as(C.POINTER(C.c_uint32)), _nthreads(nthreads))
    return lnl, dh, hh, st


def packed_spectrum(hI, hII) -> np.ndarray:
    """DFT of the packed channels h_I + i h_II (oracle FFT), natural order."""
    return fft(np.asarray(hI) + 1j * np.asarray(hII), -1)
