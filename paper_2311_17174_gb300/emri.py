"""Thin ctypes binding of ``libemri.so`` (declared in ``include/emri.h``).

Argument marshalling only: every step of the likelihood runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (passed by ``data_ptr``),
streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` ints.  A
missing or unloadable library raises ``RuntimeError`` -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libemri.so")

NPARAM = 16
FP64, MIXED = 0, 1
FORWARD, BACKWARD_FROM_LSO = 0, 1
ST_PLUNGE, ST_BADPARAM, ST_NONFINITE = 1, 2, 4
(OK, EINVAL, ENOMEM, EBUDGET, EAGAIN, ETIMEDOUT, ECUDA, ENOTFOUND) = range(8)
KERNELS = ("prologue", "delay_table", "orbit", "wave", "fft_pass1", "fft_pass2_ip", "finalize",
           "fft_pass2_store")
NKERNEL = len(KERNELS)


class EmriError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"emri error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("n", C.c_int64), ("dt", C.c_double), ("t0", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_max", C.c_int), ("doppler", C.c_int), ("pn_terms", C.c_int),
                ("mode", C.c_int), ("knot_spacing", C.c_int), ("n_xi", C.c_double),
                ("omega_m", C.c_double), ("h0", C.c_double)]


class ServeCfg(C.Structure):
    _fields_ = [("slots", C.c_int), ("queue_capacity", C.c_int), ("budget_bytes", C.c_size_t)]


class ReqStats(C.Structure):
    _fields_ = [("arrival_ns", C.c_int64), ("start_ns", C.c_int64), ("done_ns", C.c_int64),
                ("status", C.c_int32), ("slot", C.c_int32)]


class FdProp(C.Structure):
    _fields_ = [("q_m", C.c_int), ("q_t", C.c_int), ("f_star", C.c_double), ("coef_dev", C.c_void_p)]


class Work(C.Structure):
    _fields_ = [("ds", C.c_void_p), ("theta_dev", C.c_void_p), ("w", C.c_int), ("opts", Opts),
                ("lnl_dev", C.c_void_p), ("dh_dev", C.c_void_p), ("hh_dev", C.c_void_p),
                ("status_dev", C.c_void_p), ("fd", C.POINTER(FdProp))]


class StretchCfg(C.Structure):
    _fields_ = [("a", C.c_double), ("free_mask", C.c_uint32), ("lo", C.c_double * 16), ("hi", C.c_double * 16)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "emri_opts_default": (None, [C.POINTER(Opts)]),
    "emri_last_error": (C.c_char_p, []),
    "emri_version": (C.c_char_p, []),
    "emri_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    "emri_ctx_destroy": (C.c_int, [C.c_void_p]),
    "emri_ctx_set_pipeline": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "emri_ctx_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "emri_ctx_memory": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "emri_ctx_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "emri_ctx_kernel_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "emri_dataset_create": (C.c_int, [C.c_void_p, C.POINTER(Grid), C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_double, C.c_double, C.POINTER(C.c_void_p)]),
    "emri_dataset_destroy": (C.c_int, [C.c_void_p]),
    "emri_dataset_dd": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "emri_prologue": (C.c_int, [C.c_void_p, C.POINTER(Grid), C.c_void_p, C.c_int, C.POINTER(Opts),
                                C.c_void_p, C.c_void_p]),
    "emri_ak_waveform": (C.c_int, [C.c_void_p, C.POINTER(Grid), C.c_void_p, C.c_int, C.POINTER(Opts),
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "emri_fft_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "emri_fft_batch_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "emri_loglike_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "emri_loglike_batch_fd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                        C.POINTER(FdProp), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "emri_loglike_multi": (C.c_int, [C.c_void_p, C.POINTER(Work), C.c_int, C.c_void_p]),
    "emri_serve_start": (C.c_int, [C.c_void_p, C.POINTER(ServeCfg)]),
    "emri_serve_stop": (C.c_int, [C.c_void_p]),
    "emri_serve_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                    C.POINTER(C.c_uint64)]),
    "emri_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(ReqStats),
                                  C.c_int64]),
    "emri_serve_submit_fd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts), C.c_int,
                                       C.c_int, C.c_double, C.c_void_p, C.POINTER(C.c_uint64)]),
    "emri_serve_request_bytes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                           C.POINTER(C.c_size_t)]),
    "emri_stretch_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                    C.POINTER(StretchCfg), C.c_void_p, C.c_void_p, C.c_void_p]),
    "emri_stretch_half": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.POINTER(Opts), C.POINTER(StretchCfg), C.POINTER(FdProp), C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "emri_stretch_step_fd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Opts),
                                       C.POINTER(StretchCfg), C.POINTER(FdProp), C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "emri_autotune": (C.c_int, [C.c_void_p, C.POINTER(Grid), C.c_int, C.c_int, C.c_char_p,
                                C.POINTER(C.c_int64)]),
}


def load(path: str | None = None):
    """Load ``libemri.so`` (raises RuntimeError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libemri.so not found at {p}: build it with "
                                   "paper_2311_17174_gb300.build.build() (no CPU fallback exists)")
            L = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise EmriError(rc, load().emri_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def fft_batch_noalloc(z, n: int, batch: int, precision: int, direction: int = -1, stream=None):
    """emri_fft_batch_noalloc: the in-place batched FFT without a context and
    without any device allocation (fixed library scratch; see include/emri.h)."""
    _check(load().emri_fft_batch_noalloc(_ptr(z), int(n), int(batch), int(precision), int(direction),
                                         _stream(stream)))


def opts(precision=FP64, n_max=10, doppler=1, pn_terms=1, mode=FORWARD, knot_spacing=0, n_xi=2.0,
         omega_m=0.315, h0=67.4) -> Opts:
    return Opts(precision, n_max, doppler, pn_terms, mode, knot_spacing, n_xi, omega_m, h0)


def stretch_cfg(free, lo, hi, a: float = 2.0) -> StretchCfg:
    """Stretch-move configuration: ``free`` parameter indices (theta order),
    prior box ``lo``/``hi`` (16 values each; only the free entries matter)."""
    mask = 0
    for p in free:
        mask |= 1 << int(p)
    return StretchCfg(float(a), mask, (C.c_double * 16)(*[float(x) for x in lo]),
                      (C.c_double * 16)(*[float(x) for x in hi]))


def grid(n: int, dt: float, t0: float = 0.0) -> Grid:
    return Grid(int(n), float(dt), float(t0))


class Context:
    """A library context on one CUDA device (owns tables, workspaces)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = load()
        h = C.c_void_p()
        _check(self.lib.emri_ctx_create(int(device), int(budget_bytes), C.byref(h)))
        self.h = h
        self.device = device
        self._datasets = weakref.WeakSet()

    def close(self):
        if self.h:
            for ds in list(self._datasets):   # datasets die with their context
                ds.close()
            self.lib.emri_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pipeline(self, precision: int, groups: int):
        """Walker groups whose steps overlap on the device (emri_ctx_set_pipeline)."""
        _check(self.lib.emri_ctx_set_pipeline(self.h, int(precision), int(groups)))

    def launches(self) -> int:
        v = C.c_int64()
        _check(self.lib.emri_ctx_launches(self.h, C.byref(v)))
        return v.value

    def memory(self):
        u, b = C.c_size_t(), C.c_size_t()
        _check(self.lib.emri_ctx_memory(self.h, C.byref(u), C.byref(b)))
        return u.value, b.value

    def profile(self, enable: bool = True):
        _check(self.lib.emri_ctx_profile(self.h, 1 if enable else 0))

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        ms = (C.c_double * NKERNEL)()
        cnt = (C.c_int64 * NKERNEL)()
        _check(self.lib.emri_ctx_kernel_times(self.h, ms, cnt))
        return {KERNELS[i]: (ms[i], cnt[i]) for i in range(NKERNEL)}

    # --------------------------------------------------------- datasets
    def dataset(self, g: Grid, data, psd, fmin: float, fmax: float, kind: int = 0) -> "Dataset":
        """``data``: packed spectrum (complex128, n) for kind 0, or [2, n] float64
        time series for kind 1; host numpy or torch tensors; ``psd``: n/2+1 float64."""
        import numpy as np
        keep = []

        def as_ptr(a):
            if hasattr(a, "data_ptr"):
                keep.append(a)
                return a.data_ptr()
            arr = np.ascontiguousarray(a)
            keep.append(arr)
            return arr.ctypes.data

        if kind == 0:
            d = np.ascontiguousarray(np.asarray(data, dtype=np.complex128)) if not hasattr(data, "data_ptr") else data
        else:
            d = np.ascontiguousarray(np.asarray(data, dtype=np.float64)) if not hasattr(data, "data_ptr") else data
        p = np.ascontiguousarray(np.asarray(psd, dtype=np.float64)) if not hasattr(psd, "data_ptr") else psd
        h = C.c_void_p()
        _check(self.lib.emri_dataset_create(self.h, C.byref(g), as_ptr(d), int(kind), as_ptr(p), float(fmin),
                                            float(fmax), C.byref(h)))
        ds = Dataset(self, h, g)
        self._datasets.add(ds)
        return ds

    # ------------------------------------------------------- batch calls
    def prologue(self, g: Grid, theta, o: Opts, out, stream=None):
        _check(self.lib.emri_prologue(self.h, C.byref(g), _ptr(theta), int(theta.shape[1]), C.byref(o),
                                      _ptr(out), _stream(stream)))

    def ak_waveform(self, g: Grid, theta, o: Opts, z_out, status=None, stream=None):
        _check(self.lib.emri_ak_waveform(self.h, C.byref(g), _ptr(theta), int(theta.shape[1]), C.byref(o),
                                         _ptr(z_out), _ptr(status), _stream(stream)))

    def fft_batch(self, z, n: int, batch: int, precision: int, direction: int = -1, stream=None):
        _check(self.lib.emri_fft_batch(self.h, _ptr(z), int(n), int(batch), int(precision), int(direction),
                                       _stream(stream)))

    def loglike_batch(self, ds: "Dataset", theta, o: Opts, lnl, dh=None, hh=None, status=None, stream=None):
        w = int(theta.shape[1]) if theta is not None and hasattr(theta, "shape") else 0
        _check(self.lib.emri_loglike_batch(self.h, ds.h, _ptr(theta), w, C.byref(o), _ptr(lnl), _ptr(dh),
                                           _ptr(hh), _ptr(status), _stream(stream)))

    def loglike_batch_fd(self, ds: "Dataset", theta, o: Opts, q_m: int, q_t: int, f_star: float, coef, lnl,
                         dh=None, hh=None, status=None, stream=None):
        """emri_loglike_batch_fd: coef is a device tensor [q_m + q_t][W] (a_m then b_m)."""
        w = int(theta.shape[1])
        fd = FdProp(int(q_m), int(q_t), float(f_star), _ptr(coef) if coef is not None else None)
        _check(self.lib.emri_loglike_batch_fd(self.h, ds.h, _ptr(theta), w, C.byref(o), C.byref(fd), _ptr(lnl),
                                              _ptr(dh), _ptr(hh), _ptr(status), _stream(stream)))

    def loglike_multi(self, items, stream=None):
        """items: (ds, theta, opts, lnl, dh, hh, status[, fd]) per chain, fd =
        (q_m, q_t, f_star, coef device tensor [q_m + q_t][w]) or None."""
        arr = (Work * len(items))()
        fds = []
        for i, it in enumerate(items):
            ds, theta, o, lnl, dh, hh, st = it[:7]
            fd = it[7] if len(it) > 7 else None
            fp = None
            if fd is not None:
                q_m, q_t, f_star, coef = fd
                fds.append(FdProp(int(q_m), int(q_t), float(f_star), _ptr(coef)))
                fp = C.pointer(fds[-1])
            arr[i] = Work(ds.h.value, _ptr(theta), int(theta.shape[1]), o, _ptr(lnl), _ptr(dh), _ptr(hh),
                          _ptr(st), fp)
        _check(self.lib.emri_loglike_multi(self.h, arr, len(items), _stream(stream)))

    def stretch_step(self, ds: "Dataset", theta, lnp, o: Opts, cfg: StretchCfg, u, accepted=None, stream=None):
        """emri_stretch_step: one affine-invariant ensemble step in place on
        theta [16][W] and lnp [W] (device tensors), driven by the uniforms
        u [3][W] (device)."""
        w = int(theta.shape[1])
        _check(self.lib.emri_stretch_step(self.h, ds.h, _ptr(theta), _ptr(lnp), w, C.byref(o), C.byref(cfg),
                                          _ptr(u), _ptr(accepted), _stream(stream)))

    def stretch_half(self, ds: "Dataset", theta, lnp, o: Opts, cfg: StretchCfg, u, half: int, k0: int, k1: int,
                     accepted=None, stream=None, fd=None):
        """emri_stretch_half: walkers k0..k1-1 of half ``half`` of the ensemble
        theta [16][W] / lnp [W] (device tensors holding the whole ensemble);
        fd = (q_m, q_t, f_star, coef device tensor [q_m + q_t][W]) or None."""
        w = int(theta.shape[1])
        fp = None if fd is None else C.byref(FdProp(int(fd[0]), int(fd[1]), float(fd[2]), _ptr(fd[3])))
        _check(self.lib.emri_stretch_half(self.h, ds.h, _ptr(theta), _ptr(lnp), w, int(half), int(k0), int(k1),
                                          C.byref(o), C.byref(cfg), fp, _ptr(u), _ptr(accepted), _stream(stream)))

    def stretch_step_fd(self, ds: "Dataset", theta, lnp, o: Opts, cfg: StretchCfg, q_m: int, q_t: int,
                        f_star: float, coef, u, accepted=None, stream=None):
        """emri_stretch_step_fd: the ensemble step with a fixed frequency-dependent
        propagation model per walker (coef device tensor [q_m + q_t][W])."""
        w = int(theta.shape[1])
        fd = FdProp(int(q_m), int(q_t), float(f_star), _ptr(coef))
        _check(self.lib.emri_stretch_step_fd(self.h, ds.h, _ptr(theta), _ptr(lnp), w, C.byref(o), C.byref(cfg),
                                             C.byref(fd), _ptr(u), _ptr(accepted), _stream(stream)))

    # ------------------------------------------------------------ serving
    def serve_start(self, slots: int = 4, queue_capacity: int = 1024, budget_bytes: int = 0):
        cfg = ServeCfg(int(slots), int(queue_capacity), int(budget_bytes))
        _check(self.lib.emri_serve_start(self.h, C.byref(cfg)))

    def serve_stop(self):
        _check(self.lib.emri_serve_stop(self.h))

    def serve_submit(self, ds: "Dataset", theta_host, o: Opts) -> int:
        import numpy as np
        th = np.ascontiguousarray(theta_host, dtype=np.float64)
        t = C.c_uint64()
        _check(self.lib.emri_serve_submit(self.h, ds.h, th.ctypes.data, int(th.shape[1]), C.byref(o), C.byref(t)))
        return t.value

    def serve_submit_fd(self, ds: "Dataset", theta_host, o: Opts, q_m: int, q_t: int, f_star: float,
                        coef_host=None) -> int:
        """emri_serve_submit_fd: coef_host [q_m + q_t][W] host array."""
        import numpy as np
        th = np.ascontiguousarray(theta_host, dtype=np.float64)
        cf = None if coef_host is None else np.ascontiguousarray(coef_host, dtype=np.float64)
        t = C.c_uint64()
        _check(self.lib.emri_serve_submit_fd(self.h, ds.h, th.ctypes.data, int(th.shape[1]), C.byref(o), int(q_m),
                                             int(q_t), float(f_star), None if cf is None else cf.ctypes.data,
                                             C.byref(t)))
        return t.value

    def serve_request_bytes(self, ds: "Dataset", w: int, o: Opts) -> int:
        """Pool bytes a request of ``w`` walkers holds while it runs."""
        b = C.c_size_t()
        _check(self.lib.emri_serve_request_bytes(self.h, ds.h, int(w), C.byref(o), C.byref(b)))
        return b.value

    def serve_poll(self, ticket: int, w: int, timeout_us: int = -1):
        """Returns (rc, lnl[w], status[w], stats); rc is OK or ETIMEDOUT."""
        import numpy as np
        lnl = np.zeros(w)
        st = np.zeros(w, dtype=np.uint32)
        stats = ReqStats()
        rc = self.lib.emri_serve_poll(self.h, C.c_uint64(ticket), lnl.ctypes.data, st.ctypes.data,
                                      C.byref(stats), int(timeout_us))
        if rc not in (OK, ETIMEDOUT):
            _check(rc)
        return rc, lnl, st, stats

    def autotune(self, g: Grid, n_max: int, precision: int, cache_path: str | None = None):
        out = (C.c_int64 * 3)()
        _check(self.lib.emri_autotune(self.h, C.byref(g), int(n_max), int(precision),
                                      cache_path.encode() if cache_path else None, out))
        return dict(knot_spacing=out[0], wave_walkers=out[1], fft_n1=out[2])


class Dataset:
    def __init__(self, ctx: Context, h, g: Grid):
        self.ctx, self.h, self.grid = ctx, h, g

    def dd(self) -> float:
        v = C.c_double()
        _check(self.ctx.lib.emri_dataset_dd(self.h, C.byref(v)))
        return v.value

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.emri_dataset_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
