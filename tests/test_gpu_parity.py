"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances (the accuracy bar of the path):
  * FP64 waveform: ||z_gpu - z_oracle||_2 / ||z_oracle||_2 <= 1e-9 per walker,
    and element-wise max_j |z_gpu,j - z_oracle,j| <= 1e-9 max_j |z_oracle,j|
    (a defect confined to one tile or one orbit segment would be diluted in
    the norm-wise figure, not in this one);
  * FFT: max_k |Z_gpu,k - Z_oracle,k| <= tol max_k |Z_oracle,k| per sequence;
  * FP64 lnL: |dlnL| <= 1e-9 (|<d|h>| + <h|h>/2) per walker;
  * mixed lnL: |dlnL| <= 1e-2 absolute (SNR ~50).
Sizes: the 16-source 2^16 configuration in full, the 1024-walker 2^21
ensemble step in the launch configuration the benchmark times, compared on
sampled walkers and samples; ragged walker counts and the edge cases.
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = emri.Context(0)
    yield c
    c.close()


def emri_mod():
    from paper_2311_17174_gb300 import emri
    return emri


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def gpu_waveform(ctx, th, n, dt, n_max, precision=0, **kw):
    E = emri_mod()
    w = th.shape[0]
    z = torch.zeros((w, n), dtype=torch.complex128 if precision == 0 else torch.complex64, device="cuda:0")
    st = torch.zeros(w, dtype=torch.int32, device="cuda:0")
    ctx.ak_waveform(E.grid(n, dt), dev(th.T), E.opts(precision=precision, n_max=n_max, **kw), z, st)
    torch.cuda.synchronize()
    return z.cpu().numpy(), st.cpu().numpy().astype(np.uint32)


def gpu_loglike(ctx, ds, th, n_max, precision=0, **kw):
    E = emri_mod()
    w = th.shape[0]
    out = [torch.zeros(w, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    st = torch.zeros(w, dtype=torch.int32, device="cuda:0")
    ctx.loglike_batch(ds, dev(th.T), E.opts(precision=precision, n_max=n_max, **kw), out[0], out[1], out[2], st)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out] + [st.cpu().numpy().astype(np.uint32)]


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def max_rel(a, b):
    """Element-wise error relative to the largest reference value."""
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def seam_samples(n, seg, extra, seed):
    """Sample indices on both sides of every seg-sample boundary (the orbit
    integrator's segment seams), the ends, and ``extra`` random ones."""
    b = np.arange(seg, n, seg)
    return np.unique(np.concatenate([[0, 1, n - 2, n - 1], b - 1, b,
                                     np.random.default_rng(seed).integers(0, n, extra)]))


# ------------------------------------------------------------- waveform
def test_waveform_c1_full(ctx):
    wl = I.config_c1()
    hI, hII, st_o = O.waveform(wl.theta, wl.n, wl.dt, O.Opts(n_max=wl.n_max))
    z, st = gpu_waveform(ctx, wl.theta, wl.n, wl.dt, wl.n_max)
    np.testing.assert_array_equal(st, st_o)
    for k in range(wl.w):
        ref = hI[k] + 1j * hII[k]
        err = rel_l2(z[k], ref)
        assert err <= 1e-9, (k, err)
        assert max_rel(z[k], ref) <= 1e-9, (k, max_rel(z[k], ref))


@pytest.mark.parametrize("kw", [dict(doppler=0), dict(pn_terms=0), dict(knot_spacing=64), dict(knot_spacing=256)])
def test_waveform_options(ctx, kw):
    n, dt = 1 << 14, 15.0
    th = I.draw_sources(31, 5, n)
    oo = O.Opts(n_max=7, doppler=kw.get("doppler", 1), pn_terms=kw.get("pn_terms", 1))
    hI, hII, _ = O.waveform(th, n, dt, oo)
    z, _ = gpu_waveform(ctx, th, n, dt, 7, **kw)
    for k in range(th.shape[0]):
        assert rel_l2(z[k], hI[k] + 1j * hII[k]) <= 1e-9
        assert max_rel(z[k], hI[k] + 1j * hII[k]) <= 1e-9, (k, max_rel(z[k], hI[k] + 1j * hII[k]))


@pytest.mark.parametrize("dt,doppler", [(60.0, 1), (100.0, 1), (2000.0, 0)])
def test_waveform_long_sample_interval(ctx, dt, doppler):
    # The antenna patterns are a per-tile cubic in time up to 64 s (FP64) and
    # 1024 s (mixed) and exact per sample above: 60 s fits both, 100 s is
    # exact in FP64 only, 2000 s exact in both.  Knots every 64 samples and
    # slowly evolving sources keep the orbit interpolation (a cubic Hermite
    # over the knot interval, error ~ (K_s dt)^4) near 1e-11 rad, so the
    # patterns are what is tested.  At 2000 s the yearly Doppler modulation
    # of the phase (~3 rad) alone would leave a ~3e-9 rad Hermite error over
    # 64 * 2000 s, so that case runs without it.
    n = 1 << 13
    th = I.draw_sources(35, 3, n, dt=dt, t_margin=(50.0, 100.0))
    hI, hII, _ = O.waveform(th, n, dt, O.Opts(n_max=6, doppler=doppler))
    z, _ = gpu_waveform(ctx, th, n, dt, 6, knot_spacing=64, doppler=doppler)
    zm, _ = gpu_waveform(ctx, th, n, dt, 6, precision=1, knot_spacing=64, doppler=doppler)
    for k in range(th.shape[0]):
        ref = hI[k] + 1j * hII[k]
        assert rel_l2(z[k], ref) <= 1e-9, (k, rel_l2(z[k], ref))
        assert max_rel(z[k], ref) <= 1e-9, (k, max_rel(z[k], ref))
        assert rel_l2(zm[k].astype(np.complex128), ref) <= 2e-5, (k, rel_l2(zm[k], ref))


def test_waveform_eccentricity_zero_and_edges(ctx):
    # e0 = 0 (only n = 2 survives), spin 0, lambda near 0, theta_K = 0
    n, dt = 1 << 12, 15.0
    th = I.draw_sources(32, 4, n)
    th[0, I.I_E0] = 0.0
    th[1, I.I_SPIN] = 0.0
    th[2, I.I_LAM] = 1e-9
    th[3, I.I_THK] = 0.0
    hI, hII, _ = O.waveform(th, n, dt, O.Opts(n_max=8))
    z, _ = gpu_waveform(ctx, th, n, dt, 8)
    for k in range(4):
        assert rel_l2(z[k], hI[k] + 1j * hII[k]) <= 1e-9, k
        assert max_rel(z[k], hI[k] + 1j * hII[k]) <= 1e-9, k


def test_waveform_plunge_and_badparam(ctx):
    n, dt = 1 << 13, 15.0
    th = I.draw_sources(33, 3, n)
    th[0, I.I_NU0] = 0.999 * O.nu_lso(th[0, I.I_M], th[0, I.I_E0])
    th[0, I.I_MU] = 20.0
    th[1, I.I_E0] = 1.5
    hI, hII, st_o = O.waveform(th, n, dt, O.Opts(n_max=6))
    z, st = gpu_waveform(ctx, th, n, dt, 6)
    E = emri_mod()
    assert st[0] & E.ST_PLUNGE and st_o[0] & 1
    jo = np.nonzero(hI[0])[0].max() + 1
    jg = np.nonzero(z[0])[0].max() + 1
    assert jo == jg
    assert rel_l2(z[0, :jo], hI[0, :jo] + 1j * hII[0, :jo]) <= 1e-9
    # element-wise, including the samples just before the plunge
    assert max_rel(z[0, :jo], hI[0, :jo] + 1j * hII[0, :jo]) <= 1e-9
    assert st[1] & E.ST_BADPARAM and np.all(z[1] == 0)
    assert st[2] == 0


def test_waveform_mixed_error(ctx):
    wl = I.config_c1()
    th = wl.theta[:4]
    hI, hII, _ = O.waveform(th, wl.n, wl.dt, O.Opts(n_max=wl.n_max))
    z, _ = gpu_waveform(ctx, th, wl.n, wl.dt, wl.n_max, precision=1)
    for k in range(4):
        assert rel_l2(z[k].astype(np.complex128), hI[k] + 1j * hII[k]) <= 2e-5


# ----------------------------------------------------------------- FFT
@pytest.mark.parametrize("logn", [10, 11, 15, 16, 20])
def test_fft_matches_oracle(ctx, logn):
    E = emri_mod()
    n = 1 << logn
    g = np.random.default_rng(logn)
    x = g.standard_normal((3, n)) + 1j * g.standard_normal((3, n))
    ref_f = O.fft(x, -1)
    ref_i = O.fft(x, 1)
    for prec, tol in ((E.FP64, 1e-14), (E.MIXED, 3e-6)):
        dt_ = torch.complex128 if prec == E.FP64 else torch.complex64
        for sign, ref in ((-1, ref_f), (1, ref_i)):
            z = torch.tensor(x, dtype=dt_, device="cuda:0")
            ctx.fft_batch(z, n, 3, prec, sign)
            torch.cuda.synchronize()
            got = z.cpu().numpy().astype(np.complex128)
            for b in range(3):
                assert rel_l2(got[b], ref[b]) <= tol * np.sqrt(logn), (prec, sign, b)


@pytest.mark.parametrize("logn", [21, 22])
def test_fft_full_size_per_bin(ctx, logn):
    """The benchmark's length (2^21: split 2048 x 1024) and the largest grid
    (2^22: 2048 x 2048), both precisions and directions, every bin against
    the oracle's long-double FFT, through emri_fft_batch and through the
    allocation-free entry point (which takes n <= 2^21 in FP64)."""
    E = emri_mod()
    n = 1 << logn
    g = np.random.default_rng(100 + logn)
    x = g.standard_normal((1, n)) + 1j * g.standard_normal((1, n))
    for sign in (-1, 1):
        ref = O.fft(x, sign)[0]
        for prec, tol in ((E.FP64, 1e-14), (E.MIXED, 3e-6)):
            dt_ = torch.complex128 if prec == E.FP64 else torch.complex64
            calls = [lambda z: ctx.fft_batch(z, n, 1, prec, sign)]
            if prec == E.MIXED or logn <= 21:
                calls.append(lambda z: E.fft_batch_noalloc(z, n, 1, prec, sign))
            for call in calls:
                z = torch.tensor(x, dtype=dt_, device="cuda:0")
                call(z)
                torch.cuda.synchronize()
                got = z[0].cpu().numpy().astype(np.complex128)
                assert max_rel(got, ref) <= tol * np.sqrt(logn), (prec, sign, max_rel(got, ref))
                assert rel_l2(got, ref) <= tol * np.sqrt(logn), (prec, sign, rel_l2(got, ref))


def test_fft_batch_beyond_grid_limit(ctx):
    """A batch of more short sequences than one launch's grid holds (65535):
    the call splits it, and every sequence equals the same sequence
    transformed in a smaller batch."""
    E = emri_mod()
    n, batch = 1 << 10, 70000
    g = torch.Generator(device="cuda:0").manual_seed(5)
    x = torch.randn((batch, n), dtype=torch.complex64, device="cuda:0", generator=g)
    a = x.clone()
    ctx.fft_batch(a, n, batch, E.MIXED, -1)
    b = x.clone()
    ctx.fft_batch(b[:35000], n, 35000, E.MIXED, -1)
    ctx.fft_batch(b[35000:], n, batch - 35000, E.MIXED, -1)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ref = O.fft(x[-1:].cpu().numpy().astype(np.complex128), -1)[0]
    assert max_rel(a[-1].cpu().numpy().astype(np.complex128), ref) <= 3e-6 * np.sqrt(10)


# -------------------------------------------------------------- prologue
def test_prologue_matches_oracle(ctx):
    E = emri_mod()
    n, dt = 1 << 21, 15.0
    th = I.draw_sources(41, 64, n)
    th[0, I.I_ALPT] = 0.0
    th[1, I.I_XI0] = 1.0
    th[2, I.I_Z] = 1e-3
    out = torch.zeros((6, 64), dtype=torch.float64, device="cuda:0")
    ctx.prologue(E.grid(n, dt), dev(th.T), E.opts(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(64):
        ref = O.prologue(th[k], n, dt)
        np.testing.assert_allclose(got[:3, k], ref[:3], rtol=1e-13)
        assert got[3, k] == pytest.approx(ref[3], rel=1e-15, abs=0)
        # the delay fraction to ~1e-20 absolute: double-double on both sides
        dr = (got[4, k] - ref[4]) + (got[5, k] - ref[5])
        assert abs(dr) < 1e-20, (k, dr)


# ------------------------------------------------------------- likelihood
def make_dataset(ctx, th_inj, n, dt, n_max, noise_seed, snr=None):
    E = emri_mod()
    psd = I.psd_bc04(n, dt)
    d, th_inj2, w, rho = O.injection_data(th_inj, n, dt, psd, noise_seed, O.Opts(n_max=n_max), snr=snr)
    ds = ctx.dataset(E.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
    return ds, d, w, th_inj2


def lnl_tol(dh, hh):
    return 1e-9 * (np.abs(dh) + 0.5 * hh)


def test_loglike_c1_fp64_and_mixed(ctx):
    wl = I.config_c1()
    ds, d, w, _ = make_dataset(ctx, wl.injection, wl.n, wl.dt, wl.n_max, wl.noise_seed)
    ref, dh_o, hh_o, st_o = O.loglike(wl.theta, wl.n, wl.dt, d, w, O.Opts(n_max=wl.n_max))
    lnl, dh, hh, st = gpu_loglike(ctx, ds, wl.theta, wl.n_max)
    np.testing.assert_array_equal(st, st_o)
    dgw = np.array([O.prologue(t, wl.n, wl.dt)[2] for t in wl.theta])
    tol = lnl_tol(dh_o / dgw, hh_o / dgw ** 2)
    assert np.all(np.abs(lnl - ref) <= tol), (np.abs(lnl - ref) / tol).max()
    np.testing.assert_allclose(hh, hh_o, rtol=2e-9)
    assert ds.dd() == pytest.approx(O.inner(d, d, w), rel=1e-12)
    lnl_m, _, _, _ = gpu_loglike(ctx, ds, wl.theta, wl.n_max, precision=1)
    assert np.max(np.abs(lnl_m - ref)) <= 1e-2


def test_loglike_ragged_and_deterministic(ctx):
    # 37 walkers (not a multiple of any tile); results of a walker do not depend on the batch
    n, dt = 1 << 14, 15.0
    inj = I.draw_sources(51, 1, n)[0]
    th = I.scatter_walkers(52, inj, 37)
    ds, d, w, _ = make_dataset(ctx, inj, n, dt, 6, 53, snr=50.0)
    lnl, dh, hh, st = gpu_loglike(ctx, ds, th, 6)
    ref, dh_o, hh_o, _ = O.loglike(th, n, dt, d, w, O.Opts(n_max=6))
    dgw = np.array([O.prologue(t, n, dt)[2] for t in th])
    assert np.all(np.abs(lnl - ref) <= lnl_tol(dh_o / dgw, hh_o / dgw ** 2))
    for prec in (0, 1):
        full = gpu_loglike(ctx, ds, th, 6, precision=prec)[0]
        for sub in (slice(0, 1), slice(5, 6), slice(10, 29)):
            part = gpu_loglike(ctx, ds, th[sub], 6, precision=prec)[0]
            np.testing.assert_array_equal(part, full[sub])


def test_loglike_zero_walkers_and_gr_limit(ctx):
    E = emri_mod()
    n, dt = 1 << 12, 15.0
    inj = I.draw_sources(61, 1, n)[0]
    inj[I.I_XI0] = 1.0
    inj[I.I_ALPT] = 0.0
    ds, d, w, inj2 = make_dataset(ctx, inj, n, dt, 5, None)
    empty = torch.zeros((16, 0), dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, empty, E.opts(n_max=5), torch.zeros(1, dtype=torch.float64, device="cuda:0"))
    # noise-free data at the injection: lnL - <d|d>/2 = 0
    lnl, dh, hh, st = gpu_loglike(ctx, ds, inj2[None, :], 5)
    assert abs(lnl[0] - 0.5 * ds.dd()) <= 1e-9 * ds.dd()


def test_backward_from_lso_paper_workload(ctx):
    """Backward-from-LSO integration (the paper's own set-up: e_LSO = 0.3,
    fixed geometry, M, mu, S/M^2, Xi_0 free), FP64 and mixed, waveform and
    lnL against the oracle in backward mode; noise-free data at 1 Gpc."""
    wl = I.config_paper(walkers=8, n=1 << 16, n_max=10)
    n, dt, nm = wl.n, wl.dt, wl.n_max
    ob = O.Opts(n_max=nm, backward=1)
    # redshift of 1 Gpc from the oracle's distance (bisection)
    mpc = 3.0856775814913673e24
    z = I.solve_distance(1e3 * mpc, lambda zz: O.dl_cm(zz))
    th = wl.theta.copy()
    th[:, I.I_Z] = z
    inj = wl.injection.copy()
    inj[I.I_Z] = z
    hI, hII, st_o = O.waveform(th, n, dt, ob)
    z64, st = gpu_waveform(ctx, th, n, dt, nm, mode=1)
    np.testing.assert_array_equal(st, st_o)
    assert np.all(st == 0)
    for k in range(len(th)):
        assert rel_l2(z64[k], hI[k] + 1j * hII[k]) <= 1e-9, k
    zm, _ = gpu_waveform(ctx, th, n, dt, nm, precision=1, mode=1)
    assert max(rel_l2(zm[k], hI[k] + 1j * hII[k]) for k in range(len(th))) <= 1e-4
    # the signal ends at the LSO: the last sample's orbit is at nu_LSO(e_LSO)
    orb = O.orbit(th[0], n, dt, ob)
    assert orb["nu"][-1] == pytest.approx(O.nu_lso(th[0, I.I_M], 0.3), rel=1e-15)
    psd = I.psd_bc04(n, dt)
    d, _, w, _ = O.injection_data(inj, n, dt, psd, None, ob)
    ds = ctx.dataset(emri_mod().grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
    ref, dh_o, hh_o, _ = O.loglike(th, n, dt, d, w, ob)
    lnl, _, _, _ = gpu_loglike(ctx, ds, th, nm, mode=1)
    dgw = np.array([O.prologue(t, n, dt)[2] for t in th])
    assert np.all(np.abs(lnl - ref) <= lnl_tol(dh_o / dgw, hh_o / dgw ** 2))
    lnl_m, _, _, _ = gpu_loglike(ctx, ds, th, nm, precision=1, mode=1)
    assert np.max(np.abs(lnl_m - ref)) <= 1e-2
    ds.close()


@pytest.mark.slow
def test_c2_ensemble_step_sampled(ctx):
    """1024 walkers, 2^21 samples, n <= 20, SNR 50, FP64 -- the benchmark's
    launch configuration -- compared with the oracle on 4 sampled walkers
    (lnL) and on 2048 sampled time samples of their waveforms."""
    wl = I.config_c2()
    ds, d, w, inj2 = make_dataset(ctx, wl.injection, wl.n, wl.dt, wl.n_max, wl.noise_seed, snr=wl.snr)
    th = wl.theta.copy()
    th[:, I.I_Z] *= inj2[I.I_Z] / wl.injection[I.I_Z]
    pick = np.array([0, 1, 511, 1023])
    lnl, dh, hh, st = gpu_loglike(ctx, ds, th, wl.n_max)
    assert np.all(st == 0)
    ref, dh_o, hh_o, st_o = O.loglike(th[pick], wl.n, wl.dt, d, w, O.Opts(n_max=wl.n_max))
    dgw = np.array([O.prologue(t, wl.n, wl.dt)[2] for t in th[pick]])
    tol = lnl_tol(dh_o / dgw, hh_o / dgw ** 2)
    assert np.all(np.abs(lnl[pick] - ref) <= tol), (lnl[pick], ref, tol)
    lnl_m = gpu_loglike(ctx, ds, th, wl.n_max, precision=1)[0]
    assert np.max(np.abs(lnl_m[pick] - ref)) <= 1e-2
    # every walker: the two precisions each within 1e-2 of the exact value
    assert np.max(np.abs(lnl_m - lnl)) <= 2e-2
    # waveform samples: both sides of every orbit-segment seam (16384
    # samples in FP64, 65536 in mixed) and random ones
    idx = seam_samples(wl.n, 16384, 1700, 7)
    sI, sII, _ = O.waveform_sampled(th[pick], wl.n, wl.dt, idx, O.Opts(n_max=wl.n_max))
    z, _ = gpu_waveform(ctx, th[pick], wl.n, wl.dt, wl.n_max)
    zm, _ = gpu_waveform(ctx, th[pick], wl.n, wl.dt, wl.n_max, precision=1)
    for k in range(len(pick)):
        ref = sI[k] + 1j * sII[k]
        assert rel_l2(z[k, idx], ref) <= 1e-9, k
        assert max_rel(z[k, idx], ref) <= 1e-9, (k, max_rel(z[k, idx], ref))
        assert max_rel(zm[k, idx].astype(np.complex128), ref) <= 2e-5, (k, max_rel(zm[k, idx], ref))


@pytest.mark.slow
def test_poisoned_workspace_c2_subset(monkeypatch):
    """With the workspace filled with NaN bytes before every call, no kernel
    may read an intermediate value it did not write in the same call: 128
    walkers of the 2^21 ensemble give finite lnL equal (bit for bit) to a
    context without poisoning, in both precisions."""
    E = emri_mod()
    wl = I.config_c2()
    th = wl.theta[::8].copy()
    monkeypatch.setenv("EMRI_DEBUG_POISON", "1")
    cp = E.Context(0)
    monkeypatch.delenv("EMRI_DEBUG_POISON")
    cq = E.Context(0)
    try:
        psd = I.psd_bc04(wl.n, wl.dt)
        d, inj2, _, _ = O.injection_data(wl.injection, wl.n, wl.dt, psd, wl.noise_seed, O.Opts(n_max=wl.n_max),
                                         snr=wl.snr)
        th[:, I.I_Z] *= inj2[I.I_Z] / wl.injection[I.I_Z]
        res = []
        for c in (cp, cq):
            ds = c.dataset(E.grid(wl.n, wl.dt), d, psd, 1e-4, 1.0 / (2 * wl.dt))
            res.append([gpu_loglike(c, ds, th, wl.n_max, precision=p)[0] for p in (0, 1)])
            ds.close()
        for p in (0, 1):
            assert np.all(np.isfinite(res[0][p]))
            np.testing.assert_array_equal(res[0][p], res[1][p])
    finally:
        cp.close()
        cq.close()


@pytest.mark.slow
def test_maximum_length_sampled(ctx):
    """n = 2^22 (the largest grid), FP64 and mixed, two walkers: waveform on
    sampled time samples against the oracle (FP64 1e-9, mixed 1e-4)."""
    n, dt, nm = 1 << 22, 15.0, 6
    th = I.draw_sources(131, 2, n)
    idx = seam_samples(n, 16384, 500, 132)
    sI, sII, st_o = O.waveform_sampled(th, n, dt, idx, O.Opts(n_max=nm))
    z64, st = gpu_waveform(ctx, th, n, dt, nm)
    np.testing.assert_array_equal(st, st_o)
    zm, _ = gpu_waveform(ctx, th, n, dt, nm, precision=1)
    for k in range(2):
        ref = sI[k] + 1j * sII[k]
        assert rel_l2(z64[k, idx], ref) <= 1e-9, k
        assert max_rel(z64[k, idx], ref) <= 1e-9, (k, max_rel(z64[k, idx], ref))
        assert rel_l2(zm[k, idx].astype(np.complex128), ref) <= 1e-4, k


def test_mixed_extreme_options(ctx):
    """Mixed precision at n_max = 32 (the largest cutoff) and knot spacing
    512 (the autotuner's other choice), against the FP64 oracle."""
    n, dt = 1 << 14, 15.0
    th = I.draw_sources(141, 4, n)
    th[:, I.I_E0] = [0.05, 0.3, 0.5, 0.7]
    hI, hII, st_o = O.waveform(th, n, dt, O.Opts(n_max=32))
    for ks in (512, 1024):
        zm, st = gpu_waveform(ctx, th, n, dt, 32, precision=1, knot_spacing=ks)
        np.testing.assert_array_equal(st, st_o)
        for k in range(4):
            if st_o[k] & 1:
                continue
            assert rel_l2(zm[k].astype(np.complex128), hI[k] + 1j * hII[k]) <= 2e-5, (ks, k)
