"""Precision sweep: 4096 walkers, 2^20 samples, n <= 20, SNR 20/50/100.

The mixed path (FP32 harmonic sum and FFT, FP64 orbit and phase, FP64 /
compensated inner products) and the all-FP64 path are both compared with
the FP64 oracle on the 32 walkers the workload names: |dlnL| per SNR and the
waveform's relative L2 error on sampled time samples.  Bars: FP64 lnL within
1e-9 (|<d|h>| + <h|h>/2), FP64 waveform 1e-9; mixed |dlnL| <= 1e-2.  The
measured errors are printed (pytest -s) and, with EMRI_REPORT_DIR set,
written there as JSON.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2311_17174_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


def test_c3_precision_sweep():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    report = {"walkers": None, "samples": None, "oracle_walkers": 32, "snr": {}}
    try:
        wl0 = I.config_c3()
        n, dt, nm = wl0.n, wl0.dt, wl0.n_max
        idx = wl0.extra["oracle_idx"]
        psd = I.psd_bc04(n, dt)
        w = O.weights(psd, n, dt, 1e-4, 1.0 / (2 * dt))
        report["walkers"], report["samples"] = int(wl0.w), int(n)
        # waveforms do not depend on the distance: compare them once
        th_o = wl0.theta[idx]
        samp = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(8).integers(0, n, 4094)]))
        sI, sII, st_o = O.waveform_sampled(th_o, n, dt, samp, O.Opts(n_max=nm))
        ref_w = sI + 1j * sII
        werr = {}
        for prec in (0, 1):
            z = torch.zeros((len(idx), n), dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda:0")
            st = torch.zeros(len(idx), dtype=torch.int32, device="cuda:0")
            ctx.ak_waveform(emri.grid(n, dt), torch.tensor(th_o.T.copy(), device="cuda:0"),
                            emri.opts(precision=prec, n_max=nm), z, st)
            torch.cuda.synchronize()
            zz = z.cpu().numpy()[:, samp].astype(np.complex128)
            werr[prec] = max(np.linalg.norm(zz[k] - ref_w[k]) / np.linalg.norm(ref_w[k]) for k in range(len(idx)))
        report["waveform_rel_l2_max"] = {"fp64": werr[0], "mixed": werr[1]}
        assert werr[0] <= 1e-9
        assert werr[1] <= 1e-4
        for snr in (20.0, 50.0, 100.0):
            wl = I.config_c3(snr=snr)
            d, inj2, _, _ = O.injection_data(wl.injection, n, dt, psd, wl.noise_seed, O.Opts(n_max=nm), snr=snr)
            th = wl.theta.copy()
            th[:, I.I_Z] *= inj2[I.I_Z] / wl.injection[I.I_Z]
            ds = ctx.dataset(emri.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
            theta = torch.tensor(th.T.copy(), device="cuda:0")
            got = {}
            for prec in (0, 1):
                lnl = torch.zeros(th.shape[0], dtype=torch.float64, device="cuda:0")
                ctx.loglike_batch(ds, theta, emri.opts(precision=prec, n_max=nm), lnl)
                torch.cuda.synchronize()
                got[prec] = lnl.cpu().numpy()
            ds.close()
            ref, dh_o, hh_o, _ = O.loglike(th[idx], n, dt, d, w, O.Opts(n_max=nm))
            dgw = np.array([O.prologue(t, n, dt)[2] for t in th[idx]])
            tol = 1e-9 * (np.abs(dh_o / dgw) + 0.5 * hh_o / dgw ** 2)
            e64 = np.abs(got[0][idx] - ref)
            emx = np.abs(got[1][idx] - ref)
            report["snr"][f"{snr:g}"] = {
                "fp64_dlnl_max": float(e64.max()), "fp64_dlnl_over_tol_max": float((e64 / tol).max()),
                "mixed_dlnl_max": float(emx.max()),
                "mixed_vs_fp64_all_walkers_max": float(np.abs(got[1] - got[0]).max()),
                "lnl_range": [float(ref.min()), float(ref.max())]}
            assert np.all(e64 <= tol), snr
            assert emx.max() <= 1e-2, snr
    finally:
        ctx.close()
        print(json.dumps(report, indent=1))
        out = os.environ.get("EMRI_REPORT_DIR")
        if out:
            os.makedirs(out, exist_ok=True)
            with open(os.path.join(out, "precision_c3.json"), "w") as f:
                json.dump(report, f, indent=1)
