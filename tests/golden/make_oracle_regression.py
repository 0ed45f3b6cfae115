"""Writes oracle_regression.json: the oracle's lnL, <d|h_u>, <h_u|h_u> and a
few waveform samples for a fixed small case.  Calls only oracle/ (and the
seeded input draws); rerun it only with a commit message that names the
passage of the paper (or its reading) that justifies a change of the
oracle's arithmetic.  Usage: python tests/golden/make_oracle_regression.py"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2311_17174_gb300 import inputs as I  # noqa: E402


def case():
    n, dt, nm = 1 << 12, 15.0, 4
    th = I.draw_sources(301, 4, n)
    psd = I.psd_bc04(n, dt)
    w = O.weights(psd, n, dt, 1e-4, 1.0 / (2 * dt))
    data = I.noise_spectrum(302, psd, n, dt)
    return n, dt, nm, th, w, data


def compute():
    n, dt, nm, th, w, data = case()
    lnl, dh, hh, st = O.loglike(th, n, dt, data, w, O.Opts(n_max=nm))
    idx = [0, 1, 777, n - 1]
    sI, sII, _ = O.waveform_sampled(th, n, dt, idx, O.Opts(n_max=nm))
    return {"n": n, "dt": dt, "n_max": nm, "sources_seed": 301, "noise_seed": 302,
            "lnl": lnl.tolist(), "dh_u": dh.tolist(), "hh_u": hh.tolist(), "status": st.tolist(),
            "sample_idx": idx, "h_I": sI.tolist(), "h_II": sII.tolist()}


if __name__ == "__main__":
    out = compute()
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("written")
