"""Golden fixtures (tests/golden/): the paper's printed example set-up, and
a regression record of the oracle written by tests/golden/make_oracle_regression.py
(which calls only oracle/).  CPU only."""
import importlib.util
import json
import os

import numpy as np
import pytest

from paper_2311_17174_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_paper_workload_follows_the_printed_example():
    g = load("paper_example_fiducial.json")
    wl = I.config_paper(walkers=g["walkers"])
    inj = wl.injection
    assert inj[I.I_M] == g["M_sun"] and inj[I.I_MU] == g["mu_sun"] and inj[I.I_SPIN] == g["spin"]
    assert inj[I.I_XI0] == g["Xi_0"] and inj[I.I_ALPT] == 0.0          # GR speed
    assert inj[I.I_E0] == g["e_LSO"]
    assert (inj[I.I_PHI0], inj[I.I_GAM0], inj[I.I_ALP0]) == (g["Phi_LSO"], g["gamma_LSO"], g["alpha_LSO"])
    np.testing.assert_allclose([inj[I.I_THS], inj[I.I_PHS], inj[I.I_THK], inj[I.I_PHK], inj[I.I_LAM]],
                               [g["theta_S"], g["phi_S"], g["theta_K"], g["phi_K"], g["lambda"]], rtol=0, atol=1e-15)
    assert wl.extra["d_gpc"] == g["distance_Gpc"]
    assert wl.theta.shape[0] == g["walkers"]
    assert wl.n * wl.dt == pytest.approx(g["observation_years"] * 3.15576e7, rel=0.01)
    # only the free parameters are scattered
    free = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]
    fixed = [p for p in range(16) if p not in free]
    np.testing.assert_array_equal(wl.theta[:, fixed], np.repeat(inj[None, fixed], g["walkers"], axis=0))


def test_oracle_regression_record():
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(GOLDEN, "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    ref = load("oracle_regression.json")
    got = mod.compute()
    for key in ("lnl", "dh_u", "hh_u", "h_I", "h_II"):
        np.testing.assert_allclose(np.asarray(got[key]), np.asarray(ref[key]), rtol=1e-11, atol=0, err_msg=key)
    assert got["status"] == ref["status"]
