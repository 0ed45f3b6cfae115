"""The seeded input recipes: the two noise models the paper's code
implements (Sec. 3), checked against the published LISA sensitivity levels,
and the shapes the configurations promise."""
import numpy as np

from paper_2311_17174_gb300 import inputs as I


def test_cornish_robson_sensitivity_levels():
    n, dt = 1 << 21, 15.0
    k = lambda f: int(round(f * n * dt))
    s = I.psd_cornish_robson(n, dt)
    si = I.psd_cornish_robson(n, dt, None)
    assert s.shape == (n // 2 + 1,) and np.all(s > 0)
    # the instrument noise bottoms out near 1.2e-20 / sqrt(Hz) at ~10 mHz
    assert 1.1e-20 < np.sqrt(si[k(1e-2)]) < 1.3e-20
    assert np.sqrt(si[k(1e-2)]) < np.sqrt(si[k(1e-3)]) and np.sqrt(si[k(1e-2)]) < np.sqrt(si[k(3e-2)])
    # one-year galactic confusion: dominant at 1-2 mHz, switched off above a few mHz
    assert s[k(1.5e-3)] > 5 * si[k(1.5e-3)]
    assert abs(s[k(6e-3)] / si[k(6e-3)] - 1) < 1e-3
    # longer observations resolve more binaries: less confusion at 2 mHz
    assert I.psd_cornish_robson(n, dt, 4.0)[k(2e-3)] < I.psd_cornish_robson(n, dt, 0.5)[k(2e-3)]


def test_bc04_curve_shape():
    n, dt = 1 << 16, 15.0
    s = I.psd_bc04(n, dt)
    f = np.arange(n // 2 + 1) / (n * dt)
    # f^-4 acceleration noise at low f, flat shot-noise floor, f^2 at high f
    assert abs(s[1] * f[1] ** 4 / 9.18e-52 - 1) < 1e-2
    assert s.min() > 1.59e-41


def test_configuration_shapes():
    wl = I.config_c2(walkers=8, n=1 << 12)
    assert wl.theta.shape == (8, 16) and wl.name == "c2-recipe-8w-2^12-n20"
    assert I.config_c2().name == "c2-1024w-2^21-n20"
    p = I.config_paper(walkers=8, n=1 << 12)
    assert p.theta.shape == (8, 16) and p.extra["mode"] == "backward_from_lso"
