"""Autotuner: picks a schedule, records it, reads it back from its cache, and
the tuned plan leaves results within the path's tolerances."""
import numpy as np
import pytest

from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_choice_cache_and_results(tmp_path):
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 1 << 14
    cache = str(tmp_path / "plans.jsonl")
    ctx = emri.Context(0)
    psd = I.psd_bc04(n)
    data = I.noise_spectrum(77, psd, n)
    th = I.scatter_walkers(78, I.draw_sources(79, 1, n)[0], 24)
    theta = torch.tensor(th.T.copy(), device="cuda:0")
    # reference results with the default plan
    ds0 = ctx.dataset(emri.grid(n, 15.0), data, psd, 1e-4, 1 / 30.0)
    ref = {}
    for prec in (emri.FP64, emri.MIXED):
        l = torch.zeros(24, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch(ds0, theta, emri.opts(precision=prec, n_max=6), l)
        ref[prec] = l.cpu().numpy()
    ds0.close()
    for prec in (emri.FP64, emri.MIXED):
        ch = ctx.autotune(emri.grid(n, 15.0), 6, prec, cache)
        assert ch["knot_spacing"] in ((128,) if prec == emri.FP64 else (512, 1024))
        assert ch["wave_walkers"] >= 1 and n % ch["fft_n1"] == 0
    lines = open(cache).read().strip().split("\n")
    assert len(lines) == 2
    # a new context reads the cache instead of timing
    ctx2 = emri.Context(0)
    ch2 = ctx2.autotune(emri.grid(n, 15.0), 6, emri.MIXED, cache)
    assert ch2 == ctx.autotune(emri.grid(n, 15.0), 6, emri.MIXED, cache)
    assert len(open(cache).read().strip().split("\n")) == 2
    # results under the tuned plans (dataset created after tuning)
    ds = ctx.dataset(emri.grid(n, 15.0), data, psd, 1e-4, 1 / 30.0)
    for prec, tol in ((emri.FP64, 1e-9), (emri.MIXED, 1e-2)):
        l = torch.zeros(24, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch(ds, theta, emri.opts(precision=prec, n_max=6), l)
        got = l.cpu().numpy()
        err = np.abs(got - ref[prec])
        if prec == emri.FP64:
            assert np.all(err <= tol * (np.abs(ref[prec]) + 1.0))
        else:
            assert np.all(err <= tol)
    ds.close()
    ctx2.close()
    ctx.close()
