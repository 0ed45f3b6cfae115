"""Uneven batching: several chains with their own datasets, walker counts,
lengths and harmonic cutoffs in one captured multi-chain launch.

Each chain's result must equal (bitwise) the same chain run alone through
emri_loglike_batch, on the first (capturing) call and on a replay with new
parameter values in the same buffers.
"""
import numpy as np
import pytest

from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_multi_chain_matches_single_calls():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    g = np.random.default_rng(44)
    chains = []
    for c in range(6):
        logn = int(g.integers(12, 17))
        n = 1 << logn
        w = int(g.integers(1, 70))
        nm = int(g.integers(3, 12))
        prec = int(c % 2)
        psd = I.psd_bc04(n)
        ds = ctx.dataset(emri.grid(n, 15.0), I.noise_spectrum(300 + c, psd, n), psd, 1e-4, 1 / 30.0)
        th = I.scatter_walkers(400 + c, I.draw_sources(500 + c, 1, n)[0], w)
        theta = torch.tensor(th.T.copy(), device="cuda:0")
        out = [torch.zeros(w, dtype=torch.float64, device="cuda:0") for _ in range(3)]
        st = torch.zeros(w, dtype=torch.int32, device="cuda:0")
        chains.append((ds, theta, emri.opts(precision=prec, n_max=nm), out, st, th))
    for rep in range(2):
        if rep == 1:   # new parameter values, same buffers: the graph is replayed
            for (ds, theta, o, out, st, th) in chains:
                theta[2] = torch.clamp(theta[2] * 0.97, 0, 1)
        items = [(ds, theta, o, out[0], out[1], out[2], st) for (ds, theta, o, out, st, th) in chains]
        ctx.loglike_multi(items)
        torch.cuda.synchronize()
        for (ds, theta, o, out, st, th) in chains:
            ref = [torch.zeros_like(out[0]) for _ in range(3)]
            ctx.loglike_batch(ds, theta, o, ref[0], ref[1], ref[2])
            torch.cuda.synchronize()
            for a, b in zip(out, ref):
                np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    for ch in chains:
        ch[0].close()
    ctx.close()


@pytest.mark.slow
def test_c4_full_configuration():
    """The full uneven-batching configuration: 64 chains of 32-512 walkers,
    2^16-2^22 samples, n_max 5-30, mixed precision, autotuned plans, one
    graph.  Every chain is finite, and eight chains picked across the
    lengths equal (bitwise) the same chains run alone."""
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    wls = I.config_c4()
    for n in sorted({wl.n for wl in wls}):
        ctx.autotune(emri.grid(n, I.DT), 20, emri.MIXED)
    items, dsets = [], []
    for c, wl in enumerate(wls):
        psd = I.psd_bc04(wl.n)
        ds = ctx.dataset(emri.grid(wl.n, I.DT), I.noise_spectrum(wl.noise_seed, psd, wl.n), psd, 1e-4, 1 / 30.0)
        dsets.append(ds)
        w = wl.theta.shape[0]
        theta = torch.tensor(wl.theta.T.copy(), device="cuda:0")
        lnl = torch.zeros(w, dtype=torch.float64, device="cuda:0")
        items.append((ds, theta, emri.opts(precision=emri.MIXED, n_max=wl.n_max), lnl, None, None, None))
    ctx.loglike_multi(items)
    torch.cuda.synchronize()
    for it in items:
        assert bool(torch.isfinite(it[3]).all())
    order = np.argsort([wl.n for wl in wls])
    for c in order[::8]:
        ds, theta, o, lnl, _, _, _ = items[c]
        ref = torch.zeros_like(lnl)
        ctx.loglike_batch(ds, theta, o, ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lnl.cpu().numpy(), ref.cpu().numpy())
    for ds in dsets:
        ds.close()
    ctx.close()
