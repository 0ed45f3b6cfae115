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
