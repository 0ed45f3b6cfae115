"""The on-device stretch-move ensemble step (emri_stretch_step) against the
oracle's step (oracle/mcmc.py) driven by the same uniforms.

Each step starts both sides from the GPU's current ensemble, so a single
decision taken differently at a near-tie cannot cascade.  Decisions are
compared wherever the oracle's margin clears the FP64 likelihood tolerance;
accepted positions are bit-identical (both sides form the proposal with
correctly rounded operations in the same order); lnP agrees to the
likelihood tolerance and equals emri_loglike_batch at the new positions
bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mcmc as OM
from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FREE = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]   # the paper's four free parameters


def setup(ctx, emri, w, n, n_max, seed):
    dt = 15.0
    inj = I.draw_sources(seed, 1, n)[0]
    psd = I.psd_bc04(n, dt)
    d, inj2, wts, _ = O.injection_data(inj, n, dt, psd, seed + 1, O.Opts(n_max=n_max), snr=25.0)
    th = I.scatter_walkers(seed + 2, inj2, w, rel=3e-5)
    ds = ctx.dataset(emri.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
    lo = np.full(16, -np.inf)
    hi = np.full(16, np.inf)
    for p in FREE:
        lo[p], hi[p] = inj2[p] * (1 - 4e-5), inj2[p] * (1 + 4e-5)
    lo[I.I_SPIN], hi[I.I_SPIN] = 0.0, 0.99
    return ds, d, wts, th, lo, hi, dt


def test_stretch_step_matches_oracle():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    w, n, n_max = 24, 1 << 12, 4
    ds, d, wts, th, lo, hi, dt = setup(ctx, emri, w, n, n_max, 71)
    o = emri.opts(precision=emri.FP64, n_max=n_max)
    cfg = emri.stretch_cfg(FREE, lo, hi, a=2.0)
    theta = torch.tensor(th.T.copy(), device="cuda:0")
    lnp = torch.zeros(w, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, theta, o, lnp)
    acc = torch.zeros(w, dtype=torch.int32, device="cuda:0")

    def lnprob(ys):
        ll, _, _, st = O.loglike(ys, n, dt, d, wts, O.Opts(n_max=n_max))
        return ll, st

    g = np.random.default_rng(99)
    moved = 0
    for step in range(4):
        x0 = theta.cpu().numpy().T.copy()
        lp0 = lnp.cpu().numpy().copy()
        u = g.random((3, w))
        xo, lpo, acco, margin = OM.stretch_step(x0, lp0, u, 2.0, FREE, lo, hi, lnprob)
        ctx.stretch_step(ds, theta, lnp, o, cfg, torch.tensor(u, device="cuda:0"), acc)
        torch.cuda.synchronize()
        xg = theta.cpu().numpy().T
        lpg = lnp.cpu().numpy()
        ag = acc.cpu().numpy()
        clear = ~(np.abs(margin) < 1e-6 * (1 + np.abs(lp0)))   # NaN margins (rejected outright) count as clear
        np.testing.assert_array_equal(ag[clear], acco[clear])
        for k in np.nonzero(clear)[0]:
            np.testing.assert_array_equal(xg[k], xo[k])
            assert abs(lpg[k] - lpo[k]) <= 1e-9 * (1 + abs(lpo[k]))
        moved += int(ag.sum())
        # lnP is the likelihood at the current positions, bit for bit
        chk = torch.zeros(w, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch(ds, theta, o, chk)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(chk.cpu().numpy(), lpg)
        # fixed parameters never move
        fixed = [p for p in range(16) if p not in FREE]
        np.testing.assert_array_equal(xg[:, fixed], x0[:, fixed])
    assert 0 < moved < 4 * w   # the test exercises both outcomes
    ds.close()
    ctx.close()


def test_stretch_step_errors_and_odd_ensemble():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    w, n, n_max = 7, 1 << 11, 3   # odd: halves of 3 and 4 walkers
    ds, d, wts, th, lo, hi, dt = setup(ctx, emri, w, n, n_max, 81)
    o = emri.opts(precision=emri.MIXED, n_max=n_max)
    theta = torch.tensor(th.T.copy(), device="cuda:0")
    lnp = torch.zeros(w, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, theta, o, lnp)
    u = torch.tensor(np.random.default_rng(5).random((3, w)), device="cuda:0")
    ctx.stretch_step(ds, theta, lnp, o, emri.stretch_cfg(FREE, lo, hi), u)
    torch.cuda.synchronize()
    chk = torch.zeros(w, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, theta, o, chk)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(chk.cpu().numpy(), lnp.cpu().numpy())
    for bad in (emri.stretch_cfg(FREE, lo, hi, a=1.0), emri.stretch_cfg([], lo, hi),
                emri.stretch_cfg(FREE, hi, lo)):
        with pytest.raises(emri.EmriError) as ei:
            ctx.stretch_step(ds, theta, lnp, o, bad, u)
        assert ei.value.code == emri.EINVAL
    with pytest.raises(emri.EmriError):
        ctx.stretch_step(ds, theta[:, :1].contiguous(), lnp[:1], o, emri.stretch_cfg(FREE, lo, hi), u)
    ds.close()
    ctx.close()
