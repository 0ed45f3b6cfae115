"""The pipelined likelihood schedule (emri_ctx_set_pipeline): the walkers of
a call in groups whose orbits, waveforms and FFT passes run on three streams.

Each walker is computed by the same kernels on the same data whatever the
schedule, so lnL, <d|h>, <h|h> and the status words must equal the
sequential schedule's bit for bit: for ragged groups, for a call spread over
several waves of the series buffer (a later wave's groups reuse the buffer
that the previous wave's groups of a different size occupied), with the
frequency-dependent model, and inside the ensemble step.
"""
import numpy as np
import pytest

from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, DT, NMAX, W = 1 << 14, 15.0, 6, 37


def _setup(ctx, emri):
    psd = I.psd_bc04(N, DT)
    ds = ctx.dataset(emri.grid(N, DT), I.noise_spectrum(61, psd, N), psd, 1e-4, 1.0 / (2 * DT))
    th = I.scatter_walkers(62, I.draw_sources(63, 1, N)[0], W, rel=1e-3)
    return ds, torch.tensor(th.T.copy(), device="cuda:0")


def _run(ctx, ds, theta, o, fd=None):
    w = int(theta.shape[1])
    out = [torch.zeros(w, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    st = torch.zeros(w, dtype=torch.int32, device="cuda:0")
    if fd is None:
        ctx.loglike_batch(ds, theta, o, out[0], out[1], out[2], st)
    else:
        ctx.loglike_batch_fd(ds, theta, o, *fd, out[0], out[1], out[2], st)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out + [st]]


def _same(got, ref):
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_pipelined_groups_equal_sequential():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    ds, theta = _setup(ctx, emri)
    g = np.random.default_rng(64)
    coef = torch.tensor(np.concatenate([g.normal(0, 0.3, (W, 2)), g.normal(0, 0.05, (W, 1))], axis=1).T.copy(),
                        device="cuda:0")
    fd = (2, 1, 3e-3, coef)
    for prec in (emri.FP64, emri.MIXED):
        o = emri.opts(precision=prec, n_max=NMAX)
        ctx.set_pipeline(prec, 1)
        ref = _run(ctx, ds, theta, o)
        ref_fd = _run(ctx, ds, theta, o, fd)
        assert np.isfinite(ref[0]).all() and np.isfinite(ref_fd[0]).all()
        assert not np.array_equal(ref[0], ref_fd[0])
        # by size (one group at this size), ragged groups, one walker per
        # group, more groups than walkers
        for groups in (0, 2, 5, 8, 37, 64):
            ctx.set_pipeline(prec, groups)
            _same(_run(ctx, ds, theta, o), ref)
            _same(_run(ctx, ds, theta, o, fd), ref_fd)
        ctx.set_pipeline(prec, 1)
    for bad in ((emri.FP64, -1), (emri.MIXED, 65), (2, 4)):
        with pytest.raises(emri.EmriError) as ei:
            ctx.set_pipeline(*bad)
        assert ei.value.code == emri.EINVAL
    ds.close()
    ctx.close()


def test_pipelined_groups_over_several_waves(tmp_path):
    """Waves of 10 walkers (a plan read from an autotuner cache file): 37
    walkers in waves of 10, 10, 10 and 7, with groups of 4, 4, 2 and then
    3, 3, 1, so the last wave's groups straddle the previous wave's."""
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    ds, theta = _setup(ctx, emri)
    cache = tmp_path / "plans.jsonl"
    cache.write_text("".join(
        '{"n": %d, "n_max": %d, "precision": %d, "knot_spacing": 0, "wave": 10, "n2": 0}\n' % (N, NMAX, p)
        for p in (0, 1)))
    for prec in (emri.FP64, emri.MIXED):
        choice = ctx.autotune(emri.grid(N, DT), NMAX, prec, str(cache))
        assert choice["wave_walkers"] == 10
        o = emri.opts(precision=prec, n_max=NMAX)
        ctx.set_pipeline(prec, 1)
        ref = _run(ctx, ds, theta, o)
        for groups in (3, 4, 10):
            ctx.set_pipeline(prec, groups)
            _same(_run(ctx, ds, theta, o), ref)
    ds.close()
    ctx.close()


def test_pipelined_ensemble_step():
    """emri_stretch_step with pipelined likelihoods moves the ensemble
    exactly as with the sequential schedule (same uniforms)."""
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    ds, theta0 = _setup(ctx, emri)
    free = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]
    x0 = theta0.cpu().numpy().T
    lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
    for p in free:
        lo[p], hi[p] = x0[:, p].min() * (1 - 1e-3), x0[:, p].max() * (1 + 1e-3)
    cfg = emri.stretch_cfg(free, lo, hi)
    u = torch.tensor(np.random.default_rng(65).random((3, W)), device="cuda:0")
    res = {}
    for groups in (1, 6):
        ctx.set_pipeline(emri.MIXED, groups)
        o = emri.opts(precision=emri.MIXED, n_max=NMAX)
        theta = theta0.clone()
        lnp = torch.zeros(W, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch(ds, theta, o, lnp)
        acc = torch.zeros(W, dtype=torch.int32, device="cuda:0")
        ctx.stretch_step(ds, theta, lnp, o, cfg, u, acc)
        torch.cuda.synchronize()
        res[groups] = (theta.cpu().numpy(), lnp.cpu().numpy(), acc.cpu().numpy())
    for a, b in zip(res[1], res[6]):
        np.testing.assert_array_equal(a, b)
    ds.close()
    ctx.close()
