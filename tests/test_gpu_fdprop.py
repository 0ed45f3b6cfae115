"""Frequency-dependent propagation (emri_loglike_batch_fd) against the
oracle's orc_loglike_fd: FP64 lnL within 1e-9 (|<d|h>| + <h|h>/2), <h|h>
within 2e-9 relative, mixed |dlnL| <= 1e-2, with coefficients that put the
extra GW-speed phase at up to ~1e14 cycles (exact mod 1 on both sides), and
zero coefficients reproducing emri_loglike_batch."""
import numpy as np
import pytest

import oracle as O
from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fdprop_matches_oracle():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    n, dt, nm = 1 << 14, 15.0, 6
    inj = I.draw_sources(91, 1, n)[0]
    psd = I.psd_bc04(n, dt)
    d, inj2, w, _ = O.injection_data(inj, n, dt, psd, 92, O.Opts(n_max=nm), snr=40.0)
    th = I.scatter_walkers(93, inj2, 12)
    ds = ctx.dataset(emri.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
    g = np.random.default_rng(94)
    qm, qt, fstar = 2, 3, 3e-3
    coef = np.concatenate([g.normal(0, 0.3, (12, qm)), g.normal(0, 0.05, (12, qt))], axis=1)
    ref, dh_o, hh_o, st_o = O.loglike_fd(th, n, dt, d, w, qm, qt, fstar, coef, O.Opts(n_max=nm))
    theta = torch.tensor(th.T.copy(), device="cuda:0")
    cdev = torch.tensor(coef.T.copy(), device="cuda:0")
    out = {}
    for prec in (0, 1):
        lnl, dh, hh = (torch.zeros(12, dtype=torch.float64, device="cuda:0") for _ in range(3))
        ctx.loglike_batch_fd(ds, theta, emri.opts(precision=prec, n_max=nm), qm, qt, fstar, cdev, lnl, dh, hh)
        torch.cuda.synchronize()
        out[prec] = [x.cpu().numpy() for x in (lnl, dh, hh)]
    dgw = np.array([O.prologue(t, n, dt)[2] for t in th])
    tol = 1e-9 * (np.abs(dh_o / dgw) + 0.5 * hh_o / dgw ** 2)
    assert np.all(np.abs(out[0][0] - ref) <= tol), (np.abs(out[0][0] - ref) / tol).max()
    np.testing.assert_allclose(out[0][2], hh_o, rtol=2e-9)
    assert np.max(np.abs(out[1][0] - ref)) <= 1e-2
    # the model changes the answer (the test is not vacuous)
    base = torch.zeros(12, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, theta, emri.opts(n_max=nm), base)
    torch.cuda.synchronize()
    assert np.min(np.abs(base.cpu().numpy() - ref)) > 1e-3
    # zero coefficients: the standard likelihood
    zero = torch.zeros((qm + qt, 12), dtype=torch.float64, device="cuda:0")
    lz = torch.zeros(12, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch_fd(ds, theta, emri.opts(n_max=nm), qm, qt, fstar, zero, lz)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lz.cpu().numpy(), base.cpu().numpy(), rtol=1e-14)
    for bad in ((4, 0, fstar), (0, -1, fstar), (1, 1, 0.0)):
        with pytest.raises(emri.EmriError) as ei:
            ctx.loglike_batch_fd(ds, theta, emri.opts(n_max=nm), bad[0], bad[1], bad[2], cdev, lz)
        assert ei.value.code == emri.EINVAL
    ds.close()
    ctx.close()


def test_fdprop_in_multi_chain_graph_and_serving():
    """The frequency-dependent model through the uneven-batching graph (one
    chain with it, one without) and through the serving loop: each result
    equals emri_loglike_batch_fd (or emri_loglike_batch) on the same walkers,
    bit for bit, in both precisions."""
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    try:
        n, dt, nm = 1 << 14, 15.0, 6
        inj = I.draw_sources(95, 1, n)[0]
        psd = I.psd_bc04(n, dt)
        d, inj2, _, _ = O.injection_data(inj, n, dt, psd, 96, O.Opts(n_max=nm), snr=40.0)
        ds = ctx.dataset(emri.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
        g = np.random.default_rng(97)
        qm, qt, fstar = 2, 1, 3e-3
        for prec in (0, 1):
            o = emri.opts(precision=prec, n_max=nm)
            ths = [I.scatter_walkers(98 + k, inj2, w) for k, w in enumerate((9, 14))]
            coef = np.concatenate([g.normal(0, 0.3, (9, qm)), g.normal(0, 0.05, (9, qt))], axis=1).T.copy()
            theta = [torch.tensor(t.T.copy(), device="cuda:0") for t in ths]
            cdev = torch.tensor(coef, device="cuda:0")
            alone = [torch.zeros(t.shape[0], dtype=torch.float64, device="cuda:0") for t in ths]
            ctx.loglike_batch_fd(ds, theta[0], o, qm, qt, fstar, cdev, alone[0])
            ctx.loglike_batch(ds, theta[1], o, alone[1])
            outs = [torch.zeros(t.shape[0], dtype=torch.float64, device="cuda:0") for t in ths]
            items = [(ds, theta[0], o, outs[0], None, None, None, (qm, qt, fstar, cdev)),
                     (ds, theta[1], o, outs[1], None, None, None)]
            ctx.loglike_multi(items)
            ctx.loglike_multi(items)   # the replayed graph
            torch.cuda.synchronize()
            for a, b in zip(alone, outs):
                assert torch.equal(a, b)
            ctx.serve_start(slots=2, queue_capacity=8, budget_bytes=1 << 30)
            try:
                t0 = ctx.serve_submit_fd(ds, ths[0].T.copy(), o, qm, qt, fstar, coef)
                t1 = ctx.serve_submit(ds, ths[1].T.copy(), o)
                rc, l0, _, _ = ctx.serve_poll(t0, 9)
                rc1, l1, _, _ = ctx.serve_poll(t1, 14)
            finally:
                ctx.serve_stop()
            assert rc == emri.OK and rc1 == emri.OK
            np.testing.assert_array_equal(l0, alone[0].cpu().numpy())
            np.testing.assert_array_equal(l1, alone[1].cpu().numpy())
        ds.close()
    finally:
        ctx.close()


def test_fdprop_in_the_ensemble_step():
    """emri_stretch_step_fd with a fixed model per walker: after a step, the
    stored log-posterior of every walker (moved or not) is emri_loglike_batch_fd
    at its new position with its own coefficients, bit for bit; the step
    moves walkers, and the model changes its outcome."""
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    try:
        n, dt, nm, w = 1 << 14, 15.0, 6, 24
        inj = I.draw_sources(101, 1, n)[0]
        psd = I.psd_bc04(n, dt)
        d, inj2, _, _ = O.injection_data(inj, n, dt, psd, 102, O.Opts(n_max=nm), snr=40.0)
        ds = ctx.dataset(emri.grid(n, dt), d, psd, 1e-4, 1.0 / (2 * dt))
        th = I.scatter_walkers(103, inj2, w)
        g = np.random.default_rng(104)
        qm, qt, fstar = 1, 1, 3e-3
        coef = torch.tensor(np.concatenate([g.normal(0, 0.3, (1, w)), g.normal(0, 0.05, (1, w))]), device="cuda:0")
        free = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]
        lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
        for p in free:
            lo[p], hi[p] = inj2[p] * (1 - 1e-3), inj2[p] * (1 + 1e-3)
        lo[I.I_SPIN], hi[I.I_SPIN] = 0.0, 1.0
        cfg = emri.stretch_cfg(free, lo, hi)
        o = emri.opts(precision=emri.FP64, n_max=nm)
        u = torch.tensor(g.random((3, w)), device="cuda:0")
        theta = torch.tensor(th.T.copy(), device="cuda:0")
        lnp = torch.zeros(w, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch_fd(ds, theta, o, qm, qt, fstar, coef, lnp)
        theta_b, lnp_b = theta.clone(), torch.zeros(w, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch(ds, theta_b, o, lnp_b)
        acc = torch.zeros(w, dtype=torch.int32, device="cuda:0")
        ctx.stretch_step_fd(ds, theta, lnp, o, cfg, qm, qt, fstar, coef, u, acc)
        acc_b = torch.zeros(w, dtype=torch.int32, device="cuda:0")
        ctx.stretch_step(ds, theta_b, lnp_b, o, cfg, u, acc_b)
        again = torch.zeros(w, dtype=torch.float64, device="cuda:0")
        ctx.loglike_batch_fd(ds, theta, o, qm, qt, fstar, coef, again)
        torch.cuda.synchronize()
        assert int(acc.sum()) > 0
        assert torch.equal(again, lnp)
        assert not torch.equal(lnp, lnp_b)
        ds.close()
    finally:
        ctx.close()
