"""Serving loop: continuous batching, alone-vs-mix determinism, admission.

Every failure here is caused on the host (an over-budget request, a full
queue, a poll that times out, an unknown ticket); nothing faults the GPU.
"""
import threading

import numpy as np
import pytest

from paper_2311_17174_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    dsets = {}
    for logn in (14, 15, 16):
        n = 1 << logn
        psd = I.psd_bc04(n)
        dsets[logn] = ctx.dataset(emri.grid(n, 15.0), I.noise_spectrum(900 + logn, psd, n), psd, 1e-4, 1 / 30.0)
    yield emri, ctx, dsets
    for d in dsets.values():
        d.close()
    ctx.close()


def requests(seed, count):
    g = np.random.default_rng(seed)
    out = []
    for k in range(count):
        logn = int(g.integers(14, 17))
        w = int(g.integers(8, 65))
        th = I.scatter_walkers(7000 + k, I.draw_sources(8000 + k, 1, 1 << logn)[0], w)
        prec = int(g.integers(0, 2))
        out.append((logn, th, prec))
    return out


def direct(emri, ctx, ds, th, prec):
    w = th.shape[0]
    lnl = torch.zeros(w, dtype=torch.float64, device="cuda:0")
    ctx.loglike_batch(ds, torch.tensor(th.T.copy(), device="cuda:0"), emri.opts(precision=prec, n_max=8), lnl)
    torch.cuda.synchronize()
    return lnl.cpu().numpy()


def test_serve_alone_vs_mix_bitwise(env):
    emri, ctx, dsets = env
    reqs = requests(1, 16)
    alone = [direct(emri, ctx, dsets[l], th, p) for (l, th, p) in reqs]
    ctx.serve_start(slots=4, queue_capacity=64)
    try:
        tickets = [None] * len(reqs)

        def submit(i):
            l, th, p = reqs[i]
            tickets[i] = ctx.serve_submit(dsets[l], th.T.copy(), emri.opts(precision=p, n_max=8))

        ths = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        slots_used = set()
        for i, (l, th, p) in enumerate(reqs):
            rc, lnl, st, stats = ctx.serve_poll(tickets[i], th.shape[0], timeout_us=-1)
            assert rc == emri.OK
            np.testing.assert_array_equal(lnl, alone[i])
            assert stats.arrival_ns <= stats.start_ns <= stats.done_ns
            slots_used.add(stats.slot)
        assert len(slots_used) > 1   # requests overlapped on several slots
    finally:
        ctx.serve_stop()


def test_serve_admission_and_errors(env):
    emri, ctx, dsets = env
    th = I.scatter_walkers(1, I.draw_sources(2, 1, 1 << 16)[0], 64)
    ctx.serve_start(slots=2, queue_capacity=2, budget_bytes=256 << 20)
    try:
        # a request larger than the serving budget is refused up front
        big = I.scatter_walkers(3, I.draw_sources(4, 1, 1 << 16)[0], 512)
        with pytest.raises(emri.EmriError) as ei:
            ctx.serve_submit(dsets[16], big.T.copy(), emri.opts(n_max=8))
        assert ei.value.code == emri.EBUDGET
        # unknown ticket
        with pytest.raises(emri.EmriError) as ei:
            ctx.serve_poll(987654321, 1, timeout_us=0)
        assert ei.value.code == emri.ENOTFOUND
        # queue capacity: submits beyond it get EAGAIN
        got, tickets = [], []
        for _ in range(8):
            try:
                tickets.append(ctx.serve_submit(dsets[16], th.T.copy(), emri.opts(n_max=8)))
            except emri.EmriError as e:
                got.append(e.code)
        assert emri.EAGAIN in got
        # a zero timeout on a fresh request reports ETIMEDOUT or completion, never an error
        t = tickets[-1]
        rc, _, _, _ = ctx.serve_poll(t, 64, timeout_us=0)
        assert rc in (emri.OK, emri.ETIMEDOUT)
        if rc == emri.ETIMEDOUT:
            rc, _, _, _ = ctx.serve_poll(t, 64, timeout_us=-1)
            assert rc == emri.OK
        for t2 in tickets[:-1]:
            assert ctx.serve_poll(t2, 64, timeout_us=-1)[0] == emri.OK
    finally:
        ctx.serve_stop()
    with pytest.raises(emri.EmriError) as ei:
        ctx.serve_submit(dsets[16], th.T.copy(), emri.opts(n_max=8))
    assert ei.value.code == emri.ENOTFOUND


def test_stop_while_pollers_wait_and_direct_calls_in_parallel(env):
    """Pollers blocked on their tickets while another thread stops serving
    get either their results or a clean error (never a crash); direct
    emri_loglike_batch calls on the same context meanwhile are unaffected."""
    emri, ctx, dsets = env
    reqs = requests(5, 12)
    ctx.serve_start(slots=2, queue_capacity=64)
    tickets = [ctx.serve_submit(dsets[l], th.T.copy(), emri.opts(precision=p, n_max=8)) for (l, th, p) in reqs]
    outcomes = [None] * len(reqs)

    def poll(i):
        try:
            rc, lnl, st, stats = ctx.serve_poll(tickets[i], reqs[i][1].shape[0], timeout_us=-1)
            outcomes[i] = ("ok", lnl)
        except emri.EmriError as e:
            outcomes[i] = ("err", e.code)

    ths = [threading.Thread(target=poll, args=(i,)) for i in range(len(reqs))]
    for t in ths:
        t.start()
    # a direct call on the same context while the loop runs
    l0, th0, p0 = reqs[0]
    alone = direct(emri, ctx, dsets[l0], th0, p0)
    ctx.serve_stop()
    for t in ths:
        t.join(timeout=120)
        assert not t.is_alive()
    for i, (kind, val) in enumerate(outcomes):
        if kind == "ok":
            l, th, p = reqs[i]
            np.testing.assert_array_equal(val, direct(emri, ctx, dsets[l], th, p))
        else:
            assert val == emri.ENOTFOUND   # never admitted before the stop
    assert outcomes[0][0] == "ok" or outcomes[0][1] == emri.ENOTFOUND
    np.testing.assert_array_equal(alone, direct(emri, ctx, dsets[l0], th0, p0))
    with pytest.raises(emri.EmriError) as ei:
        ctx.serve_poll(tickets[0], 1, timeout_us=0)
    assert ei.value.code == emri.ENOTFOUND


def test_pool_admission_backfill(env):
    """A serving pool that holds one large request and two small ones at a
    time, with large (FP64, 512 walkers) and small (mixed, 8 walkers)
    requests submitted alternately: every admitted request completes without
    a memory error, the large ones run one after another, a small request
    submitted behind a waiting large one is served before it, and every
    result equals the same request run alone."""
    emri, ctx, dsets = env
    o_l, o_s = emri.opts(precision=emri.FP64, n_max=8), emri.opts(precision=emri.MIXED, n_max=8)
    ds_l, ds_s = dsets[16], dsets[14]
    th_l = [I.scatter_walkers(40 + k, I.draw_sources(50 + k, 1, 1 << 16)[0], 512) for k in range(3)]
    th_s = [I.scatter_walkers(60 + k, I.draw_sources(70 + k, 1, 1 << 14)[0], 8) for k in range(6)]
    need_l = ctx.serve_request_bytes(ds_l, 512, o_l)
    need_s = ctx.serve_request_bytes(ds_s, 8, o_s)
    assert need_l > 4 * need_s
    order = [("L", 0), ("L", 1), ("S", 0), ("S", 1), ("L", 2), ("S", 2), ("S", 3), ("S", 4), ("S", 5)]
    alone = {(k, i): direct(emri, ctx, ds_l if k == "L" else ds_s, (th_l if k == "L" else th_s)[i],
                            emri.FP64 if k == "L" else emri.MIXED) for k, i in order}
    ctx.serve_start(slots=4, queue_capacity=64, budget_bytes=need_l + 2 * need_s + 4096)
    try:
        tickets = []
        for k, i in order:
            th = (th_l if k == "L" else th_s)[i]
            tickets.append(ctx.serve_submit(ds_l if k == "L" else ds_s, th.T.copy(), o_l if k == "L" else o_s))
        stats = {}
        for (k, i), t in zip(order, tickets):
            w = 512 if k == "L" else 8
            rc, lnl, st, s = ctx.serve_poll(t, w, timeout_us=-1)
            assert rc == emri.OK and s.status == emri.OK
            np.testing.assert_array_equal(lnl, alone[(k, i)])
            stats[(k, i)] = (s.arrival_ns, s.start_ns, s.done_ns)
    finally:
        ctx.serve_stop()
    # the pool holds one large request: each starts after the previous one is done
    assert stats[("L", 1)][1] >= stats[("L", 0)][2]
    assert stats[("L", 2)][1] >= stats[("L", 1)][2]
    # small requests submitted after the second large one passed it while it waited
    assert min(stats[("S", i)][1] for i in range(2)) < stats[("L", 1)][1]
