"""One ensemble spread over several ranks (paper Sec. 3, "Posterior
sampling": the walkers of a half of the parallel stretch move are
independent given the other half).

CPU (gloo, two ranks): the package's sharded step -- each rank moves its own
block of each half, then the blocks are all-gathered -- with the block update
taken from the oracle's stretch move and the oracle's likelihood, equals the
oracle's unsharded ensemble step bit for bit over two steps.

GPU: the library's block update (emri_stretch_half) over the blocks of two
ranks, run in turn on one GPU, equals emri_stretch_step bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2311_17174_gb300 import ensemble as E


@pytest.mark.parametrize("w,world", [(2, 1), (10, 2), (11, 3), (1024, 8), (7, 4)])
def test_shard_blocks_cover_each_half(w, world):
    h = w // 2
    for half, (s0, s1) in enumerate(((0, h), (h, w))):
        blocks = [E.shard_block(w, world, r, half) for r in range(world)]
        assert blocks[0][0] == s0 and blocks[-1][1] == s1
        for (a0, a1), (b0, _) in zip(blocks, blocks[1:]):
            assert a1 == b0 and a0 <= a1
        widths = [b - a for a, b in blocks]
        assert max(widths) - min(widths) <= 1


W, N, DT, NMAX = 10, 1 << 10, 15.0, 4
FREE = [0, 1, 2, 14]   # M, mu, spin, Xi_0


def _problem():
    """Deterministic small ensemble with the oracle's likelihood."""
    import oracle as O
    from paper_2311_17174_gb300 import inputs as I
    inj = I.draw_sources(91, 1, N)[0]
    theta0 = I.scatter_walkers(92, inj, W)
    psd = I.psd_bc04(N, DT)
    d, _, wts, _ = O.injection_data(inj, N, DT, psd, 93, O.Opts(n_max=NMAX), nthreads=1)

    def lnprob(ys):
        lnl, _, _, st = O.loglike(ys, N, DT, d, wts, O.Opts(n_max=NMAX), nthreads=1)
        return lnl, st

    lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
    for p in FREE:
        c = inj[p]
        lo[p], hi[p] = c * (1 - 1e-3), c * (1 + 1e-3)
    lo[2], hi[2] = 0.0, 1.0
    g = np.random.default_rng(94)
    us = [g.random((3, W)) for _ in range(2)]
    return theta0, lnprob(theta0)[0], us, lnprob, lo, hi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    from oracle import mcmc as M
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    theta0, lnp0, us, lnprob, lo, hi = _problem()
    theta = torch.tensor(theta0.T.copy())
    lnp = torch.tensor(lnp0)
    acc = torch.zeros(W, dtype=torch.int32)
    for u in us:
        def move(half, k0, k1):
            x, lp = theta.T.numpy().copy(), lnp.numpy().copy()
            a, mg = np.zeros(W, dtype=np.int32), np.full(W, np.nan)
            M.stretch_block(x, lp, a, mg, u, 2.0, FREE, lo, hi, lnprob, half, k0, k1)
            theta[:, k0:k1] = torch.from_numpy(x[k0:k1].T.copy())
            lnp[k0:k1] = torch.from_numpy(lp[k0:k1])
            acc[k0:k1] = torch.from_numpy(a[k0:k1])

        E.sharded_stretch_step(theta, lnp, acc, rank, world, move, E.dist_all_gather)
    q.put((rank, theta.numpy().copy(), lnp.numpy().copy(), acc.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_unsharded_oracle_step():
    import torch.multiprocessing as mp
    from oracle import mcmc as M
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    theta0, lnp0, us, lnprob, lo, hi = _problem()
    x, lp = theta0, lnp0
    for u in us:
        x, lp, acc, _ = M.stretch_step(x, lp, u, 2.0, FREE, lo, hi, lnprob)
    assert acc.sum() > 0   # the step moved some walkers
    for _, th, l, a in res:   # every replica holds the same ensemble
        np.testing.assert_array_equal(th, x.T)
        np.testing.assert_array_equal(l, lp)
        np.testing.assert_array_equal(a, acc)


@pytest.mark.gpu
def test_gpu_blocks_equal_the_ensemble_step():
    from paper_2311_17174_gb300 import emri, inputs as I
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    ctx = emri.Context(0)
    try:
        n, w = 1 << 14, 37
        inj = I.draw_sources(95, 1, n)[0]
        th = I.scatter_walkers(96, inj, w)
        psd = I.psd_bc04(n, 15.0)
        d, _, _, _ = O.injection_data(inj, n, 15.0, psd, 97, O.Opts(n_max=6))
        ds = ctx.dataset(emri.grid(n, 15.0), d, psd, 1e-4, 1 / 30.0)
        lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
        for p in FREE:
            lo[p], hi[p] = inj[p] * (1 - 1e-3), inj[p] * (1 + 1e-3)
        lo[2], hi[2] = 0.0, 1.0
        cfg = emri.stretch_cfg(FREE, lo, hi)
        o = emri.opts(precision=emri.FP64, n_max=6)
        u = torch.tensor(np.random.default_rng(98).random((3, w)), device="cuda")
        theta_a = torch.tensor(th.T.copy(), device="cuda")
        lnp_a = torch.zeros(w, dtype=torch.float64, device="cuda")
        ctx.loglike_batch(ds, theta_a, o, lnp_a)
        theta_b, lnp_b = theta_a.clone(), lnp_a.clone()
        acc_a = torch.zeros(w, dtype=torch.int32, device="cuda")
        acc_b = torch.full((w,), -1, dtype=torch.int32, device="cuda")
        ctx.stretch_step(ds, theta_a, lnp_a, o, cfg, u, acc_a)
        # two ranks' blocks of each half, in turn, on one device holding the whole ensemble
        for half in (0, 1):
            for r in range(2):
                k0, k1 = E.shard_block(w, 2, r, half)
                ctx.stretch_half(ds, theta_b, lnp_b, o, cfg, u, half, k0, k1, acc_b)
        torch.cuda.synchronize()
        assert torch.equal(theta_a, theta_b) and torch.equal(lnp_a, lnp_b) and torch.equal(acc_a, acc_b)
        assert int(acc_a.sum()) > 0
        # a block outside its half is refused
        with pytest.raises(emri.EmriError) as ei:
            ctx.stretch_half(ds, theta_b, lnp_b, o, cfg, u, 0, 10, w // 2 + 1, acc_b)
        assert ei.value.code == emri.EINVAL
        ds.close()
    finally:
        ctx.close()
