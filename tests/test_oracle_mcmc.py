"""Pins of the stretch-move oracle (oracle/mcmc.py) against what the
mathematics fixes, independent of the GPU path:

* the stretch factor's first two moments against the closed forms of the
  density g(z) ~ z^-1/2 on [1/a, a];
* a hand-worked 4-walker step (partners, the half ordering, the box);
* affine invariance: the step commutes with x -> A x + b;
* stationarity: sampling a correlated 4-D Gaussian reproduces its
  covariance (a dropped or wrong z^(d-1) factor fails this).
"""
import numpy as np
import pytest

from oracle import mcmc as M


def const_lnprob(ys):
    return np.zeros(len(ys)), np.zeros(len(ys), dtype=np.uint32)


@pytest.mark.parametrize("a", [1.5, 2.0, 3.0])
def test_stretch_factor_moments(a):
    u = (np.arange(2_000_000) + 0.5) / 2_000_000
    z = M.stretch_z(u, a)
    assert z.min() >= 1 / a and z.max() <= a
    s = np.sqrt(a) - 1 / np.sqrt(a)
    m1 = (a ** 1.5 - a ** -1.5) / (3 * s)
    m2 = (a ** 2.5 - a ** -2.5) / (5 * s)
    assert z.mean() == pytest.approx(m1, rel=1e-10)
    assert (z * z).mean() == pytest.approx(m2, rel=1e-10)


def test_worked_four_walker_step():
    # 1 free coordinate; halves {0, 1} then {2, 3}; lnP constant => every
    # in-box proposal is accepted (margin = -ln u > 0).
    x = np.zeros((4, 16))
    x[:, 0] = [0.0, 1.0, 2.0, 4.0]
    x[:, 5] = 7.25                       # a fixed coordinate
    u = np.array([[0.1, 0.9, 0.7, 0.2],  # partners: 0->2, 1->3, then 2->1', 3->0'
                  [0.0, 0.5, 0.0, 0.5],  # z = 1/2, 9/8, 1/2, 9/8
                  [0.5, 0.5, 0.5, 0.5]])
    lo, hi = np.full(16, -10.0), np.full(16, 10.0)
    xn, lp, acc, mg = M.stretch_step(x, np.zeros(4), u, 2.0, [0], lo, hi, const_lnprob)
    # walker 0: 2 + (1/2)(0 - 2) = 1;    walker 1: 4 + (9/8)(1 - 4) = 0.625
    # walker 2: 0.625 + (1/2)(2 - 0.625) = 1.3125 (partner already moved)
    # walker 3: 1 + (9/8)(4 - 1) = 4.375
    np.testing.assert_array_equal(xn[:, 0], [1.0, 0.625, 1.3125, 4.375])
    np.testing.assert_array_equal(acc, [1, 1, 1, 1])
    np.testing.assert_array_equal(xn[:, 5], 7.25)
    np.testing.assert_allclose(mg, -np.log(0.5))
    # a box that excludes walker 3's proposal keeps it in place
    hi[0] = 4.2
    xn, lp, acc, mg = M.stretch_step(x, np.zeros(4), u, 2.0, [0], lo, hi, const_lnprob)
    np.testing.assert_array_equal(xn[:, 0], [1.0, 0.625, 1.3125, 4.0])
    np.testing.assert_array_equal(acc, [1, 1, 1, 0])
    assert np.isnan(mg[3])
    # an invalid likelihood point is rejected as well
    def bad_lnprob(ys):
        return np.zeros(len(ys)), np.full(len(ys), 2, dtype=np.uint32)
    xn, _, acc, _ = M.stretch_step(x, np.zeros(4), u, 2.0, [0], lo, np.full(16, 10.0), bad_lnprob)
    np.testing.assert_array_equal(xn, x)
    assert not acc.any()


def gauss(cov):
    prec = np.linalg.inv(cov)

    def lnprob(ys):
        y = np.asarray(ys)[:, :cov.shape[0]]
        return -0.5 * np.einsum("ij,jk,ik->i", y, prec, y), np.zeros(len(y), dtype=np.uint32)
    return lnprob


def test_affine_invariance():
    g = np.random.default_rng(5)
    d = 3
    A = g.normal(size=(d, d)) + 3 * np.eye(d)
    b = g.normal(size=d)
    cov = np.array([[1.0, 0.3, 0.1], [0.3, 2.0, -0.4], [0.1, -0.4, 0.5]])
    base = gauss(cov)
    Ainv = np.linalg.inv(A)

    def moved(ys):
        y = np.asarray(ys).copy()
        y[:, :d] = (y[:, :d] - b) @ Ainv.T
        return base(y)

    W = 16
    x = np.zeros((W, 16))
    x[:, :d] = g.normal(size=(W, d))
    xt = x.copy()
    xt[:, :d] = x[:, :d] @ A.T + b
    lo, hi = np.full(16, -1e9), np.full(16, 1e9)
    lp = base(x)[0]
    lpt = moved(xt)[0]
    free = list(range(d))
    for step in range(5):
        u = g.random((3, W))
        x, lp, acc, mg = M.stretch_step(x, lp, u, 2.0, free, lo, hi, base)
        xt, lpt, acct, mgt = M.stretch_step(xt, lpt, u, 2.0, free, lo, hi, moved)
        assert np.all(np.abs(mg) > 1e-6)          # no near-ties in this seed
        np.testing.assert_array_equal(acc, acct)
        np.testing.assert_allclose(xt[:, :d], x[:, :d] @ A.T + b, rtol=1e-12, atol=1e-12)


def test_gaussian_target_is_stationary():
    g = np.random.default_rng(11)
    d = 4
    L = np.tril(g.normal(size=(d, d))) + 2 * np.eye(d)
    cov = L @ L.T
    lnprob = gauss(cov)
    W = 32
    x = np.zeros((W, 16))
    x[:, :d] = 0.1 * g.normal(size=(W, d))
    lp = lnprob(x)[0]
    lo, hi = np.full(16, -1e9), np.full(16, 1e9)
    free = list(range(d))
    samples = []
    for step in range(3000):
        x, lp, acc, _ = M.stretch_step(x, lp, g.random((3, W)), 2.0, free, lo, hi, lnprob)
        if step >= 600:
            samples.append(x[:, :d].copy())
    s = np.concatenate(samples)
    est = np.cov(s.T)
    ratio = np.diag(est) / np.diag(cov)
    assert np.all((ratio > 0.85) & (ratio < 1.15)), ratio
    assert np.linalg.norm(est - cov) / np.linalg.norm(cov) < 0.15
    assert np.all(np.abs(s.mean(0)) < 0.25 * np.sqrt(np.diag(cov)))
