"""Oracle of the affine-invariant ensemble step (stretch move).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): imported by
``tests/`` alone; the product package never imports it.

The paper samples its posterior with an affine-invariant ensemble sampler
(Sec. 1 and Sec. 3, "Posterior sampling": the emcee package, after Goodman
& Weare 2010, Commun. Appl. Math. Comput. Sci. 5, 65).  One ensemble step of
the parallel stretch move, written out plainly:

* the W walkers are split into two halves, S0 = [0, h) and S1 = [h, W) with
  h = floor(W/2); S0 is updated first against the current S1, then S1
  against the updated S0 (Goodman & Weare Sec. 5, the parallel variant);
* walker k of the active half draws a partner X_j from the other half,
  j = floor(u_partner[k] * |other half|);
* a stretch factor z with density g(z) ~ 1/sqrt(z) on [1/a, a], by inverse
  CDF of a uniform: z = ((a - 1) u_stretch[k] + 1)^2 / a;
* proposal Y = X_j + z (X_k - X_j) in the free coordinates (the others are
  copied from X_k);
* accept with probability min(1, z^(d-1) P(Y) / P(X_k)), d = number of free
  coordinates, i.e. accept iff ln u_accept[k] < (d - 1) ln z + lnP(Y) - lnP(X_k).

The uniforms are inputs (drawn by the caller), so the oracle and the GPU step
see the same random numbers.  lnP = lnL + ln prior with a flat prior on a
box (lo <= theta_p <= hi for every free p) and -inf outside it or where the
likelihood reports an invalid parameter point.
"""
from __future__ import annotations

import numpy as np

#: status bits of the likelihood that make a point invalid (bad parameters,
#: non-finite orbit)
INVALID = 2 | 4


def stretch_z(u, a: float):
    """Stretch factor of the uniform u in [0, 1): inverse CDF of g(z) ~ z^-1/2 on [1/a, a]."""
    t = (a - 1.0) * np.asarray(u, dtype=np.float64) + 1.0
    return t * t / a


def in_box(y, free, lo, hi) -> bool:
    return all(lo[p] <= y[p] <= hi[p] for p in free)


def halves_of(w: int):
    """The two halves S0 = [0, h), S1 = [h, W), h = floor(W/2)."""
    h = w // 2
    return [np.arange(0, h), np.arange(h, w)]


def stretch_block(x, lp, acc, margin, u, a: float, free, lo, hi, lnprob, s: int, k0: int, k1: int):
    """Update the walkers k0 <= k < k1 of half s (in place) against the whole
    other half, as one part of the half-step of ``stretch_step``: walker k
    uses only its own uniforms u[:, k] and the other half's positions, so the
    half-step over its walkers in any partition gives the same result."""
    w = x.shape[0]
    halves = halves_of(w)
    other = halves[1 - s]
    active = [k for k in halves[s] if k0 <= k < k1]
    nc = len(other)
    if not len(active) or not nc:
        return
    d = len(free)
    ys, zs = [], []
    for k in active:
        j = other[min(int(np.floor(u[0][k] * nc)), nc - 1)]
        z = float(stretch_z(u[1][k], a))
        y = x[k].copy()
        for p in free:
            y[p] = x[j][p] + z * (x[k][p] - x[j][p])
        ys.append(y)
        zs.append(z)
    ll, st = lnprob(np.array(ys))
    for i, k in enumerate(active):
        y = ys[i]
        if not in_box(y, free, lo, hi) or (int(st[i]) & INVALID) or not np.isfinite(ll[i]):
            continue
        margin[k] = (d - 1) * np.log(zs[i]) + ll[i] - lp[k] - np.log(u[2][k])
        if margin[k] > 0:
            x[k] = y
            lp[k] = ll[i]
            acc[k] = 1


def stretch_step(theta, lnp, u, a: float, free, lo, hi, lnprob):
    """One ensemble step.

    theta: [W][P] positions; lnp: [W] log-posterior of the positions;
    u: [3][W] uniforms (partner, stretch, accept) in [0, 1); free: indices of
    the free coordinates; lo, hi: [P] prior box; lnprob(Y[m][P]) -> (lnL[m],
    status[m]) evaluates the likelihood of m proposals at once.
    Returns new (theta, lnp, accepted[W], margin[W]); margin is
    (d-1) ln z + lnP(Y) - lnP(X) - ln u_accept (accept iff > 0), NaN where
    the proposal is rejected outright (outside the box or invalid).
    """
    x = np.array(theta, dtype=np.float64, copy=True)
    lp = np.array(lnp, dtype=np.float64, copy=True)
    w = x.shape[0]
    acc = np.zeros(w, dtype=np.int32)
    margin = np.full(w, np.nan)
    for s in (0, 1):
        stretch_block(x, lp, acc, margin, u, a, free, lo, hi, lnprob, s, 0, w)
    return x, lp, acc, margin
