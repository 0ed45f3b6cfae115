"""The waveform kernels evaluate the LISA response of Sec. 2 (Eq. 2 with the
Barack-Cutler antenna patterns) in a fixed polarisation basis of the sky plane
instead of through the angles psi and beta.  These CPU tests pin that
reformulation to the oracle's angle-based response:

  * h_I, h_II from the fixed-basis form equal the oracle's (geometry, antenna
    patterns, polarisations) to rounding, for random sources, times, alpha,
    gamma~ and harmonic sums;
  * the per-tile cubic of the four fixed-basis patterns (nodes at tile
    offsets 0, 256/3, 512/3, 256) stays within 2e-12 of the exact patterns up
    to the 64 s sample interval where the FP64 kernel switches to exact
    per-sample patterns, and within 1e-7 up to the mixed kernel's 1024 s.
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_17174_gb300 import inputs as I

H3 = 0.5 * np.sqrt(3.0)
YEAR = 31557600.0


def basis(th):
    ths, phs, thk, phk, lam = th[I.I_THS], th[I.I_PHS], th[I.I_THK], th[I.I_PHK], th[I.I_LAM]
    S = np.array([np.sin(thk) * np.cos(phk), np.sin(thk) * np.sin(phk), np.cos(thk)])
    e1 = (np.array([0.0, 0.0, 1.0]) - S * np.cos(thk)) / np.sin(thk)
    e2 = np.cross(S, e1)
    P = np.array([-np.sin(phs), np.cos(phs), 0.0])
    Q = np.array([np.cos(phs) * np.cos(ths), np.sin(phs) * np.cos(ths), -np.sin(ths)])
    return S, e1, e2, P, Q, np.cos(lam), np.sin(lam)


def double_angle(x, y):
    r = x * x + y * y
    return (x * x - y * y) / r, 2 * x * y / r


def patterns(th, phibar):
    """sqrt3/2 (F+_I, Fx_I, F+_II, Fx_II) at the polarisation angle of P."""
    cts, sts = np.cos(th[I.I_THS]), np.sin(th[I.I_THS])
    cps, sps = np.cos(th[I.I_PHS]), np.sin(th[I.I_PHS])
    cb, sb = np.cos(phibar), np.sin(phibar)
    cdp, sdp = cb * cps + sb * sps, sb * cps - cb * sps
    ct = 0.5 * cts - H3 * sts * cdp
    c2x, s2x = double_angle(2 * sts * sdp, np.sqrt(3.0) * cts + sts * cdp)
    c2p, s2p = double_angle(H3 * sdp, H3 * cts * cdp + 0.5 * sts)
    c2b, s2b = cb * cb - sb * sb, 2 * sb * cb
    c2f, s2f = c2b * c2x - s2b * s2x, s2b * c2x + c2b * s2x
    q = 0.5 * (1 + ct * ct)
    return H3 * np.array([q * c2f * c2p - ct * s2f * s2p, q * c2f * s2p + ct * s2f * c2p,
                          q * s2f * c2p + ct * c2f * s2p, q * s2f * s2p - ct * c2f * c2p])


def fixed_basis_channels(th, t, alpha, gamma_t, Cs, Ss, Rs):
    S, e1, e2, P, Q, cl, sl = basis(th)
    ca, sa = np.cos(alpha), np.sin(alpha)
    z1 = (sa * P @ e1 - ca * P @ e2) + 1j * (sa * Q @ e1 - ca * Q @ e2)
    z2 = (cl * (ca * P @ e1 + sa * P @ e2) - sl * P @ S) + 1j * (cl * (ca * Q @ e1 + sa * Q @ e2) - sl * Q @ S)
    c2g, s2g = np.cos(2 * gamma_t), np.sin(2 * gamma_t)
    X, Y = Cs * c2g - Ss * s2g, Cs * s2g + Ss * c2g
    H = (Rs + X) * z1 * z1 + (Rs - X) * z2 * z2 + 2 * Y * z1 * z2
    F = patterns(th, 2 * np.pi * t / YEAR)
    return F[0] * H.real + F[1] * H.imag, F[2] * H.real + F[3] * H.imag


def oracle_channels(th, t, alpha, gamma_t, A, B, C):
    """The oracle's response with harmonic sums A = sum a_n cos, B = sum b_n
    sin, C = sum c_n cos (the brackets of its polarisations)."""
    c, psi, beta, thd, phid, _ = O.geometry(th, t, alpha)
    fI, fII = O.antenna(thd, phid, psi), O.antenna(thd, phid - np.pi / 4, psi)
    g2 = 2 * gamma_t + 2 * beta
    hp = -(1 + c * c) * (A * np.cos(g2) - B * np.sin(g2)) + (1 - c * c) * C
    hx = 2 * c * (B * np.cos(g2) + A * np.sin(g2))
    return H3 * (fI[0] * hp + fI[1] * hx), H3 * (fII[0] * hp + fII[1] * hx)


def test_fixed_basis_response_equals_angle_form():
    g = np.random.default_rng(11)
    ths = I.draw_sources(12, 24, 1 << 16)
    ths[0, I.I_LAM] = 1e-6          # L nearly along S
    ths[1, I.I_THS] = 0.02          # source near the ecliptic pole
    ths[2, I.I_THK] = np.pi - 1e-3  # spin nearly antiparallel to z
    worst = 0.0
    for th in ths:
        for _ in range(25):
            t, al, gt = g.uniform(0, 3.2e7), g.uniform(0, 2 * np.pi), g.uniform(0, 2 * np.pi)
            A, B, C = g.normal(size=3)
            ref = oracle_channels(th, t, al, gt, A, B, C)
            # the kernels' sums are Cs = -A, Ss = -B, Rs = C (amplitude signs folded in)
            got = fixed_basis_channels(th, t, al, gt, -A, -B, C)
            worst = max(worst, max(abs(got[0] - ref[0]), abs(got[1] - ref[1])) / (abs(A) + abs(B) + abs(C)))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("dt,bound", [(15.0, 1e-13), (64.0, 2e-12), (1024.0, 1e-7)])
def test_pattern_tile_cubic(dt, bound):
    g = np.random.default_rng(12)
    ths = I.draw_sources(13, 16, 1 << 16)
    worst = 0.0
    for th in ths:
        for _ in range(10):
            t0 = g.uniform(0, 3.2e7)
            y = np.array([patterns(th, 2 * np.pi * (t0 + 256 * dt * q / 3) / YEAR) for q in range(4)])
            d1 = y[1] - y[0]
            d2 = (y[2] - y[1]) - d1
            d3 = ((y[3] - y[2]) - (y[2] - y[1])) - d2
            c = [y[0], 3 * (d1 - 0.5 * d2 + d3 / 3), 4.5 * (d2 - d3), 4.5 * d3]
            for so in np.linspace(0, 255 / 256, 18):
                exact = patterns(th, 2 * np.pi * (t0 + 256 * dt * so) / YEAR)
                fit = ((c[3] * so + c[2]) * so + c[1]) * so + c[0]
                worst = max(worst, np.abs(fit - exact).max())
    assert worst < bound, worst
