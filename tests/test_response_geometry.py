"""Independent pin of the oracle's LISA response (paper Sec. 2: the detector
response of the Barack-Cutler AK model, channels h_I, h_II of Eq. (2)).

The oracle evaluates the response through angles: the detector-frame source
direction (theta_d, phi_d) from closed forms in the LISA orbital phase
phibar, the polarisation angle psi and the in-plane angle beta from atan2 of
vector products, and the antenna patterns F+, Fx as trigonometric polynomials
of those angles.  None of those formulas is used here.  The same channels are
built from explicit 3-vectors instead:

  * the detector frame from the constellation's geometry: the guiding centre
    at r = (cos phibar, sin phibar, 0) on the ecliptic, the constellation
    plane tilted by 60 degrees with its normal z_d = z/2 - (sqrt3/2) r
    leaning towards the Sun, the reference in-plane axis x0 along the line
    where that plane meets the ecliptic (z x z_d), y0 = z_d x x0, and the
    arms turning about z_d against the orbital motion (cartwheel phase
    2 pi t / T, zero at t = 0): x_d = cos(a) x0 - sin(a) y0,
    y_d = sin(a) x0 + cos(a) y0;
  * the two Michelson channels as the contractions of the strain tensor with
    the detector tensors sqrt3/2 * (x_d x_d - y_d y_d)/2 and
    sqrt3/2 * (x_d y_d + y_d x_d)/2 (a 60-degree interferometer is sqrt3/2
    times an L-shaped one; channel II is that L turned by 45 degrees);
  * the strain tensor as twice the transverse-traceless projection, onto the
    plane normal to N, of the orbit's quadrupole tensor
      M = -a (r1 r1 - r2 r2) - b (r1 r2 + r2 r1) + c (r1 r1 + r2 r2),
    a, b, c the Peters-Mathews harmonic sums of Eq. (2) (Bessel functions
    from scipy), r1 the pericentre direction -- at angle gamma~ from L x S
    about L -- and r2 = L x r1;
  * the Doppler phase from the projection of the guiding centre on N:
    Phi_D = Phi + 2 pi nu (R/c) N.r.

Mutations of the oracle's angle formulas are planted on the CPU, in a copy
of the oracle's own composition of its exposed geometry, antenna and
polarisation routines, and each is shown to break the agreement:
  * the two atan2 arguments of phi_d swapped;
  * the sign of the cross term of the antenna patterns flipped;
  * phibar -> -phibar.
"""
import numpy as np
import pytest
from scipy.special import jv

import oracle as O
from paper_2311_17174_gb300 import inputs as I

YEAR = 31557600.0          # LISA orbital period [s] (the oracle's constant)
AU_C = 499.004783836       # 1 AU / c [s]
H3 = 0.5 * np.sqrt(3.0)
ZHAT = np.array([0.0, 0.0, 1.0])


def unit(v):
    return v / np.linalg.norm(v)


def source_vectors(th, alpha):
    """N (source direction), S (spin direction) and L (orbital angular
    momentum: L = S cos(lam) + sin(lam) (e1 cos(alpha) + e2 sin(alpha)), with
    e1 along the projection of the ecliptic pole normal to S, e2 = S x e1)."""
    ths, phs, thk, phk, lam = th[I.I_THS], th[I.I_PHS], th[I.I_THK], th[I.I_PHK], th[I.I_LAM]
    N = np.array([np.sin(ths) * np.cos(phs), np.sin(ths) * np.sin(phs), np.cos(ths)])
    S = np.array([np.sin(thk) * np.cos(phk), np.sin(thk) * np.sin(phk), np.cos(thk)])
    e1 = unit(ZHAT - S * (S @ ZHAT))
    e2 = np.cross(S, e1)
    L = S * np.cos(lam) + np.sin(lam) * (e1 * np.cos(alpha) + e2 * np.sin(alpha))
    return N, S, L


def detector_frame(t):
    """(x_d, y_d, z_d, r) of the LISA constellation at time t (see the module
    docstring); r is the direction of the guiding centre from the Sun."""
    phib = 2 * np.pi * t / YEAR
    r = np.array([np.cos(phib), np.sin(phib), 0.0])
    zd = 0.5 * ZHAT - H3 * r
    x0 = unit(np.cross(ZHAT, zd))
    y0 = np.cross(zd, x0)
    a = 2 * np.pi * t / YEAR
    xd = np.cos(a) * x0 - np.sin(a) * y0
    yd = np.sin(a) * x0 + np.cos(a) * y0
    return xd, yd, zd, r


def harmonic_sums(n_max, e, amp, phi_cycles):
    """(a, b, c) = sum_n (a_n, b_n, c_n) of Eq. (2) at orbital phase Phi
    (cycles): a_n = -n A [J_{n-2} - 2e J_{n-1} + (2/n) J_n + 2e J_{n+1} - J_{n+2}] cos(n Phi),
    b_n = -n A sqrt(1-e^2) [J_{n-2} - 2 J_n + J_{n+2}] sin(n Phi),
    c_n = 2 A J_n cos(n Phi), all J at n e."""
    a = b = c = 0.0
    for n in range(1, n_max + 1):
        x = n * e
        j = {m: jv(m, x) for m in range(n - 2, n + 3)}
        ph = 2 * np.pi * ((n * phi_cycles) % 1.0)
        a += -n * amp * (j[n - 2] - 2 * e * j[n - 1] + (2.0 / n) * j[n] + 2 * e * j[n + 1] - j[n + 2]) * np.cos(ph)
        b += -n * amp * np.sqrt(1 - e * e) * (j[n - 2] - 2 * j[n] + j[n + 2]) * np.sin(ph)
        c += 2 * amp * j[n] * np.cos(ph)
    return a, b, c


def tensor_channels(th, t, alpha, phi_cycles, nu, gamma_t, e, amp, n_max, doppler=True):
    """h_I, h_II from the explicit detector and strain tensors."""
    N, S, L = source_vectors(th, alpha)
    xd, yd, _, r = detector_frame(t)
    phd = phi_cycles + (nu * AU_C * (N @ r) if doppler else 0.0)
    a, b, c = harmonic_sums(n_max, e, amp, phd)
    u1 = unit(np.cross(L, S))
    u2 = np.cross(L, u1)
    r1 = np.cos(gamma_t) * u1 + np.sin(gamma_t) * u2
    r2 = np.cross(L, r1)
    M = -a * (np.outer(r1, r1) - np.outer(r2, r2)) - b * (np.outer(r1, r2) + np.outer(r2, r1)) \
        + c * (np.outer(r1, r1) + np.outer(r2, r2))
    P = np.eye(3) - np.outer(N, N)
    PMP = P @ M @ P
    h = 2.0 * (PMP - 0.5 * P * np.trace(PMP))
    hI = H3 * 0.5 * (xd @ h @ xd - yd @ h @ yd)
    hII = H3 * 0.5 * (xd @ h @ yd + yd @ h @ xd)
    return hI, hII


# ------------------------------------------------ the oracle's composition
def antenna_mutated(theta_d, phi_d, psi):
    """orc_antenna with the sign of its cross term flipped (a planted mistake)."""
    ct = np.cos(theta_d)
    return np.array([0.5 * (1 + ct * ct) * np.cos(2 * phi_d) * np.cos(2 * psi) + ct * np.sin(2 * phi_d) * np.sin(2 * psi),
                     0.5 * (1 + ct * ct) * np.cos(2 * phi_d) * np.sin(2 * psi) - ct * np.sin(2 * phi_d) * np.cos(2 * psi)])


def oracle_channels(th, t, alpha, phi_cycles, nu, gamma_t, e, amp, n_max, mutate=None):
    """The oracle's per-sample response, composed from its exposed geometry,
    antenna-pattern and polarisation routines exactly as its waveform does;
    ``mutate`` plants one mistake in the angle formulas."""
    geo = O.geometry(th, -t if mutate == "phibar_sign" else t, alpha)
    c, psi, beta, thd, phid, dop = geo
    if mutate == "phibar_sign":      # only the Doppler delay keeps the true phibar
        dop = O.geometry(th, t, alpha)[5]
    if mutate == "atan2_swap":
        ths, phs = th[I.I_THS], th[I.I_PHS]
        phib = 2 * np.pi * t / YEAR
        phid = phib + np.arctan2(2 * np.sin(ths) * np.sin(phib - phs),
                                 np.sqrt(3.0) * np.cos(ths) + np.sin(ths) * np.cos(phib - phs))
    ant = antenna_mutated if mutate == "antenna_cross_sign" else O.antenna
    fI, fII = ant(thd, phid, psi), ant(thd, phid - np.pi / 4, psi)
    two_gamma = 2 * np.pi * ((2 * gamma_t / (2 * np.pi)) % 1.0) + 2 * beta
    hp, hx = O.polarizations(n_max, e, amp, phi_cycles + nu * dop, two_gamma, c)
    return H3 * (fI[0] * hp + fI[1] * hx), H3 * (fII[0] * hp + fII[1] * hx)


def _cases(count, seed):
    g = np.random.default_rng(seed)
    ths = I.draw_sources(seed, count, 1 << 16)
    for k in range(count):
        yield (ths[k], g.uniform(0, 3.2e7), g.uniform(0, 2 * np.pi), g.uniform(0, 1), g.uniform(1e-4, 1e-2),
               g.uniform(0, 2 * np.pi), g.uniform(0.0, 0.6), 1.0, int(g.integers(2, 12)))


def _rel(a, b):
    scale = max(abs(b[0]), abs(b[1]), 1e-300)
    return max(abs(a[0] - b[0]), abs(a[1] - b[1])) / scale


def test_response_equals_detector_and_strain_tensors():
    """120 random sources, times, alpha, phases, gamma~, e and n_max: the
    oracle's angle-based channels equal the tensor construction to 1e-12 of
    the larger channel."""
    worst = 0.0
    for case in _cases(120, 31):
        worst = max(worst, _rel(oracle_channels(*case), tensor_channels(*case)))
    assert worst < 1e-12, worst


@pytest.mark.parametrize("mutate", ["atan2_swap", "antenna_cross_sign", "phibar_sign"])
def test_planted_angle_mistakes_break_the_pin(mutate):
    """Each planted mistake in the oracle's angle formulas moves the channels
    by more than 1e-2 of their size on some of the cases."""
    worst = 0.0
    for case in _cases(40, 32):
        worst = max(worst, _rel(oracle_channels(*case, mutate=mutate), tensor_channels(*case)))
    assert worst > 1e-2, (mutate, worst)


def test_waveform_samples_equal_tensor_construction():
    """End to end: the oracle's waveform at sampled times (its own orbit,
    Doppler and amplitude x^(2/3) mu c) equals the tensor construction fed
    with the oracle's orbit state at those samples."""
    n, dt, n_max = 1 << 12, 15.0, 8
    ths = I.draw_sources(33, 4, n)
    idx = np.unique(np.r_[0, 1, np.random.default_rng(34).integers(0, n, 40), n - 1])
    gm_c3 = 1.32712440018e26 / 2.99792458e10 ** 3   # G M_sun / c^3 [s]
    worst = 0.0
    for th in ths:
        orb = O.orbit(th, n, dt)
        assert orb["n_valid"] == n
        hI, hII, st = O.waveform_sampled(th, n, dt, idx, O.Opts(n_max=n_max), nthreads=1)
        assert st[0] == 0
        for k, j in enumerate(idx):
            nu, e = orb["nu"][j], orb["e"][j]
            x = 2 * np.pi * nu * th[I.I_M] * gm_c3
            amp = x ** (2.0 / 3.0) * th[I.I_MU] * gm_c3 * 2.99792458e10
            got = tensor_channels(th, j * dt, orb["alpha"][j], orb["phi"][j] / (2 * np.pi), nu, orb["gamma"][j],
                                  e, amp, n_max)
            worst = max(worst, _rel((hI[0, k], hII[0, k]), got))
    assert worst < 1e-10, worst
