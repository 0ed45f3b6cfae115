"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks one oracle function against something other than itself: a
library special function, a closed form, an invariant of the equations, a
brute-force definition or high-precision quadrature.  A plausible slip (a
dropped term, a wrong sign or index, a transposed operand) in the oracle makes
at least one of them fail.  No GPU needed.
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
from paper_2311_17174_gb300 import inputs as I

C_CGS = 2.99792458e10
GM_SUN = 1.32712440018e26
MPC = 3.0856775814913673e24
TSUN = GM_SUN / C_CGS ** 3


def theta_base(**kw):
    t = np.zeros(16)
    t[[I.I_M, I.I_MU, I.I_SPIN, I.I_E0, I.I_NU0]] = [1e6, 10.0, 0.0, 0.0, 1e-3]
    t[[I.I_THS, I.I_PHS, I.I_THK, I.I_PHK, I.I_LAM, I.I_Z, I.I_XI0]] = [0.7, 1.0, 0.3, 2.0, 0.5, 0.5, 1.0]
    names = dict(M=I.I_M, mu=I.I_MU, spin=I.I_SPIN, e0=I.I_E0, nu0=I.I_NU0, phi0=I.I_PHI0,
                 gam0=I.I_GAM0, alp0=I.I_ALP0, ths=I.I_THS, phs=I.I_PHS, thk=I.I_THK, phk=I.I_PHK,
                 lam=I.I_LAM, z=I.I_Z, xi0=I.I_XI0, alpt=I.I_ALPT)
    for k, v in kw.items():
        t[names[k]] = v
    return t


# ------------------------------------------------------------------ Bessel
def test_bessel_matches_scipy(oracle_mod):
    # the oracle evaluates J_m(n e) with m >= n - 2 and e <= 0.6: x <= 0.6 (|m| + 2)
    for n in range(-2, 33):
        for x in np.linspace(0.0, 0.6 * (abs(n) + 2), 9):
            ref = sp.jv(n, x)
            got = O.bessel_j(n, x)
            assert abs(got - ref) <= 3e-15 * max(1.0, abs(ref)) + 1e-300, (n, x, got, ref)


def test_bessel_neumann_sum(oracle_mod):
    # J_0(x)^2 + 2 sum_{n>=1} J_n(x)^2 = 1
    for x in (0.3, 2.0, 7.5):
        s = O.bessel_j(0, x) ** 2 + 2 * sum(O.bessel_j(n, x) ** 2 for n in range(1, 60))
        assert abs(s - 1.0) < 1e-14


def test_bessel_negative_order(oracle_mod):
    for m in range(0, 6):
        assert O.bessel_j(-m, 1.3) == pytest.approx((-1) ** m * O.bessel_j(m, 1.3), rel=1e-15)


# ------------------------------------------------- Peters-Mathews brackets
def test_brackets_e0_only_n2(oracle_mod):
    for n in range(1, 12):
        pa, pb, pc = O.pm_brackets(n, 0.0)
        if n == 2:
            assert (pa, pb, pc) == (1.0, 1.0, 0.0)
        else:
            assert pa == 0.0 and pb == 0.0 and pc == 0.0


@pytest.mark.parametrize("e", [0.05, 0.2, 0.4, 0.6])
def test_peters_mathews_power_sum_rule(oracle_mod, e):
    # sum_n g(n,e) = (1 + 73 e^2/24 + 37 e^4/96)(1 - e^2)^(-7/2)   (Peters & Mathews 1963)
    tot = 0.0
    for n in range(1, 160):
        pa, pb, pc = O.pm_brackets(n, e)
        tot += n ** 4 / 32.0 * (pa ** 2 + (1 - e * e) * pb ** 2 + 4.0 / (3 * n * n) * pc ** 2)
    ref = (1 + 73 / 24 * e ** 2 + 37 / 96 * e ** 4) * (1 - e * e) ** -3.5
    assert tot == pytest.approx(ref, rel=1e-11)


def test_polarizations_e0_closed_form(oracle_mod):
    # e = 0: only n = 2 survives, h+ = 2A(1+c^2) cos(2Phi + 2g), hx = -4Ac sin(2Phi + 2g)
    g = np.random.default_rng(0)
    for _ in range(20):
        amp, ph, tg, c = g.uniform(0.1, 3), g.uniform(0, 1e4), g.uniform(-7, 7), g.uniform(-1, 1)
        hp, hx = O.polarizations(12, 0.0, amp, ph, tg, c)
        arg = 4 * np.pi * (ph % 1.0) + tg
        assert hp == pytest.approx(2 * amp * (1 + c * c) * np.cos(arg), abs=1e-12 * amp)
        assert hx == pytest.approx(-4 * amp * c * np.sin(arg), abs=1e-12 * amp)


def test_polarizations_face_on_circular_power(oracle_mod):
    # c = 1 (face-on), 2g = 0: h+ = sum 2nA pa cos(n Phi), hx = -sum 2nA sqrt(1-e^2) pb sin(n Phi),
    # so the orbit average of h+^2 + hx^2 is sum_n 4 n^2 A^2 [pa^2 + (1-e^2) pb^2] / 2.
    e, amp, n_max = 0.3, 1.0, 3
    phis = np.linspace(0, 1, 4096, endpoint=False)
    p = np.array([O.polarizations(n_max, e, amp, ph, 0.0, 1.0) for ph in phis])
    mean_pow = np.mean(p[:, 0] ** 2 + p[:, 1] ** 2)
    ref = 0.0
    for n in range(1, n_max + 1):
        pa, pb, _ = O.pm_brackets(n, e)
        ref += 4 * (n * amp) ** 2 * (pa ** 2 + (1 - e * e) * pb ** 2) / 2
    assert mean_pow == pytest.approx(ref, rel=1e-12)


# -------------------------------------------------------------------- LSO
def test_nu_lso_schwarzschild_isco(oracle_mod):
    # e = 0: orbital frequency at r = 6M, Kepler: c^3 / (2 pi 6^(3/2) G M)
    assert O.nu_lso(1.0, 0.0) == pytest.approx(1.0 / (2 * np.pi * 6 ** 1.5 * TSUN), rel=1e-15)
    assert O.nu_lso(1.0, 0.0) == pytest.approx(2198.6, abs=0.1)  # textbook 4.4 kHz GW / 2


@pytest.mark.parametrize("e", [0.1, 0.3, 0.6])
def test_nu_lso_separatrix(oracle_mod, e):
    # Schwarzschild separatrix p = 6 + 2e; semi-major axis a = p/(1-e^2); nu = a^(-3/2)/(2 pi M)
    p = 6 + 2 * e
    a = p / (1 - e * e)
    assert O.nu_lso(1e6, e) == pytest.approx(a ** -1.5 / (2 * np.pi * 1e6 * TSUN), rel=1e-14)


# ---------------------------------------------------------------- AK orbit
def test_newtonian_chirp_closed_form(oracle_mod):
    # pn_terms = 0, e = 0: nu(t) = nu0 (1 - t/tau)^(-3/8), tau = (5/256) M (M/mu) (2 pi M nu0)^(-8/3)
    th = theta_base(M=1e6, mu=10.0, e0=0.0, nu0=1e-3, spin=0.0)
    n, dt = 20000, 15.0
    orb = O.orbit(th, n, dt, O.Opts(pn_terms=0))
    m_s, mu_s = 1e6 * TSUN, 10.0 * TSUN
    tau = 5.0 / 256.0 * m_s * (m_s / mu_s) * (2 * np.pi * m_s * 1e-3) ** (-8.0 / 3.0)
    t = np.arange(n) * dt
    nu_ref = 1e-3 * (1 - t / tau) ** (-3.0 / 8.0)
    phi_ref = 2 * np.pi * 1e-3 * tau * 8.0 / 5.0 * (1 - (1 - t / tau) ** (5.0 / 8.0))
    assert np.max(np.abs(orb["nu"] / nu_ref - 1)) < 1e-13
    assert np.max(np.abs(orb["phi"] - phi_ref)) < 1e-9
    assert np.all(orb["e"] == 0.0)


def test_peters_eccentric_invariant(oracle_mod):
    # Newtonian radiation reaction: a(e) = c0 e^(12/19) (1-e^2)^-1 (1 + 121 e^2/304)^(870/2299)
    # (Peters 1964) and nu ~ a^(-3/2): nu * [a(e)/c0]^(3/2) is constant along the orbit.
    th = theta_base(M=5e5, mu=20.0, e0=0.35, nu0=2e-3, spin=0.0)
    orb = O.orbit(th, 200000, 15.0, O.Opts(pn_terms=0))
    e, nu = orb["e"], orb["nu"]
    a_e = e ** (12 / 19) / (1 - e * e) * (1 + 121 / 304 * e * e) ** (870 / 2299)
    inv = nu * a_e ** 1.5
    assert e[-1] < e[0] - 1e-3
    assert np.max(np.abs(inv / inv[0] - 1)) < 1e-12


def test_periastron_advance_leading_order(oracle_mod):
    # textbook 1PN periastron advance per orbit 6 pi M/(a(1-e^2)) -> rate 3 x^(2/3)/(1-e^2) * 2 pi nu
    th = theta_base(M=1e6, mu=10.0, spin=0.0)
    for e in (0.0, 0.3):
        nu = 1e-9 / (2 * np.pi * 1e6 * TSUN)        # x = 1e-9
        r = O.rhs(th, nu, e, 1)
        x23 = 1e-9 ** (2 / 3)
        lead = 3 * x23 / (1 - e * e) * 2 * np.pi * nu
        assert r[3] / lead == pytest.approx(1.0, abs=1e-4)
        assert r[0] == pytest.approx(2 * np.pi * nu, rel=1e-15)


def test_nu_dot_1pn_circular_from_chirp_and_periastron_advance(oracle_mod):
    # The AK frequency nu is the radial (anomalistic) one.  For a test mass on
    # a circular orbit the textbook 1PN chirp of the azimuthal frequency is
    #   d w_phi/dt ∝ w_phi^(11/3) (1 - (743/336) x),
    # and the 1PN periastron advance relates the two, w_phi = w_r (1 + 3 x),
    # x ∝ w^(2/3).  Then d w_r/dt = d w_phi/dt (1 - 3x - 2x) and
    # w_phi^(11/3) = w_r^(11/3) (1 + 11 x), so at 1PN
    #   d nu/dt ∝ nu^(11/3) (1 + (11 - 5 - 743/336) x).
    # The ratio of the full to the Newtonian rate at e = 0, spin 0 must be that.
    th = theta_base(M=1e6, mu=10.0, spin=0.0)
    for x in (1e-4, 1e-3, 1e-2):
        nu = x ** 1.5 / (2 * np.pi * 1e6 * TSUN)
        full = O.rhs(th, nu, 0.0, 1)[1]
        newt = O.rhs(th, nu, 0.0, 0)[1]
        assert full / newt == pytest.approx(1 + (6 - 743 / 336) * x, rel=1e-12)


def test_periastron_advance_2pn_circular_schwarzschild(oracle_mod):
    # Test mass on a circular Schwarzschild orbit: w_r = w_phi sqrt(1 - 6 x_phi)
    # exactly (x_phi = (M w_phi)^(2/3) = M/r), so the advance per radial period,
    # k = w_phi/w_r - 1, is known in closed form; in the radial variable
    # x = (M w_r)^(2/3) it expands as 3 x (1 + 6.5 x + O(x^2)).  The oracle's
    # dgamma~/dt / (2 pi nu) at e = 0, spin 0 must carry that 2PN coefficient.
    def k_exact(xr):
        xp = xr
        for _ in range(200):
            xp = xr * (1 - 6 * xp) ** (-1 / 3)
        return (1 - 6 * xp) ** -0.5 - 1
    th = theta_base(M=1e6, mu=10.0, spin=0.0)
    for x in (1e-5, 1e-4, 1e-3):
        nu = x ** 1.5 / (2 * np.pi * 1e6 * TSUN)
        k_or = O.rhs(th, nu, 0.0, 1)[3] / (2 * np.pi * nu)
        coef_or = (k_or / (3 * x) - 1) / x
        coef_ex = (k_exact(x) / (3 * x) - 1) / x
        assert abs(coef_or - coef_ex) < 60 * x, (x, coef_or, coef_ex)


def test_lense_thirring_rates(oracle_mod):
    # Lense-Thirring precession of L about S: 2 S / (r^3 (1-e^2)^(3/2)), Kepler r^3 = M/(2 pi nu)^2
    # (G = c = 1, seconds); spin-orbit part of the periastron rate = -3 cos(lambda) x that.
    for e, spin, lam in ((0.0, 0.5, 0.4), (0.3, 0.9, 2.0)):
        th = theta_base(M=2e6, mu=10.0, spin=spin, lam=lam)
        m_s = 2e6 * TSUN
        nu = 2e-3
        r3 = m_s / (2 * np.pi * nu) ** 2
        lt = 2 * spin * m_s ** 2 / (r3 * (1 - e * e) ** 1.5)
        r = O.rhs(th, nu, e, 1)
        assert r[4] == pytest.approx(lt, rel=1e-13)
        r0 = O.rhs(theta_base(M=2e6, mu=10.0, spin=0.0, lam=lam), nu, e, 1)
        assert r[3] - r0[3] == pytest.approx(-3 * math.cos(lam) * lt, rel=1e-10)


def test_spin_terms_vanish_at_zero_spin(oracle_mod):
    a = O.rhs(theta_base(spin=0.0, lam=0.3), 2e-3, 0.25, 1)
    b = O.rhs(theta_base(spin=0.0, lam=2.5), 2e-3, 0.25, 1)
    np.testing.assert_array_equal(a, b)
    assert a[4] == 0.0


def test_integrator_step_halving(oracle_mod):
    th = I.draw_sources(1, 1, 1 << 16)[0]
    n, dt = 1 << 14, 15.0
    a = O.orbit(th, n, dt)
    b = O.orbit(th, 2 * n - 1, dt / 2)
    assert abs(a["phi"][-1] - b["phi"][-1]) < 1e-9
    assert abs(a["nu"][-1] / b["nu"][-1] - 1) < 1e-15
    assert abs(a["gamma"][-1] - b["gamma"][-1]) < 1e-9


def test_backward_newtonian_chirp_closed_form(oracle_mod):
    # backward mode (paper Sec. 3: initial conditions at the LSO, integrated
    # back in time): pn_terms = 0, e = 0, the last sample sits at nu_LSO and
    # nu(t) = nu_L (1 + (T - t)/tau_L)^(-3/8), tau_L = (5/256) M (M/mu) (2 pi M nu_L)^(-8/3)
    m, mu = 1e6, 10.0
    th = theta_base(M=m, mu=mu, e0=0.0, nu0=0.0, spin=0.0, phi0=0.25)
    n, dt = 20000, 15.0
    orb = O.orbit(th, n, dt, O.Opts(pn_terms=0, backward=1))
    nu_l = O.nu_lso(m, 0.0)
    assert nu_l == pytest.approx(1 / (6 ** 1.5 * 2 * np.pi * m * TSUN), rel=1e-15)
    m_s, mu_s = m * TSUN, mu * TSUN
    tau = 5.0 / 256.0 * m_s * (m_s / mu_s) * (2 * np.pi * m_s * nu_l) ** (-8.0 / 3.0)
    back = (n - 1 - np.arange(n)) * dt            # time before the LSO
    nu_ref = nu_l * (1 + back / tau) ** (-3.0 / 8.0)
    phi_ref = 0.25 - 2 * np.pi * nu_l * tau * 8.0 / 5.0 * ((1 + back / tau) ** (5.0 / 8.0) - 1)
    assert orb["nu"][-1] == nu_l and orb["phi"][-1] == 0.25
    assert np.max(np.abs(orb["nu"] / nu_ref - 1)) < 1e-13
    assert np.max(np.abs(orb["phi"] - phi_ref)) < 1e-8
    assert orb["n_valid"] == n


def test_backward_then_forward_returns_to_the_lso(oracle_mod):
    # full AK equations: integrating forward from the backward orbit's first
    # sample reproduces the LSO state at the last sample (time reversibility)
    th = theta_base(M=8e5, mu=15.0, e0=0.3, spin=0.6, lam=0.9, phi0=0.1, gam0=0.2, alp0=0.3)
    n, dt = 1 << 14, 15.0
    b = O.orbit(th, n, dt, O.Opts(backward=1))
    f_th = th.copy()
    f_th[[I.I_PHI0, I.I_NU0, I.I_E0, I.I_GAM0, I.I_ALP0]] = [b["phi"][0], b["nu"][0], b["e"][0], b["gamma"][0],
                                                             b["alpha"][0]]
    # forward mode stops at the LSO: shorten by one sample so the check stays inside it
    f = O.orbit(f_th, n - 1, dt)
    for k in ("phi", "gamma", "alpha"):
        assert abs(f[k][-1] - b[k][-2]) < 1e-8, k
    assert abs(f["nu"][-1] / b["nu"][-2] - 1) < 1e-13
    assert abs(f["e"][-1] - b["e"][-2]) < 1e-14
    assert b["e"][0] > 0.3 and b["nu"][0] < b["nu"][-1]


def test_plunge_detected(oracle_mod):
    # start just below the LSO: the orbit plunges and the waveform is zero after it
    m, e0 = 1e6, 0.2
    th = theta_base(M=m, mu=20.0, e0=e0, nu0=0.999 * O.nu_lso(m, e0))
    hI, hII, st = O.waveform(th, 4096, 15.0, O.Opts(n_max=4))
    assert st[0] & 1
    k = np.nonzero(hI[0])[0].max() + 1
    assert 0 < k < 4096 and np.all(hI[0, k:] == 0) and np.all(hII[0, k:] == 0)


# ---------------------------------------------------------------- response
def test_antenna_invariants(oracle_mod):
    g = np.random.default_rng(1)
    for _ in range(50):
        th, ph, p1, p2 = g.uniform(0, np.pi), g.uniform(0, 2 * np.pi), g.uniform(0, np.pi), g.uniform(0, np.pi)
        a, b = O.antenna(th, ph, p1), O.antenna(th, ph, p2)
        assert a[0] ** 2 + a[1] ** 2 == pytest.approx(b[0] ** 2 + b[1] ** 2, rel=1e-13)
        ct = np.cos(th)
        # psi-independent magnitude: (1/4)(1+cos^2)^2 cos^2 2phi + cos^2 sin^2 2phi
        ref = 0.25 * (1 + ct * ct) ** 2 * np.cos(2 * ph) ** 2 + ct * ct * np.sin(2 * ph) ** 2
        assert a[0] ** 2 + a[1] ** 2 == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_geometry_vectors(oracle_mod):
    g = np.random.default_rng(2)
    for _ in range(30):
        th = theta_base(ths=g.uniform(0.1, 3.0), phs=g.uniform(0, 6.2), thk=g.uniform(0.1, 3.0),
                        phk=g.uniform(0, 6.2), lam=g.uniform(0.1, 3.0))
        t, alp = g.uniform(0, 3e7), g.uniform(0, 50)
        c, psi, beta, thd, phd, dop = O.geometry(th, t, alp)
        # L.N from the explicit precession cone: S cos(lam) + sin(lam)(e1 cos a + e2 sin a)
        ths, phs, thk, phk, lam = th[I.I_THS], th[I.I_PHS], th[I.I_THK], th[I.I_PHK], th[I.I_LAM]
        N = np.array([np.sin(ths) * np.cos(phs), np.sin(ths) * np.sin(phs), np.cos(ths)])
        S = np.array([np.sin(thk) * np.cos(phk), np.sin(thk) * np.sin(phk), np.cos(thk)])
        e1 = np.array([-np.cos(thk) * np.cos(phk), -np.cos(thk) * np.sin(phk), np.sin(thk)])
        e2 = np.cross(S, e1)
        L = S * np.cos(lam) + np.sin(lam) * (e1 * np.cos(alp) + e2 * np.sin(alp))
        assert c == pytest.approx(L @ N, abs=1e-12)
        # cos(theta_d) is the source direction on the detector normal
        phib = 2 * np.pi * t / 31557600.0
        zd = np.array([-np.sqrt(3) / 2 * np.cos(phib), -np.sqrt(3) / 2 * np.sin(phib), 0.5])
        assert np.cos(thd) == pytest.approx(zd @ N, abs=1e-12)
        assert dop == pytest.approx(499.004783836 * np.sin(ths) * np.cos(phib - phs), rel=1e-12, abs=1e-9)
        # beta: rotating L x N by beta about L gives the direction of L x S
        u, v = np.cross(L, N), np.cross(L, S)
        u, v = u / np.linalg.norm(u), v / np.linalg.norm(v)
        rot = u * np.cos(beta) + np.cross(L, u) * np.sin(beta)
        assert np.allclose(rot, v, atol=1e-10)


def test_waveform_e0_reduces_to_quadrupole(oracle_mod):
    # e0 = 0 stays circular: the full channel output equals the closed-form n = 2
    # quadrupole projected with the oracle's own geometry at each sample.
    th = theta_base(M=1e6, mu=10.0, e0=0.0, nu0=1e-3, spin=0.4)
    n, dt = 512, 15.0
    opts = O.Opts(n_max=8, doppler=1)
    hI, hII, st = O.waveform(th, n, dt, opts)
    orb = O.orbit(th, n, dt, opts)
    m_s, mu_cm = 1e6 * TSUN, 10.0 * TSUN * C_CGS
    for j in (0, 100, 511):
        t = j * dt
        c, psi, beta, thd, phd, dop = O.geometry(th, t, orb["alpha"][j])
        amp = (2 * np.pi * m_s * orb["nu"][j]) ** (2 / 3) * mu_cm
        phi_d = orb["phi"][j] + 2 * np.pi * orb["nu"][j] * dop
        arg = 2 * phi_d + 2 * orb["gamma"][j] + 2 * beta
        hp = 2 * amp * (1 + c * c) * np.cos(arg)
        hx = -4 * amp * c * np.sin(arg)
        fI, fII = O.antenna(thd, phd, psi), O.antenna(thd, phd - np.pi / 4, psi)
        assert hI[0, j] == pytest.approx(np.sqrt(3) / 2 * (fI[0] * hp + fI[1] * hx), rel=1e-9, abs=1e-9 * amp)
        assert hII[0, j] == pytest.approx(np.sqrt(3) / 2 * (fII[0] * hp + fII[1] * hx), rel=1e-9, abs=1e-9 * amp)


def test_waveform_sampled_matches_full(oracle_mod):
    th = I.draw_sources(1, 2, 1 << 12)
    hI, hII, _ = O.waveform(th, 4096, 15.0, O.Opts(n_max=6))
    idx = np.array([0, 1, 7, 1000, 4095])
    sI, sII, _ = O.waveform_sampled(th, 4096, 15.0, idx, O.Opts(n_max=6))
    np.testing.assert_array_equal(sI, hI[:, idx])
    np.testing.assert_array_equal(sII, hII[:, idx])


# -------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 512, 1024])
def test_fft_matches_brute_force_dft(oracle_mod, n):
    g = np.random.default_rng(n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    for sign in (-1, 1):
        a = O.fft(x, sign)
        b = O.dft(x, sign)
        assert np.max(np.abs(a - b)) < 1e-13 * np.sqrt(n) * np.max(np.abs(b))


def test_fft_parseval_impulse_tone(oracle_mod):
    n = 1 << 14
    g = np.random.default_rng(3)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    X = O.fft(x)
    assert np.sum(np.abs(X) ** 2) == pytest.approx(n * np.sum(np.abs(x) ** 2), rel=1e-13)
    d = np.zeros(n, complex)
    d[0] = 1
    assert np.max(np.abs(O.fft(d) - 1)) < 1e-15
    k0 = 37
    tone = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    T = O.fft(tone)
    assert abs(T[k0] - n) < 1e-9 and np.max(np.abs(np.delete(T, k0))) < 1e-9


# ---------------------------------------------------------- inner product
def test_inner_product_time_domain(oracle_mod):
    # white weight on every bin: sum_k w Re(conj(A_k)B_k) = w N sum_j (a_j b_j) per channel (Parseval)
    n = 4096
    g = np.random.default_rng(4)
    a = g.standard_normal((2, n))
    b = g.standard_normal((2, n))
    A = O.fft(a[0] + 1j * a[1])
    B = O.fft(b[0] + 1j * b[1])
    w = np.full(n, 0.37)
    assert O.inner(A, B, w) == pytest.approx(0.37 * n * np.sum(a * b), rel=1e-13)


def test_weights_match_one_sided_form(oracle_mod):
    # packed two-channel sum with the oracle's weights equals the textbook
    # one-sided 4 Re sum a~* b~ / S df per channel (a~ = dt * DFT), via numpy rfft
    n, dt = 1 << 12, 15.0
    psd = I.psd_bc04(n, dt)
    w = O.weights(psd, n, dt, 1e-4, 1.0)
    g = np.random.default_rng(5)
    a = g.standard_normal((2, n))
    b = g.standard_normal((2, n))
    A = O.fft(a[0] + 1j * a[1])
    B = O.fft(b[0] + 1j * b[1])
    df = 1 / (n * dt)
    ref = 0.0
    for c in range(2):
        fa, fb = dt * np.fft.rfft(a[c]), dt * np.fft.rfft(b[c])
        f = np.arange(n // 2 + 1) * df
        k = (np.arange(n // 2 + 1) > 0) & (np.arange(n // 2 + 1) < n // 2) & (f >= 1e-4)
        ref += 4 * np.sum((np.conj(fa[k]) * fb[k]).real / psd[k]) * df
    assert O.inner(A, B, w) == pytest.approx(ref, rel=1e-12)
    assert np.all(w[:1] == 0) and w[n // 2] == 0
    np.testing.assert_array_equal(w[1:], w[1:][::-1])


def test_noise_inner_product_statistics(oracle_mod):
    # <n|n> over the band ~ 2 per channel per bin (sigma^2 = 8 N_bins in total)
    n, dt = 1 << 16, 15.0
    psd = I.psd_bc04(n, dt)
    w = O.weights(psd, n, dt, 1e-4, 1.0)
    nn = I.noise_spectrum(7, psd, n, dt)
    nb = np.count_nonzero(w[: n // 2])
    val = O.inner(nn, nn, w)
    assert abs(val - 4 * nb) < 5 * np.sqrt(8 * nb)


# --------------------------------------------------------------- cosmology
def test_dl_einstein_de_sitter(oracle_mod):
    o = O.Opts(omega_m=1.0)
    for z in (0.1, 0.5, 1.0, 3.0):
        ref = 2 * C_CGS * MPC / (67.4e5) * (1 + z) * (1 - 1 / np.sqrt(1 + z))
        assert O.dl_cm(z, o) == pytest.approx(ref, rel=1e-14)


def test_dl_and_lookback_vs_quadrature(oracle_mod):
    om = 0.315
    E = lambda z: np.sqrt(om * (1 + z) ** 3 + 1 - om)
    hinv = MPC / 67.4e5
    for z in (0.05, 0.3, 1.0, 2.0):
        dc, _ = si.quad(lambda x: 1 / E(x), 0, z, epsabs=0, epsrel=1e-13)
        assert O.dl_cm(z) == pytest.approx((1 + z) * C_CGS * hinv * dc, rel=1e-13)
        tl, _ = si.quad(lambda x: 1 / ((1 + x) * E(x)), 0, z, epsabs=0, epsrel=1e-13)
        assert O.lookback_s(z) == pytest.approx(hinv * tl, rel=1e-13)


def test_xi_limits(oracle_mod):
    for xi0 in (0.7, 1.0, 1.3):
        assert O.xi(0.0, xi0) == 1.0
        assert O.xi(1e6, xi0, 2.0) == pytest.approx(xi0, abs=1e-11)
    assert O.xi(0.8, 1.0) == 1.0
    # n = 1: Xi = Xi0 + (1 - Xi0)/(1+z)
    assert O.xi(1.0, 0.5, 1.0) == pytest.approx(0.75, rel=1e-15)


def test_delay_fraction_high_precision(oracle_mod):
    # r = frac(dt_GW / T) with dt_GW = -(alpha_T/2) t_LB(z), against 60-digit quadrature
    mpmath.mp.dps = 60
    n, dt = 1 << 21, 15.0
    for at, z in ((0.05, 1.0), (-0.13, 0.3), (1e-3, 0.7)):
        om = mpmath.mpf(0.315)
        E = lambda x: mpmath.sqrt(om * (1 + x) ** 3 + 1 - om)
        hinv = mpmath.mpf(3.0856775814913673e24) / (mpmath.mpf(67.4) * 100000)
        tl = hinv * mpmath.quad(lambda x: 1 / ((1 + x) * E(x)), [0, mpmath.mpf(z)])
        dtgw = -mpmath.mpf(at) / 2 * tl
        q = dtgw / (mpmath.mpf(n) * mpmath.mpf(dt))
        r = q - mpmath.floor(q)
        d = O.delay(at, z, n, dt)
        assert d[0] == pytest.approx(float(dtgw), rel=1e-15)
        assert abs(mpmath.mpf(d[1]) + mpmath.mpf(d[2]) - r) < mpmath.mpf(10) ** -24
    assert np.all(O.delay(0.0, 0.5, n, dt) == 0.0)
    assert O.delay(0.05, 0.5, n, dt)[0] < 0   # faster GWs arrive earlier


# -------------------------------------------------------------------- lnL
def _noise_free(th_inj, n, dt, opts):
    hI, hII, _ = O.waveform(th_inj, n, dt, opts)
    H = O.packed_spectrum(hI[0], hII[0])
    pro = O.prologue(th_inj, n, dt, opts)
    ks = np.where(np.arange(n) * 2 <= n, np.arange(n), np.arange(n) - n)
    r = mpmath.mpf(pro[4]) + mpmath.mpf(pro[5])
    mpmath.mp.dps = 40
    ph = np.array([float((k * r) % 1) for k in ks])
    return H * np.exp(-2j * np.pi * ph) / pro[2], H, pro


def test_lnl_noise_free_injection_is_zero(oracle_mod):
    n, dt = 1 << 12, 15.0
    opts = O.Opts(n_max=6)
    inj = I.draw_sources(11, 1, n)[0]
    inj[I.I_ALPT] = 0.04
    d, H, pro = _noise_free(inj, n, dt, opts)
    w = O.weights(I.psd_bc04(n, dt), n, dt, 1e-4, 1.0)
    lnl, dh, hh, st = O.loglike(inj, n, dt, d, w, opts)
    dd = O.inner(d, d, w)
    assert st[0] == 0
    assert lnl[0] - 0.5 * dd == pytest.approx(0.0, abs=1e-10 * dd)
    # a walker with another GW speed is less likely; the delay leaves <h|h> unchanged
    other = inj.copy()
    other[I.I_ALPT] = 0.0401
    lnl2, dh2, hh2, _ = O.loglike(other, n, dt, d, w, opts)
    assert lnl2[0] < lnl[0]
    assert hh2[0] == pytest.approx(hh[0], rel=1e-13)


def test_lnl_gr_limit(oracle_mod):
    # Xi0 = 1 and alpha_T = 0: d_GW = d_L, no delay; lnL = <d|h_u>/d_L - <h_u|h_u>/(2 d_L^2)
    n, dt = 1 << 12, 15.0
    opts = O.Opts(n_max=5)
    th = I.draw_sources(12, 3, n)
    th[:, I.I_XI0] = 1.0
    th[:, I.I_ALPT] = 0.0
    psd = I.psd_bc04(n, dt)
    w = O.weights(psd, n, dt, 1e-4, 1.0)
    data = I.noise_spectrum(8, psd, n, dt)
    lnl, dh, hh, _ = O.loglike(th, n, dt, data, w, opts)
    hI, hII, _ = O.waveform(th, n, dt, opts)
    for k in range(3):
        H = O.packed_spectrum(hI[k], hII[k])
        dl = O.dl_cm(th[k, I.I_Z], opts)
        ref = O.inner(data, H, w) / dl - 0.5 * O.inner(H, H, w) / dl ** 2
        assert lnl[k] == pytest.approx(ref, rel=1e-12, abs=1e-12 * abs(O.inner(H, H, w)) / dl ** 2)


# ------------------------------------------- frequency-dependent propagation
def test_fd_zero_coefficients_and_pure_phase(oracle_mod):
    # all coefficients zero: the standard likelihood, bit for bit; a pure
    # speed term (a_m = 0) is a phase: <h|h> unchanged bit for bit
    n, dt = 1 << 12, 15.0
    opts = O.Opts(n_max=4)
    th = I.draw_sources(21, 3, n)
    psd = I.psd_bc04(n, dt)
    w = O.weights(psd, n, dt, 1e-4, 1.0)
    data = I.noise_spectrum(9, psd, n, dt)
    ref = O.loglike(th, n, dt, data, w, opts)
    got = O.loglike_fd(th, n, dt, data, w, 2, 3, 1e-2, np.zeros((3, 5)), opts)
    for a, b in zip(ref[:3], got[:3]):
        np.testing.assert_array_equal(a, b)
    coef = np.zeros((3, 5))
    coef[:, 2:] = np.random.default_rng(3).normal(0, 0.05, (3, 3))
    ph = O.loglike_fd(th, n, dt, data, w, 2, 3, 1e-2, coef, opts)
    np.testing.assert_array_equal(ph[2], ref[2])
    assert np.all(np.abs(ph[1] - ref[1]) > 0)


def test_fd_factor_against_closed_form(oracle_mod):
    # One bin of data at a time (D = delta_k0 and D = i delta_k0) reads the
    # factor G_k0 = F_k0 exp(-2 pi i f dt_GW) applied to H_k0 off <d|h>.
    # Independent closed form at 50 digits: G = (1+z)^(-alpha_M(|f|)/2)
    # exp(-2 pi i f dt_GW(f)), dt_GW(f) = -(alpha_T + sum b_m (|f|/f*)^m)/2
    # t_LB(z), with t_LB from mpmath quadrature; both signs of f.
    mpmath.mp.dps = 50
    n, dt = 1 << 12, 15.0
    opts = O.Opts(n_max=3)
    th = I.draw_sources(22, 1, n)
    th[0, I.I_ALPT] = 0.037
    z = th[0, I.I_Z]
    fstar = 3e-3
    a_m = [0.4, -0.25]
    b_m = [0.05, -0.02, 0.011]
    coef = np.array([a_m + b_m])
    hI, hII, _ = O.waveform(th, n, dt, opts)
    H = O.packed_spectrum(hI[0], hII[0])
    psd = np.ones(n // 2 + 1)
    w = O.weights(psd, n, dt, 0.0, 1.0)
    om = mpmath.mpf(0.315)
    E = lambda x: mpmath.sqrt(om * (1 + x) ** 3 + 1 - om)
    hinv = mpmath.mpf(3.0856775814913673e24) / (mpmath.mpf(67.4) * 100000)
    tlb = hinv * mpmath.quad(lambda x: 1 / ((1 + x) * E(x)), [0, mpmath.mpf(z)])
    for k0 in (5, 301, 1777, n - 1777, n - 3):
        ks = k0 if 2 * k0 <= n else k0 - n
        f = mpmath.mpf(ks) / (mpmath.mpf(n) * mpmath.mpf(dt))
        x = abs(f) / mpmath.mpf(fstar)
        am = sum(mpmath.mpf(a) * x ** (m + 1) for m, a in enumerate(a_m))
        at = mpmath.mpf(th[0, I.I_ALPT]) + sum(mpmath.mpf(b) * x ** (m + 1) for m, b in enumerate(b_m))
        dtgw = -at / 2 * tlb
        cyc = f * dtgw
        cyc -= mpmath.floor(cyc)
        g = (1 + mpmath.mpf(z)) ** (-am / 2) * mpmath.expjpi(-2 * cyc)
        out = []
        for dval in (1.0, 1j):
            d = np.zeros(n, dtype=np.complex128)
            d[k0] = dval
            _, dh, _, _ = O.loglike_fd(th, n, dt, d, w, len(a_m), len(b_m), fstar, coef, opts)
            out.append(dh[0] / w[k0])
        hg = out[0] + 1j * out[1]
        G = hg / H[k0]
        assert abs(G - complex(g)) < 1e-12 * abs(complex(g)), (k0, G, complex(g))
