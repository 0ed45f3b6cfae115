"""CPU pins of the numerical schemes the CUDA kernels use, each restated here
in numpy from its definition (no kernel code is imported or run):

  * the Bessel power series J_m(x) = (x/2)^m/m! sum_k a_k y^k, y = x^2/4, cut
    after K = min(ceil(12 + 1.05 x), 48) terms: the omitted tail is below
    1e-16 of the sum for every order the waveform kernels use (m = n+1, n+2
    at x = n e, n <= 32, e < 0.999), and Horner's rule over the rounded
    coefficient table matches scipy's J_m;
  * the FP64 FFT's FMA-folded radix-4 / radix-2 Stockham stages with
    (cos, tan) twiddles (|cos| floored at 2^-60): the whole transform, with the
    kernels' index arithmetic, equals numpy's FFT in both directions;
  * the FP64 sin/cos of a reduced phase from a 512-point exp table and
    Taylor polynomials to x^5 / x^4: absolute error ~2 ulp;
  * the mixed path's fixed-point phases (Q0.64 base + tau * increment, the
    increment reduced mod 1 so that it fits a signed 64-bit integer): the
    phase mod 1 is exact to 1e-9 cycles at any cycles per sample.
"""
import math

import numpy as np
import pytest
from scipy.special import gammaln, jv

K_TERMS = 48


def series_terms(x: float) -> int:
    return min(int(12.0 + 1.05 * x) + 1, K_TERMS)


def test_bessel_term_count_leaves_tail_below_1e16():
    for n in range(1, 33):
        for m in (n + 1, n + 2):
            for e in np.linspace(0.001, 0.998, 120):
                x = n * e
                y = x * x / 4
                k = np.arange(0, 120)
                t = np.exp(gammaln(m + 1) - gammaln(k + 1) - gammaln(m + k + 1) + k * np.log(y)) * (-1.0) ** k
                K = series_terms(x)
                tail = np.abs(t[K:]).sum()
                assert tail <= 1e-16 * abs(t.sum()), (n, m, e, K)


def bessel_horner(m: int, x: float, table: np.ndarray) -> float:
    half = 0.5 * x
    lead = half ** m / math.factorial(m)
    y = half * half
    K = series_terms(x)
    s = table[m, K - 1]
    for k in range(K - 2, -1, -1):
        s = s * y + table[m, k]
    return lead * s


def test_bessel_horner_matches_scipy():
    from fractions import Fraction
    table = np.zeros((35, K_TERMS))
    for m in range(35):
        a = Fraction(1)
        for k in range(K_TERMS):
            if k:
                a = -a / (k * (m + k))
            table[m, k] = float(a)
    worst = 0.0
    for n in range(1, 31):
        for m in (n + 1, n + 2):
            for e in np.linspace(0.01, 0.6, 25):
                ref = jv(m, n * e)
                worst = max(worst, abs(bessel_horner(m, n * e, table) - ref) / abs(ref))
    assert worst < 1e-13, worst


# ------------------------------------------------------------------ FFT
def ct_table():
    i = np.arange(4096)
    c = np.cos(-2 * np.pi * i / 4096)
    s = np.sin(-2 * np.pi * i / 4096)
    c[i % 1024 == 0] = np.rint(c[i % 1024 == 0])          # exact values at quarter turns
    s[i % 1024 == 0] = np.rint(s[i % 1024 == 0])
    cf = np.where(np.abs(c) < 2.0 ** -60, 2.0 ** -60, c)
    return cf, s / cf


def stockham_fma(x: np.ndarray, sign: int) -> np.ndarray:
    """The FP64 shared-memory transform of one row: radix-4 stages (the first
    without twiddles, the rest FMA-folded), then one FMA-folded radix-2 stage
    when log2(L) is odd; Stockham indexing as in the kernels."""
    L = x.size
    LG = int(np.log2(L))
    cf, tf = ct_table()
    if sign > 0:
        tf = -tf
    buf = x.astype(np.complex128).copy()
    Q4 = L // 4
    for st in range(LG // 2):
        ns = 1 << (2 * st)
        j = np.arange(Q4)
        k = j & (ns - 1)
        a0, a1, a2, a3 = buf[j], buf[j + Q4], buf[j + 2 * Q4], buf[j + 3 * Q4]
        if st > 0:
            u = (k * 4096) >> (2 * st + 2)
            c1, t1, c2, t2 = cf[u], tf[u], cf[2 * u], tf[2 * u]
            v2 = (a2.real - t2 * a2.imag) + 1j * (a2.imag + t2 * a2.real)
            v3 = (a3.real - t2 * a3.imag) + 1j * (a3.imag + t2 * a3.real)
            pp, pm = a0 + c2 * v2, a0 - c2 * v2
            qp, qm = a1 + c2 * v3, a1 - c2 * v3
            e = (qp.real - t1 * qp.imag) + 1j * (qp.imag + t1 * qp.real)
            f = (qm.real - t1 * qm.imag) + 1j * (qm.imag + t1 * qm.real)
            c1s = c1 if sign < 0 else -c1
            y = [pp + c1 * e, (pm.real + c1s * f.imag) + 1j * (pm.imag - c1s * f.real),
                 pp - c1 * e, (pm.real - c1s * f.imag) + 1j * (pm.imag + c1s * f.real)]
        else:
            b0, b1, b2, d = a0 + a2, a0 - a2, a1 + a3, a1 - a3
            b3 = -1j * d if sign < 0 else 1j * d
            y = [b0 + b2, b1 + b3, b0 - b2, b1 - b3]
        dst = ((j >> (2 * st)) << (2 * st + 2)) + k
        out = np.empty_like(buf)
        for q in range(4):
            out[dst + q * ns] = y[q]
        buf = out
    if LG & 1:
        H2 = L // 2
        NS = 1 << (2 * (LG // 2))
        j = np.arange(H2)
        k = j & (NS - 1)
        a0, a1 = buf[j], buf[j + H2]
        w = (k * 4096) // (NS * 2)
        c, t = cf[w], tf[w]
        v = (a1.real - t * a1.imag) + 1j * (a1.imag + t * a1.real)
        dst = (j // NS) * NS * 2 + k
        out = np.empty_like(buf)
        out[dst] = a0 + c * v
        out[dst + NS] = a0 - c * v
        buf = out
    return buf


@pytest.mark.parametrize("lg", [4, 5, 10, 11])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fma_folded_stockham_equals_dft(lg, sign):
    g = np.random.default_rng(lg)
    x = g.standard_normal(1 << lg) + 1j * g.standard_normal(1 << lg)
    got = stockham_fma(x, sign)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * x.size
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-15 * lg


def r8_rows_fft(x):
    """The register-resident FP32 pass-2 row FFT, replayed with the kernel's
    indexing (threads as array lanes): T = N1/8 threads hold points t + q T;
    radix-8 Stockham stages with stage twiddles W_{8 NS}^k (powers by
    products), outputs to (t / NS) 8 NS + k + q NS, then a radix-4 (two
    butterflies) or radix-2 (four) last stage; slot q ends as bin t + q T."""
    n1 = x.size
    lg = n1.bit_length() - 1
    T = n1 // 8
    t = np.arange(T)
    h = np.sqrt(0.5)

    def dft4(a0, a1, a2, a3):
        s0, s1, s2, s3 = a0 + a2, a0 - a2, a1 + a3, -1j * (a1 - a3)
        return s0 + s2, s1 + s3, s0 - s2, s1 - s3

    def dft8(a):
        b = [a[r] + a[r + 4] for r in range(4)]
        d = [a[r] - a[r + 4] for r in range(4)]
        c = [d[0], h * (1 - 1j) * d[1], -1j * d[2], -h * (1 + 1j) * d[3]]
        e, o = dft4(*b), dft4(*c)
        return [e[0], o[0], e[1], o[1], e[2], o[2], e[3], o[3]]

    def tw(m, k):
        return np.exp(-2j * np.pi * k / m)

    v = [x[t + q * T] for q in range(8)]
    for st in range(lg // 3):
        ns = 8 ** st
        k = t & (ns - 1)
        if ns > 1:
            w1 = tw(8 * ns, k)
            w2 = w1 * w1; w3 = w2 * w1; w4 = w2 * w2
            w = [1, w1, w2, w3, w4, w4 * w1, w4 * w2, w4 * w3]
            v = [v[q] * w[q] for q in range(8)]
        v = dft8(v)
        if 8 * ns < n1:
            xb = np.zeros(n1, dtype=complex)
            d0 = (t // ns) * ns * 8 + k
            for q in range(8):
                xb[d0 + q * ns] = v[q]
            v = [xb[t + q * T] for q in range(8)]
    if lg % 3 == 2:
        for hh in range(2):
            w1 = tw(n1, t + hh * T)
            a = dft4(v[hh], v[hh + 2] * w1, v[hh + 4] * w1 * w1, v[hh + 6] * w1 * w1 * w1)
            v[hh], v[hh + 2], v[hh + 4], v[hh + 6] = a
    elif lg % 3 == 1:
        for i in range(4):
            b = v[i + 4] * tw(n1, t + i * T)
            v[i], v[i + 4] = v[i] + b, v[i] - b
    out = np.zeros(n1, dtype=complex)
    for q in range(8):
        out[t + q * T] = v[q]
    return out


@pytest.mark.parametrize("lg", [8, 9, 10, 11, 12])
def test_register_radix8_rows_equal_dft(lg):
    """Pass 2 of the FP32 path (rows of 256..4096 points): the kernel's
    stage structure and bin mapping give the forward DFT."""
    g = np.random.default_rng(lg)
    x = g.standard_normal(1 << lg) + 1j * g.standard_normal(1 << lg)
    got = r8_rows_fft(x)
    ref = np.fft.fft(x)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-14


@pytest.mark.parametrize("lg", [8, 9, 10, 11, 12])
def test_register_stage_padded_addresses_are_affine(lg):
    """The register kernels address the padded exchange buffer (element i at
    i + i // 16) as pad(base) plus compile-time offsets: writes d0 + q NS at
    pad(d0) + q NS + (q NS >> 4), reads t + q T at pad(t) + q (T + T/16),
    for every thread and radix-8 stage that writes."""
    n = 1 << lg
    T = n // 8

    def pad(i):
        return i + (i >> 4)

    t = np.arange(T)
    for st in range(lg // 3):
        ns = 8 ** st
        if 8 * ns >= n:
            continue
        d0 = (t // ns) * ns * 8 + (t & (ns - 1))
        for q in range(8):
            assert np.array_equal(pad(d0 + q * ns), pad(d0) + q * ns + ((q * ns) >> 4)), (lg, st, q)
    for q in range(8):
        assert np.array_equal(pad(t + q * T), pad(t) + q * (T + T // 16))


def test_stage_twiddle_table_layout():
    """tt[M/2 + k] = exp(-2 pi i k / M): entry i belongs to M = 2 * 2^floor(log2 i)
    and equals the 4096-point table at k * 4096 / M (same double angle)."""
    for i in range(1, 4096):
        half = 1 << (i.bit_length() - 1)
        k, m = i - half, 2 * half
        assert k < m // 2
        assert (-2.0 * k / m) == (-2.0 * (k * (4096 // m)) / 4096.0)


def test_sincos_512_table():
    """The FP64 kernel's sin/cos of phases in cycles (whole cycles kept):
    nearest integer k of 512 f by adding 1.5 * 2^52 (the sum's low word is k,
    subtracting the constant gives k exactly), table entry k mod 512, Taylor
    polynomials of the exact residual d = f - k/512."""
    pil = np.longdouble("3.14159265358979323846264338327950288")
    ks = np.arange(512).astype(np.longdouble)
    tc = np.cos(2 * pil * ks / 512).astype(np.float64)
    ts = np.sin(2 * pil * ks / 512).astype(np.float64)
    g = np.random.default_rng(3)
    f = np.concatenate([g.uniform(-0.5, 0.5, 300_000), g.uniform(-40.0, 40.0, 300_000),
                        np.array([0.0, -0.0, 1 / 1024, -1 / 1024, 0.5, -0.5, 39.998046875])])
    big = 6755399441055744.0
    kb = f * 512.0 + big                        # f * 512 is exact: one rounding, as the FMA
    kd = kb - big
    assert np.array_equal(kd, np.rint(f * 512.0))   # round to nearest even
    k = kb.view(np.int64).astype(np.int32)      # the low word, two's complement
    assert np.array_equal(k, kd.astype(np.int64).astype(np.int32))
    d = f - kd / 512.0
    assert np.abs(d).max() <= 1 / 1024
    x = d * 6.283185307179586
    x2 = x * x
    sx = (x2 * x) * (x2 * (1 / 120) - 1 / 6) + x
    cx = x2 * (x2 * (1 / 24) - 0.5) + 1.0
    idx = k & 511
    s = ts[idx] * cx + tc[idx] * sx
    c = tc[idx] * cx - ts[idx] * sx
    fl = f.astype(np.longdouble)
    assert np.abs(s - np.sin(2 * pil * fl)).max() < 4e-16
    assert np.abs(c - np.cos(2 * pil * fl)).max() < 4e-16


# ------------------------------------------------- fixed-point phases (mixed)
def to_q64(f):
    """Phase fraction in [0, 1) -> unsigned Q0.64."""
    f = f - math.floor(f)
    return int(f * 2.0 ** 64) % 2 ** 64


def to_q64s(f):
    """Per-sample increment -> signed Q0.64, reduced mod 1 to [-1/2, 1/2);
    the kernels convert with a 64-bit signed integer, so the value must fit
    (without the reduction an increment above half a cycle would not)."""
    f = f - round(f)
    if f >= 0.5:
        f -= 1.0
    v = int(round(f * 2.0 ** 64))
    assert -2 ** 63 <= v < 2 ** 63
    return v


@pytest.mark.parametrize("cycles_per_sample", [1e-4, 0.3, 0.7, 3.2, 41.9])
def test_fixed_point_phase_wraps_mod_one(cycles_per_sample):
    """The mixed kernels keep a phase as base + tau * inc (mod 2^64) plus a
    small polynomial correction; the increment is reduced mod 1 first, which
    matters once a phase moves more than half a cycle per sample (long
    sample intervals).  The phase mod 1 stays within 1e-9 cycles of the exact
    value (before the FP32 rounding of the final conversion)."""
    g = np.random.default_rng(int(cycles_per_sample * 1000))
    ks = 1024
    for _ in range(20):
        c0 = g.uniform(0, 1)
        c1 = cycles_per_sample * ks          # linear term over the interval [cycles]
        base, inc = to_q64(c0), to_q64s(c1 / ks)
        for tau in g.integers(0, ks, 16):
            p = (base + int(tau) * inc) % 2 ** 64
            got = p / 2.0 ** 64
            exact = (c0 + c1 * tau / ks) % 1.0
            d = abs(got - exact)
            assert min(d, 1 - d) < 1e-9, (tau, got, exact)


def dd_to_fx128(hi, lo):
    """The kernels' double-double fraction -> 128-bit fixed point, replayed
    in IEEE doubles (every step exact: scalings by 2^64, floor, and the
    difference of a double and its floor)."""
    two64 = 18446744073709551616.0
    t = hi * two64
    H = math.floor(t)
    r = (t - H) + lo * two64
    F = math.floor(r)
    rem = r - F
    return (int(H) + int(F)) % 2 ** 64, int(rem * two64) % 2 ** 64


def test_fp32_delay_phase_in_fixed_point():
    """FP32 delay tables: frac(m r) for m = mult * k < 2^22 from the 128-bit
    fraction of r by two 64-bit products (m R_hi mod 2^64 plus the high word
    of m R_lo), top 32 bits as a signed phase in [-1/2, 1/2) cycles.  Against
    exact rational arithmetic the phase is within 2^-32 cycles (the
    truncation to 32 bits) at every m."""
    from fractions import Fraction
    g = np.random.default_rng(11)
    for _ in range(200):
        hi = float(g.uniform(0.0, 1.0))
        lo = float(g.uniform(-0.5, 0.5)) * math.ulp(hi)
        if not (0.0 <= hi + lo < 1.0):
            continue
        Rh, Rl = dd_to_fx128(hi, lo)
        r = Fraction(hi) + Fraction(lo)
        assert abs(Fraction(Rh * 2 ** 64 + Rl, 2 ** 128) - r) <= Fraction(1, 2 ** 128)
        for m in (1, 3, 1023, 1 << 20, (1 << 22) - 1, int(g.integers(1, 1 << 22))):
            ph = (m * Rh + ((m * Rl) >> 64)) % 2 ** 64
            top = ph >> 32
            f = (top - 2 ** 32 if top >= 2 ** 31 else top) * 2.0 ** -32
            exact = (m * r) % 1
            if exact >= Fraction(1, 2):
                exact -= 1
            d = abs(Fraction(f) - exact)
            d = min(d, 1 - d)   # on the circle
            assert d <= Fraction(1, 2 ** 32) + Fraction(m + 1, 2 ** 128), (hi, lo, m, float(d))


def smem_stage(buf, R, L, NS, sign):
    """One shared-memory Stockham stage of the FP32 tile transform, replayed
    with the kernel's indexing (one transform, NB = 1): butterfly j reads
    j + q L/R, multiplies slot q by w^q (w = W_{R NS}^k from the 4096-point
    table at k 4096/(R NS), k = j mod NS; conjugated for the inverse), takes
    the R-point DFT and writes slot q to (j / NS) NS R + k + q NS.  The
    16-point DFT is the kernel's: two 8-point halves, the odd one times
    W16^q from the cos/sin(pi q / 8) constants (q = 4: -+i)."""
    Q = L // R
    out = np.empty_like(buf)
    ta = np.exp(-2j * np.pi * np.arange(4096) / 4096)
    step = 4096 // (R * NS)

    def dft(a):
        n = np.arange(len(a))
        return np.exp(sign * 2j * np.pi * np.outer(n, n) / len(a)) @ a

    c1, s1, h = 0.92387953251128675613, 0.38268343236508977173, np.sqrt(0.5)
    cq = [1, c1, h, s1, 0, -s1, -h, -c1]
    sq = [0, s1, h, c1, 1, c1, h, s1]
    for j in range(Q):
        k = j & (NS - 1)
        y = np.array([buf[j + q * Q] for q in range(R)])
        if NS > 1:
            w1 = ta[k * step] if sign < 0 else np.conj(ta[k * step])
            y = y * w1 ** np.arange(R)
        if R == 16:
            e, o = dft(y[0::2]), dft(y[1::2])
            for q in range(1, 8):
                o[q] = o[q] * (-1j if sign < 0 else 1j) if q == 4 else \
                    o[q] * complex(cq[q], -sq[q] if sign < 0 else sq[q])
            y = np.concatenate([e + o, e - o])
        else:
            y = dft(y)
        d = (j // NS) * NS * R + k
        for q in range(R):
            out[d + q * NS] = y[q]
    return out


@pytest.mark.parametrize("lg", [7, 10])
@pytest.mark.parametrize("sign", [-1, 1])
def test_smem_radix16_last_stage_equals_dft(lg, sign):
    """FP32 tile transforms of 2^(3k+1) points (pass 1 at 128 and 1024 rows):
    radix-8 stages, then one radix-16 stage instead of radix 8 + radix 2."""
    L = 1 << lg
    g = np.random.default_rng(lg)
    x = g.standard_normal(L) + 1j * g.standard_normal(L)
    b, ns = x.copy(), 1
    for _ in range(lg // 3 - 1):
        b = smem_stage(b, 8, L, ns, sign)
        ns *= 8
    b = smem_stage(b, 16, L, ns, sign)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * L
    assert np.abs(b - ref).max() / np.abs(ref).max() < 1e-14
