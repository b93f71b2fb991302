"""Error bounds of the fixed-point dispersion phase used by the FP32 kernels.

The kernels evaluate theta = frac(k'^2 a + k'^3 b) turns (a = pi I2 / T^2,
b = 2 pi^2 I3 / (3 T^3), the phase of beta after Eq. (2)) in unsigned
Q0.64 arithmetic, from 128-bit binary fractions of a and b. Runs of
elements with k' in arithmetic progression follow by exact finite
differences of the cubic. exp(2 pi i theta) is then taken as the nearest
quarter turn times a Taylor series of the residual angle.

This file restates that integer arithmetic in Python integers (wrapping at
2^64 like the device's) and checks the stated error bounds against exact
rationals: a direct evaluation is within 2 ulp of 2^-64 (two truncations,
the second negated for k' < 0); a 32-value run stays within 2^-48 turns;
the quarter-turn split loses less than 2^-32 turns; the series truncate
below 2.5e-8 (cos) and 1.8e-9 (sin).
The compiled kernels themselves are checked against the oracle by the GPU
parity tests.
"""
import math
import random
from fractions import Fraction

import pytest

M64 = (1 << 64) - 1


def frac_q128(x):
    """x mod 1 as a 128-bit binary fraction (x is an FP64 value, so exact)."""
    q = math.floor(Fraction(abs(x)) * (1 << 128)) % (1 << 128)
    return (-q) % (1 << 128) if x < 0 else q


def umulhi(a, b):
    return (a * b) >> 64


def phase_q64(kp, qa, qb):
    a_hi, a_lo, b_hi, b_lo = qa >> 64, qa & M64, qb >> 64, qb & M64
    ak = abs(kp)
    u = ak * ak
    ta = (u * a_hi + umulhi(u, a_lo)) & M64
    f_lo = (u * b_lo) & M64
    f_hi = (u * b_hi + umulhi(u, b_lo)) & M64
    tb = (ak * f_hi + umulhi(ak, f_lo)) & M64
    if kp < 0:
        tb = (-tb) & M64
    return (ta + tb) & M64


def error_ulp(t64, kp, qa, qb):
    """Signed error of a Q0.64 phase against the exact k'^2 A + k'^3 B mod 1,
    in units of 2^-64 turns (A, B the stored 128-bit fractions)."""
    exact = (kp * kp * qa + kp ** 3 * qb) % (1 << 128)
    d = ((t64 << 64) - exact) % (1 << 128)
    if d >= 1 << 127:
        d -= 1 << 128
    return d / (1 << 64)


def run(k_first, D, qa, qb, n):
    """n phases at k_first + s D by finite differences, as the kernels do."""
    t = [phase_q64(k_first + i * D, qa, qb) for i in range(4)]
    d1 = (t[3] - t[2]) & M64
    d2 = (t[3] - 2 * t[2] + t[1]) & M64
    d3 = (t[3] - 3 * t[2] + 3 * t[1] - t[0]) & M64
    out, cur = list(t), t[3]
    for _ in range(4, n):
        d2 = (d2 + d3) & M64
        d1 = (d1 + d2) & M64
        cur = (cur + d1) & M64
        out.append(cur)
    return out


def coefficients(rng, T=102400.0):
    # I2 up to a few thousand ps^2 (kilometres of DM fiber), I3 up to a few ps^3, either sign
    I2, I3 = rng.uniform(-3000, 3000), rng.uniform(-5, 5)
    return frac_q128(math.pi * I2 / T ** 2), frac_q128(2 * math.pi ** 2 * I3 / (3 * T ** 3))


def test_direct_phase_is_within_two_ulp():
    # both products truncate (each low by < 1 ulp); for k' < 0 the k'^3 term
    # is negated, and with it its truncation
    rng = random.Random(11)
    lo = {1: 0.0, -1: 0.0}
    hi = {1: -1.0, -1: -1.0}
    for _ in range(200):
        qa, qb = coefficients(rng)
        for kp in [rng.randint(-(1 << 24), (1 << 24) - 1) for _ in range(20)] + [0, 1, -1, (1 << 24) - 1, -(1 << 24)]:
            e = error_ulp(phase_q64(kp, qa, qb), kp, qa, qb)
            sg = 1 if kp >= 0 else -1
            lo[sg], hi[sg] = min(lo[sg], e), max(hi[sg], e)
    assert -2.0 < lo[1] and hi[1] <= 0.0
    assert -1.0 < lo[-1] and hi[-1] < 1.0


def test_finite_difference_runs_stay_within_2_to_minus_48_turns():
    rng = random.Random(12)
    worst = 0.0
    for _ in range(150):
        qa, qb = coefficients(rng)
        for _ in range(4):
            # the column passes' runs: R = 32 elements D = N1 L / 32 apart, centred on the thread's element
            D = (1 << rng.randint(8, 13)) * ((1 << rng.randint(8, 11)) // 32)
            k_first = rng.randint(-(1 << 24), (1 << 24) - 32 * D)
            for s, t in enumerate(run(k_first, D, qa, qb, 32)):
                worst = max(worst, abs(error_ulp(t, k_first + s * D, qa, qb)))
    assert worst < 2.0 ** 16  # 2^-48 turns
    # the bound: the direct values' errors spread over less than 3 ulp, times the
    # positive part of the cubic extrapolation weights at the run's last value
    w = [math.prod(31 - j for j in range(4) if j != i) / math.prod(i - j for j in range(4) if j != i)
         for i in range(4)]
    assert sum(x for x in w if x > 0) == 17081 and 3 * 17081 < 2.0 ** 16


def expi_turns_poly(th):
    """The kernels' exp(2 pi i theta), in FP64: quarter turn, residual, series, rotation."""
    q = ((th + (1 << 61)) & M64) >> 62
    r = (th - (q << 62)) & M64
    d = (r - (1 << 64) if r >= 1 << 63 else r) >> 32
    x = d * 2 * math.pi * 2.0 ** -32
    x2 = x * x
    c = 1 + x2 * (-0.5 + x2 * (1 / 24 + x2 * (-1 / 720 + x2 / 40320)))
    s = x + x * x2 * (-1 / 6 + x2 * (1 / 120 + x2 * (-1 / 5040 + x2 / 362880)))
    if q & 1:
        c, s = -s, c
    if q & 2:
        c, s = -c, -s
    return complex(c, s), q, d


@pytest.mark.parametrize("seed", [0, 1])
def test_quarter_turn_split_and_series(seed):
    rng = random.Random(seed)
    ths = [rng.getrandbits(64) for _ in range(4000)] + [0, M64, 1 << 62, (1 << 61) - 1, 1 << 61, 1 << 63]
    for th in ths:
        z, q, d = expi_turns_poly(th)
        assert abs(d) <= 1 << 29
        # q/4 + d 2^-32 turns reproduces theta up to the dropped bits (< 2^-32 turn)
        err = (Fraction(th, 1 << 64) - Fraction(q, 4) - Fraction(d, 1 << 32)) % 1
        assert min(err, 1 - err) < Fraction(1, 1 << 32)
        ang = 2 * math.pi * th / 2.0 ** 64
        assert abs(z - complex(math.cos(ang), math.sin(ang))) < 2.5e-8 + 2 * math.pi * 2.0 ** -32 + 1e-12
    # the series' first dropped terms at |x| = pi/4
    assert (math.pi / 4) ** 10 / math.factorial(10) < 2.5e-8
    assert (math.pi / 4) ** 11 / math.factorial(11) < 1.8e-9


def _series(mp, x, last_cos, last_sin):
    c = sum((-1) ** k * x ** (2 * k) / mp.factorial(2 * k) for k in range(last_cos // 2 + 1))
    s = sum((-1) ** k * x ** (2 * k + 1) / mp.factorial(2 * k + 1) for k in range(last_sin // 2 + 1))
    return c, s


def test_series_truncation_bounds():
    """The truncation errors stated for the phase series (|x| <= pi/4, through
    x^8 and x^9) and for the split-step's Kerr series (|phi| <= 1/16, through
    phi^8/phi^9 in FP64 and phi^4/phi^5 in FP32; sin relative), at 200-bit
    precision."""
    mp = pytest.importorskip("mpmath").mp
    mp.prec = 200
    cases = [(mp.pi / 4, 8, 9, 2.5e-8, 1.8e-9, False),
             (mp.mpf(1) / 16, 8, 9, 2.6e-19, 2.3e-20, True),
             (mp.mpf(1) / 16, 4, 5, 8.3e-11, 1.2e-11, True)]
    for xmax, lc, ls, bound_c, bound_s, rel_sin in cases:
        worst_c = worst_s = mp.mpf(0)
        for i in range(1, 257):
            x = xmax * i / 256
            c, s = _series(mp, x, lc, ls)
            worst_c = max(worst_c, abs(c - mp.cos(x)))
            worst_s = max(worst_s, abs(s - mp.sin(x)) / (mp.sin(x) if rel_sin else 1))
        assert worst_c < bound_c and worst_s < bound_s, (xmax, lc, worst_c, worst_s)
