"""Pins of the oracle's linear part: with sigma = 0 the interaction-picture
spectrum is constant (text after Eq. (2)), so both methods must reproduce the
exact linear flow A_hat(z) = A_hat(0) exp(i beta(w, z) - gamma z) times the
amplifier gains.  The sign of each dispersion term is pinned separately by
textbook pulse-propagation results."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import FiberMap, Segment, chirped_gaussian, gamma_from_db_per_km


def omega_grid(N, T):
    return 2 * np.pi * np.fft.fftfreq(N, d=T / N)


def closed_form_linear(A0, T, I2, I3, gain):
    """exp(i (w^2/2 I2 + w^3/6 I3)) * gain applied with numpy's FFT
    (numpy ifft*N is the exp(+i w t) transform)."""
    N = len(A0)
    w = omega_grid(N, T)
    X = np.fft.ifft(A0) * N
    X = X * np.exp(1j * (0.5 * w**2 * I2 + w**3 * I3 / 6.0)) * gain
    return np.fft.fft(X) / N


def test_sigma_zero_matches_exact_linear_flow_across_amplifiers():
    N, T = 1024, 400.0
    segs = (Segment(45.0, -21.7, 0.1, 0.0), Segment(5.0, 190.0, 0.1, 0.0))
    g = gamma_from_db_per_km(0.2)
    fm = FiberMap(segs, g, 50.0, 4)
    A0 = chirped_gaussian(N, T, 8.0, 1.0, chirp=-0.7, centre_ps=150.0)
    z1 = 130.0
    # int beta2, beta3 over [0, 130]: two full spans + 30 km of the first segment
    I2 = 2 * (45.0 * -21.7 + 5.0 * 190.0) + 30.0 * -21.7
    I3 = 130.0 * 0.1
    gain = math.exp(-g * z1) * math.exp(2 * 50.0 * g)  # amplifiers at 50 and 100 km
    ref = closed_form_linear(A0, T, I2, I3, gain)
    ss = oracle.ss(A0, fm, T, 0.0, z1, 1.0)
    mpa = oracle.mpa(A0, fm, T, 0.0, z1, 10.0, 7, 3)
    assert oracle.rel_l2(ss, ref) < 1e-12
    assert oracle.rel_l2(mpa, ref) < 1e-12


def test_amplifier_restores_span_loss():
    N, T = 256, 200.0
    g = gamma_from_db_per_km(0.2)
    fm = FiberMap((Segment(50.0, 0.0, 0.0, 0.0),), g, 50.0, 2)
    A0 = chirped_gaussian(N, T, 10.0, 1.0)
    # exactly at an amplifier the field is restored; just before it it is down 10 dB
    np.testing.assert_allclose(oracle.mpa(A0, fm, T, 0.0, 50.0, 50.0, 4, 1), A0, atol=1e-14)
    before = oracle.mpa(A0, fm, T, 0.0, 49.0, 49.0, 4, 1)
    assert abs(np.vdot(before, before).real / np.vdot(A0, A0).real - 10 ** (-0.1 * 49 * 0.2 / 1.0)) < 1e-12


def rms_width_and_centroid(A, T):
    N = len(A)
    t = np.arange(N) * T / N
    p = np.abs(A) ** 2
    c = np.sum(t * p) / np.sum(p)
    return math.sqrt(np.sum((t - c) ** 2 * p) / np.sum(p)), c


@pytest.mark.parametrize("C", [-2.0, 0.0, 1.5])
def test_beta2_sign_chirped_gaussian_width(C):
    # Textbook (Agrawal, Nonlinear Fiber Optics, Sec. 3.2, same NLSE sign):
    # a chirped Gaussian exp(-(1+iC) t^2/(2 t0^2)) has width ratio
    # sqrt((1 + C b2 z/t0^2)^2 + (b2 z/t0^2)^2).
    N, T, t0, b2, z = 2048, 400.0, 6.0, -20.0, 1.5
    fm = FiberMap((Segment(10.0, b2, 0.0, 0.0),), 0.0, 0.0, 1)
    A0 = chirped_gaussian(N, T, t0, 1.0, chirp=C)
    out = oracle.ss(A0, fm, T, 0.0, z, z)
    w0, _ = rms_width_and_centroid(A0, T)
    w1, _ = rms_width_and_centroid(out, T)
    xi = b2 * z / t0**2
    assert abs(w1 / w0 - math.sqrt((1 + C * xi) ** 2 + xi**2)) < 1e-9


def test_beta3_sign_delays_centroid():
    # Group delay d beta/d w = beta3 w^2 z/2 >= 0: every component is delayed
    # (F[A(t - t0)] = exp(+i w t0) F[A] under exp(+i w t)), so the centroid of
    # a Gaussian with |A_hat|^2 ~ exp(-w^2 t0^2) moves by beta3 z /(4 t0^2).
    N, T, t0, b3, z = 4096, 400.0, 3.0, 0.5, 10.0
    fm = FiberMap((Segment(10.0, 0.0, b3, 0.0),), 0.0, 0.0, 1)
    A0 = chirped_gaussian(N, T, t0, 1.0)
    out = oracle.mpa(A0, fm, T, 0.0, z, z, 2, 1)
    _, c0 = rms_width_and_centroid(A0, T)
    _, c1 = rms_width_and_centroid(out, T)
    assert abs((c1 - c0) - b3 * z / (4 * t0**2)) < 1e-9


def test_inconsistent_grids_are_rejected():
    N, T = 64, 100.0
    fm = FiberMap((Segment(5.0, -1.0, 0.0, 1.0),), 0.0, 50.0, 20)
    A0 = chirped_gaussian(N, T, 5.0, 1.0)
    with pytest.raises(ValueError):
        oracle.mpa(A0, fm, T, 0.0, 60.0, 40.0, 4, 1)  # amplifier at 50 km inside an interval
    with pytest.raises(ValueError):
        oracle.mpa(A0, fm, T, 0.0, 10.0, 3.0, 4, 1)  # 10 km is not a whole number of intervals
    with pytest.raises(ValueError):
        oracle.ss(A0, fm, T, 0.0, 200.0, 1.0)  # beyond the end of the link
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12), +1)  # N not a power of two


def test_fine_intervals_ending_on_amplifiers_are_accepted():
    """Intervals much shorter than the tolerance of the amplifier count
    (L < 1e-3 z_a) that end exactly on amplifiers are valid grids: with
    sigma = 0 the MPA reproduces the exact linear flow with both lumped
    gains, while the same fine grid shifted by L/2 (an amplifier strictly
    inside an interval) is still rejected."""
    N, T = 64, 100.0
    g = gamma_from_db_per_km(0.2)
    fm = FiberMap((Segment(5.0, -1.0, 0.05, 0.0),), g, 50.0, 20)
    A0 = chirped_gaussian(N, T, 5.0, 1.0)
    L = 50.0 / 1024
    out = oracle.mpa(A0, fm, T, 0.0, 100.0, L, 1, 1)
    ref = closed_form_linear(A0, T, 100.0 * -1.0, 100.0 * 0.05, math.exp(-g * 100.0) * math.exp(2 * 50.0 * g))
    assert oracle.rel_l2(out, ref) < 1e-12
    with pytest.raises(ValueError):
        oracle.mpa(A0, fm, T, 0.5 * L, 100.0 - 0.5 * L, L, 1, 1)


def test_distributed_gain_linear_flow_and_energy():
    """A distributed gain g on a segment enters G = g - gamma (Eq. (1)): with
    sigma = 0 both methods give the closed-form flow times exp(int G), and
    with sigma != 0, gamma = 0 and no lumped amplifiers the split-step (a
    unitary linear step times exp(int g), a modulus-preserving kick) scales
    the energy by exactly exp(2 int g)."""
    N, T = 1024, 400.0
    g = gamma_from_db_per_km(0.2)
    segs = (Segment(45.0, -21.7, 0.1, 0.0, 0.03), Segment(5.0, 190.0, 0.1, 0.0, -0.01))
    fm = FiberMap(segs, g, 50.0, 4)
    A0 = chirped_gaussian(N, T, 8.0, 1.0, chirp=-0.7, centre_ps=150.0)
    z1 = 130.0
    I2 = 2 * (45.0 * -21.7 + 5.0 * 190.0) + 30.0 * -21.7
    I3 = 130.0 * 0.1
    Ig = 2 * (45.0 * 0.03 + 5.0 * -0.01) + 30.0 * 0.03
    gain = math.exp(-g * z1 + Ig) * math.exp(2 * 50.0 * g)
    ref = closed_form_linear(A0, T, I2, I3, gain)
    assert oracle.rel_l2(oracle.ss(A0, fm, T, 0.0, z1, 1.0), ref) < 1e-12
    assert oracle.rel_l2(oracle.mpa(A0, fm, T, 0.0, z1, 10.0, 7, 3), ref) < 1e-12
    segs = (Segment(3.0, -20.0, 0.1, 1.3, 0.04), Segment(1.0, 60.0, 0.1, 1.3, -0.02))
    fm = FiberMap(segs, 0.0, 0.0, 3)
    A1 = chirped_gaussian(N, T, 8.0, 30.0, centre_ps=200.0)
    out = oracle.ss(A1, fm, T, 0.0, 10.0, 0.05)
    Ig = 2 * (3.0 * 0.04 - 1.0 * 0.02) + 2.0 * 0.04
    ratio = np.vdot(out, out).real / np.vdot(A1, A1).real
    assert abs(ratio / math.exp(2 * Ig) - 1) < 1e-12
