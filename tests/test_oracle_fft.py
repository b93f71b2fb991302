"""Pins of the oracle's own FFT: brute-force DFT, numpy, Parseval and the
sign convention of the Fourier transform defined after Eq. (1)."""
import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import random_field


def brute_dft(x, sign):
    n = len(x)
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        acc = 0j
        for j in range(n):
            acc += x[j] * complex(np.cos(2 * np.pi * k * j / n), sign * np.sin(2 * np.pi * k * j / n))
        out[k] = acc
    return out if sign > 0 else out / n


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [+1, -1])
def test_fft_matches_bruteforce_dft(N, sign):
    x = random_field(N, seed=N + (sign > 0))
    got = oracle.fft(x, sign)
    ref = brute_dft(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N", [128, 1024, 1 << 14])
def test_fft_matches_library(N):
    x = random_field(N, seed=7)
    # paper's forward transform uses exp(+i w t): numpy's ifft * N
    np.testing.assert_allclose(oracle.fft(x, +1), np.fft.ifft(x) * N, rtol=0, atol=1e-12 * np.sqrt(N) * 4)
    np.testing.assert_allclose(oracle.fft(x, -1), np.fft.fft(x) / N, rtol=0, atol=1e-14 * 4)


def test_round_trip_and_parseval():
    N = 4096
    x = random_field(N, seed=3)
    X = oracle.fft(x, +1)
    assert abs(np.vdot(X, X).real / N - np.vdot(x, x).real) <= 1e-12 * np.vdot(x, x).real
    assert np.max(np.abs(oracle.fft(X, -1) - x)) <= 1e-14 * 8


def test_sign_convention_places_carrier_at_positive_omega():
    # A(t) = exp(-i w0 t) transforms to 2 pi delta(w - w0) under exp(+i w t):
    # with w_k = 2 pi k'/T the peak must sit at k' = +m.
    N, T = 256, 10.0
    t = np.arange(N) * T / N
    for m in (3, -5, 17):
        X = oracle.fft(np.exp(-2j * np.pi * m * t / T), +1)
        k = int(np.argmax(np.abs(X)))
        kp = k if k < N // 2 else k - N
        assert kp == m
        assert abs(abs(X[k]) - N) < 1e-9


def test_derivative_maps_to_minus_i_omega():
    # F[dA/dt] = -i w F[A] under the exp(+i w t) convention
    N, T = 512, 20.0
    t = np.arange(N) * T / N
    w0 = 2 * np.pi / T
    a = np.exp(np.cos(w0 * t) + 1j * np.sin(2 * w0 * t))
    da = a * (-w0 * np.sin(w0 * t) + 2j * w0 * np.cos(2 * w0 * t))
    om = 2 * np.pi * np.fft.fftfreq(N, d=T / N)
    lhs = oracle.fft(da, +1)
    rhs = -1j * om * oracle.fft(a, +1)
    assert np.max(np.abs(lhs - rhs)) <= 1e-9 * np.max(np.abs(rhs))
