"""Pins of the seeded input generator shared by the CUDA path and the oracle.

The field recipe is demodulated channel by channel: after undoing channel c's
carrier, a low-pass filter of half the channel spacing leaves that channel's
pulse train alone. Its samples at the slot centres must then carry the
recipe's symbols: quarter-turn phases of one amplitude for QPSK, that
amplitude or nothing for OOK. The amplitude is sqrt(peak power). The fiber
map helper must give a span loss that the lumped amplifier restores
exactly.
"""
import math

import numpy as np
import pytest

from paper_1101_0086_gb300.workloads import WORKLOADS, dm_map, gamma_from_db_per_km, wdm_field

N, T, CH, SPACING, NSYM, FWHM, PEAK = 1 << 12, 1280.0, 4, 100.0, 8, 30.0, 2.0  # 160-ps slots: tails < 1e-17


def channel_samples(field, c):
    """Channel c's complex envelope at the slot centres."""
    t = np.arange(N) * T / N
    fc = (c - 0.5 * (CH - 1)) * SPACING * 1e-3
    base = field * np.exp(2j * math.pi * fc * t)          # undo exp(-2 pi i f_c t)
    f = np.fft.fftfreq(N, d=T / N)
    base = np.fft.ifft(np.fft.fft(base) * (np.abs(f) < 0.5 * SPACING * 1e-3))
    spp = N // NSYM
    return base[np.arange(NSYM) * spp + spp // 2]


@pytest.mark.parametrize("seed", [0, 1, 7])
def test_qpsk_channels_carry_quarter_turn_symbols_at_the_peak_amplitude(seed):
    A = wdm_field(N, T, CH, SPACING, NSYM, FWHM, PEAK, "qpsk", seed)
    amp = math.sqrt(PEAK * 1e-3)
    for c in range(CH):
        s = channel_samples(A, c)
        np.testing.assert_allclose(np.abs(s), amp, rtol=1e-6)
        q = np.angle(s) / (0.5 * math.pi)
        np.testing.assert_allclose(q, np.round(q), atol=1e-6)
    # the spectrum's weight sits at +f_c (exp(+i w t) transform: numpy ifft * N)
    spec = np.abs(np.fft.ifft(A)) ** 2
    f = np.fft.fftfreq(N, d=T / N)
    for c in range(CH):
        fc = (c - 0.5 * (CH - 1)) * SPACING * 1e-3
        near = np.abs(f - fc) < 0.5 * SPACING * 1e-3
        assert spec[near].sum() > 0.24 * spec.sum()


def test_ook_channels_are_on_off_and_seeded():
    A = wdm_field(N, T, CH, SPACING, NSYM, FWHM, PEAK, "ook", 3)
    amp = math.sqrt(PEAK * 1e-3)
    ones = 0
    for c in range(CH):
        s = np.abs(channel_samples(A, c))
        on = s > 0.5 * amp
        np.testing.assert_allclose(s[on], amp, rtol=1e-6)
        assert np.all(s[~on] < 1e-6 * amp)
        ones += int(on.sum())
    assert 0 < ones < CH * NSYM
    np.testing.assert_array_equal(A, wdm_field(N, T, CH, SPACING, NSYM, FWHM, PEAK, "ook", 3))
    assert not np.array_equal(A, wdm_field(N, T, CH, SPACING, NSYM, FWHM, PEAK, "ook", 4))


def test_recipe_rejects_off_grid_inputs():
    with pytest.raises(ValueError):
        wdm_field(N, T, CH, SPACING, 24, FWHM, PEAK, "qpsk", 0)  # N not a multiple of the symbols
    with pytest.raises(ValueError):
        wdm_field(N, 1000.0, CH, 33.0, NSYM, FWHM, PEAK, "qpsk", 0)  # carriers off the 1/T grid
    with pytest.raises(ValueError):
        wdm_field(N, T, CH, SPACING, NSYM, FWHM, PEAK, "16qam", 0)


def test_dm_span_loss_is_restored_by_the_amplifier():
    fib = dm_map(3)
    assert fib.period_km == 50.0 and fib.z_a_km == 50.0 and fib.length_km == 150.0
    # 0.2 dB/km power loss: exp(-2 gamma z) = 10^(-0.02 z); the gain exp(z_a gamma) undoes one span
    assert math.exp(-2 * fib.gamma_per_km * 50.0) == pytest.approx(10 ** (-1.0), rel=1e-12)
    assert gamma_from_db_per_km(0.2) == fib.gamma_per_km
    (s1, s2) = fib.segments
    assert (s1.length_km, s1.beta2_ps2_per_km, s2.length_km, s2.beta2_ps2_per_km) == (45.0, -21.7, 5.0, 190.0)


@pytest.mark.parametrize("key", sorted(WORKLOADS))
def test_named_workloads_lie_on_their_grids(key):
    w = WORKLOADS[key]()
    assert w.N & (w.N - 1) == 0 and w.N % w.n_symbols == 0
    for c in range(w.n_channels):
        cycles = (c - 0.5 * (w.n_channels - 1)) * w.spacing_GHz * 1e-3 * w.T_ps
        assert abs(cycles - round(cycles)) < 1e-9
    # every interval boundary and amplifier on the MPA grid; the split-step step divides the span
    assert w.fiber.period_km % w.mpa_L_km == 0 or w.mpa_L_km % w.fiber.period_km == 0
    assert abs(w.fiber.z_a_km / w.ss_dz_km - round(w.fiber.z_a_km / w.ss_dz_km)) < 1e-9
    # the band fits the window's Nyquist range with room for the pulses' spectra
    f_nyq = 0.5 * w.N / w.T_ps
    f_edge = 0.5 * (w.n_channels - 1) * w.spacing_GHz * 1e-3
    assert f_edge + 5.0 / w.fwhm_ps < f_nyq
