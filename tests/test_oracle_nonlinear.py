"""Pins of the oracle's nonlinear part: invariants, the fundamental soliton,
second-order convergence, Picard convergence and agreement of the two
independent methods on a WDM link with loss, beta3 and amplifiers."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import FiberMap, Segment, chirped_gaussian, dm_map, wdm_field


def sech_soliton(N, T, t0, P0, phase):
    t = np.arange(N) * T / N
    d = t - 0.5 * T
    return math.sqrt(P0) / np.cosh(d / t0) * np.exp(1j * phase)


def test_ss_conserves_energy_without_loss():
    # gamma = 0: the linear step is a unimodular Fourier multiplier and the
    # nonlinear step a pointwise phase rotation, so sum |A|^2 is invariant.
    N, T = 512, 200.0
    fm = FiberMap((Segment(3.0, -20.0, 0.3, 1.5), Segment(1.0, 60.0, 0.3, 1.5)), 0.0, 0.0, 10)
    A0 = chirped_gaussian(N, T, 5.0, 50.0, chirp=0.3)
    out = oracle.ss(A0, fm, T, 0.0, 20.0, 0.05)
    assert abs(np.vdot(out, out).real / np.vdot(A0, A0).real - 1.0) < 1e-13


@pytest.mark.parametrize("method", ["ss", "mpa"])
def test_fundamental_soliton_second_order(method):
    # i A_z + |b2|/2 A_tt + sigma |A|^2 A = 0 (beta2 < 0, beta3 = gamma = 0) has
    # A = sqrt(P0) sech(t/t0) exp(i sigma P0 z / 2), P0 = |b2|/(sigma t0^2).
    N, T, t0, b2, sig = 512, 40.0, 1.0, -1.0, 1.0
    P0 = abs(b2) / (sig * t0 * t0)
    z = 0.5  # half a dispersion length
    fm = FiberMap((Segment(1.0, b2, 0.0, sig),), 0.0, 0.0, 10)
    A0 = sech_soliton(N, T, t0, P0, 0.0)
    ref = sech_soliton(N, T, t0, P0, 0.5 * sig * P0 * z)
    errs = []
    for M in (2, 4, 8):
        if method == "ss":
            out = oracle.ss(A0, fm, T, 0.0, z, 0.05 / M)
        else:
            out = oracle.mpa(A0, fm, T, 0.0, z, 0.05, M, 5)
        errs.append(oracle.rel_l2(out, ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), (errs, slopes)
    assert errs[-1] < 1e-4


def test_picard_iterations_converge_geometrically_and_saturate():
    # Iterating Eq. (6) at fixed M converges to the trapezoidal fixed point;
    # the text after Eq. (7) and Fig. 3: the 4th and 5th iterations coincide
    # on the scale of the discretisation error.
    N, T = 512, 200.0
    fm = FiberMap((Segment(2.0, -20.0, 0.1, 1.3),), 0.0, 0.0, 5)
    A0 = chirped_gaussian(N, T, 6.0, 20.0, chirp=0.2)
    L, M = 2.0, 16
    outs = [oracle.mpa(A0, fm, T, 0.0, L, L, M, n) for n in range(1, 7)]
    diffs = [np.linalg.norm(outs[i + 1] - outs[i]) for i in range(5)]
    assert all(diffs[i + 1] < 0.2 * diffs[i] for i in range(4)), diffs
    ex = oracle.ss(A0, fm, T, 0.0, L, L / 2048)
    r2 = np.linalg.norm(ex - outs[3])
    assert np.linalg.norm(outs[4] - outs[3]) < 1e-3 * r2


@pytest.mark.slow
def test_mpa_and_ss_converge_to_the_same_wdm_solution():
    # Two independent discretisations of Eq. (1) (trapezoid + Picard in the
    # interaction picture vs Strang splitting) meet as dz -> 0 on a 3-channel
    # DM link with beta3, loss, a dispersion-map jump and an amplifier.  The
    # steps are small enough for the +190 ps^2/km segment to be in the
    # asymptotic O(dz^2) regime, and n_tot = 6 puts the M-independent Picard
    # term O((L/z_nl)^(n+1)) of Eq. (7) below the comparison.
    fm = dm_map(2)
    N, T = 2048, 1600.0
    A0 = wdm_field(N, T, 3, 50.0, 16, 30.0, 4.0, "qpsk", seed=11)
    z1 = 60.0
    s1 = oracle.ss(A0, fm, T, 0.0, z1, 0.02)
    s2 = oracle.ss(A0, fm, T, 0.0, z1, 0.01)
    ss_x = s2 + (s2 - s1) / 3.0
    m1 = oracle.mpa(A0, fm, T, 0.0, z1, 5.0, 250, 6)
    m2 = oracle.mpa(A0, fm, T, 0.0, z1, 5.0, 500, 6)
    mpa_x = m2 + (m2 - m1) / 3.0
    e_ss = oracle.rel_l2(s2, ss_x)
    e_mpa = oracle.rel_l2(m2, mpa_x)
    assert e_ss > 1e-7 and e_mpa > 1e-7  # the comparison is not vacuous
    assert oracle.rel_l2(mpa_x, ss_x) < 0.25 * e_ss


def test_mpa_and_split_step_agree_with_distributed_gain():
    """With a distributed gain (G = g - gamma, Eq. (1)) both discretisations
    converge to the same field: the MPA-SS difference at fine steps is far
    below the difference at coarse steps, and it shrinks like dz^2."""
    N, T = 512, 400.0
    segs = (Segment(3.0, -20.0, 0.1, 1.3, 0.05), Segment(1.0, 60.0, 0.1, 1.3, -0.03))
    fm = FiberMap(segs, 0.02, 4.0, 2)
    A0 = chirped_gaussian(N, T, 10.0, 40.0, centre_ps=200.0)
    d = []
    for M, dz in ((40, 0.1), (80, 0.05)):
        mpa = oracle.mpa(A0, fm, T, 0.0, 8.0, 4.0, M, 6)
        ss = oracle.ss(A0, fm, T, 0.0, 8.0, dz)
        d.append(oracle.rel_l2(mpa, ss))
    assert d[1] < d[0] / 3.0
    assert d[1] < 1e-3
