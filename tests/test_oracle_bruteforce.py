"""Tiny brute-force pin of the oracle's MPA (MPA steps 1-7, Eq. (6)).

Eq. (6) is evaluated literally with dense DFT matrices (the forward
transform with exp(+i omega t), text after Eq. (1)) on N = 8 or 16 modes
and M = 2..4 nodes, and compared with the oracle's radix-2, node-parallel
implementation.  The phases beta(w, z) = w^2/2 int beta2 + w^3/6 int beta3
(text after Eq. (2)) and the gain factor exp(int G), G = g - gamma, are
integrated segment by segment; sigma at a node on a segment boundary is the
mean of the one-sided values inside the interval and the inner value at its
ends (the composite trapezoid on each smooth piece); a lumped amplifier at
the interval end multiplies the result by exp(z_a gamma) (G of Eq. (1))."""
import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import FiberMap, Segment


def dft_matrices(N):
    n = np.arange(N)
    F = np.exp(2j * np.pi * np.outer(n, n) / N)  # F[x]_k = sum_n x_n e^{+2 pi i k n / N}
    return F, np.conj(F) / N


def omegas(N, T):
    k = np.arange(N)
    return 2 * np.pi * np.where(k < N // 2, k, k - N) / T


def integral(fib, za, zb, f):
    """int_za^zb f(segment) dz over the periodic map, piece by piece."""
    out, a = 0.0, 0.0
    for p in range(fib.n_periods):
        for s in fib.segments:
            b = a + s.length_km
            lo, hi = max(a, za), min(b, zb)
            if hi > lo:
                out += f(s) * (hi - lo)
            a = b
    return out


def sigma_at(fib, z, z0, z1):
    """sigma(z_j): one-sided values at a boundary, averaged inside (z0, z1)."""
    eps = 1e-9
    left = [s for s in _pieces(fib) if s[0] < z - eps / 2 <= s[1]]
    right = [s for s in _pieces(fib) if s[0] <= z + eps / 2 < s[1]]
    sl, sr = left[0][2].sigma_per_W_km if left else None, right[0][2].sigma_per_W_km if right else None
    if abs(z - z0) < eps:
        return sr
    if abs(z - z1) < eps:
        return sl
    return 0.5 * (sl + sr)


def _pieces(fib):
    a = 0.0
    for p in range(fib.n_periods):
        for s in fib.segments:
            yield (a, a + s.length_km, s)
            a += s.length_km


def brute_mpa(A0, fib, T, z0, L, M, n_tot, psi_last=False):
    """Steps 1-7 with dense matrices; psi_last=True returns psi^{(n_tot)} at
    node M (natural frequency order) instead, before step 7."""
    N = A0.size
    F, Fi = dft_matrices(N)
    w = omegas(N, T)
    dz = L / M
    z = z0 + dz * np.arange(M + 1)
    z[M] = z0 + L

    def beta(zz):
        b2 = integral(fib, z0, zz, lambda s: s.beta2_ps2_per_km)
        b3 = integral(fib, z0, zz, lambda s: s.beta3_ps3_per_km)
        return w ** 2 / 2 * b2 + w ** 3 / 6 * b3

    def intG(zz):
        return integral(fib, z0, zz, lambda s: s.gain_per_km - fib.gamma_per_km)

    psi0 = F @ A0                                  # step 1: A_hat(z0)
    psi = np.tile(psi0, (M + 1, 1))                # psi^{(0)}_j = psi_0
    for _ in range(n_tot):                         # step 6
        V = np.empty_like(psi)
        for j in range(M + 1):
            Ahat = psi[j] * np.exp(1j * beta(z[j]) + intG(z[j]))      # step 2
            A = Fi @ Ahat                                             # step 3
            U = np.abs(A) ** 2 * A                                    # step 4
            V[j] = sigma_at(fib, z[j], z0, z0 + L) * dz * (F @ U) * np.exp(-1j * beta(z[j]) - intG(z[j]))
        new = np.empty_like(psi)                   # step 5: the trapezoid of Eq. (6)
        new[0] = psi0
        for l in range(1, M + 1):
            new[l] = psi0 + 1j * (V[0] / 2 + V[1:l].sum(axis=0) + V[l] / 2)
        psi = new
    if psi_last:
        return psi[M]
    out = psi[M] * np.exp(1j * beta(z0 + L) + intG(z0 + L))        # step 7
    k_end = (z0 + L) / fib.z_a_km
    if abs(k_end - round(k_end)) < 1e-9 and round(k_end) >= 1:
        out = out * np.exp(fib.z_a_km * fib.gamma_per_km)          # lumped gain at z_k
    return Fi @ out


CASES = {
    # one segment, interval inside the span (no amplifier), distributed gain
    "uniform": (FiberMap((Segment(4.0, -1.3, 0.12, 1.1, 0.02),), 0.05, 4.0, 1), 16, 8.0, 0.0, 2.0, 3, 2),
    # two segments, the boundary on node 2 of 4, the interval ends at the amplifier
    "boundary_on_node": (FiberMap((Segment(1.0, -1.0, 0.1, 1.2), Segment(1.0, 2.0, -0.05, 0.8, 0.03)), 0.07, 2.0, 2),
                         16, 8.0, 0.0, 2.0, 4, 3),
    # the same map, the boundary between nodes (M = 3), a later interval
    "boundary_between_nodes": (FiberMap((Segment(1.0, -1.0, 0.1, 1.2), Segment(1.0, 2.0, -0.05, 1.2, 0.03)), 0.07,
                                        2.0, 2), 8, 6.0, 2.0, 2.0, 3, 2),
    # a single node step (M = 2) at n_tot = 1
    "one_level": (FiberMap((Segment(3.0, 0.8, 0.0, 0.9),), 0.0, 3.0, 1), 8, 6.0, 0.0, 1.5, 2, 1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_mpa_equals_literal_eq6(case):
    fib, N, T, z0, L, M, n_tot = CASES[case]
    rng = np.random.default_rng(7)
    A0 = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * 0.6
    ref = brute_mpa(A0, fib, T, z0, L, M, n_tot)
    got = oracle.mpa(A0, fib, T, z0, z0 + L, L, M, n_tot)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    # the nonlinear part is not negligible: the linear flow alone is far off
    lin = brute_mpa(A0, FiberMap(tuple(Segment(s.length_km, s.beta2_ps2_per_km, s.beta3_ps3_per_km, 0.0,
                                               s.gain_per_km) for s in fib.segments),
                                 fib.gamma_per_km, fib.z_a_km, fib.n_periods), T, z0, L, M, n_tot)
    assert np.linalg.norm(got - lin) / np.linalg.norm(ref) > 1e-3


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_mpa_interval_equals_literal_eq6(case):
    """The exported single-interval entry (steps 2-6 from a given spectrum,
    no step 7), which the full-size GPU parity tests compare against, equals
    the dense evaluation of Eq. (6) at node M."""
    fib, N, T, z0, L, M, n_tot = CASES[case]
    rng = np.random.default_rng(7)
    A0 = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * 0.6
    F, _ = dft_matrices(N)
    ref = brute_mpa(A0, fib, T, z0, L, M, n_tot, psi_last=True)
    got = oracle.mpa_interval(F @ A0, fib, T, z0, L, M, n_tot)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def step7(psiM, fib, T, z0, L):
    """Step 7 written out with numpy: A(z0+L) = F^-1[psi_M exp(i beta(w, L)
    + int G)], times exp(z_a gamma) when z0+L is an amplifier location."""
    N = psiM.size
    w = omegas(N, T)
    b2 = integral(fib, z0, z0 + L, lambda s: s.beta2_ps2_per_km)
    b3 = integral(fib, z0, z0 + L, lambda s: s.beta3_ps3_per_km)
    G = integral(fib, z0, z0 + L, lambda s: s.gain_per_km - fib.gamma_per_km)
    out = psiM * np.exp(1j * (w ** 2 / 2 * b2 + w ** 3 / 6 * b3) + G)
    k_end = (z0 + L) / fib.z_a_km
    if abs(k_end - round(k_end)) < 1e-9 and round(k_end) >= 1:
        out = out * np.exp(fib.z_a_km * fib.gamma_per_km)
    return np.fft.fft(out) / N  # F^-1 with the exp(+i w t) forward sign: (1/N) sum_k X_k e^{-2 pi i kn/N}


@pytest.mark.parametrize("N,M,n_tot,z0", [(1 << 10, 8, 2, 0.0), (1 << 12, 12, 3, 5.0), (1 << 9, 5, 1, 45.0)])
def test_oracle_mpa_interval_then_step7_equals_oracle_mpa(N, M, n_tot, z0):
    """oracle.mpa_interval followed by step 7 in numpy reproduces oracle.mpa
    over that interval on the benchmark DM map (natural frequency order in,
    interval start z0 anywhere in the span, including the interval that ends
    at the amplifier)."""
    from paper_1101_0086_gb300.workloads import dm_map, wdm_field
    fib = dm_map(2)
    T = 100.0 * N / 256
    L = 5.0
    A0 = wdm_field(N, T, 2, 50.0, N // 256, 30.0, 2.0, "qpsk", seed=N + M)
    ref = oracle.mpa(A0, fib, T, z0, z0 + L, L, M, n_tot)
    psi0 = N * np.fft.ifft(A0)  # F[A]_k = sum_n A_n e^{+2 pi i kn/N}
    got = step7(oracle.mpa_interval(psi0, fib, T, z0, L, M, n_tot), fib, T, z0, L)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    # the nonlinear correction itself (beyond the linear flow) is what matches
    lin = step7(psi0, fib, T, z0, L)
    assert np.linalg.norm(ref - lin) / np.linalg.norm(ref) > 1e-5


def brute_ss(A0, fib, T, z_from, z_to, dz):
    """Eq. (4) as Strang splitting, literally: a half linear step, then per
    step a Kerr rotation exp(i |A|^2 int sigma) and a full linear step (the
    last one a half step); each linear step is the exact multiplier
    exp(i beta + int G) times exp(z_a gamma) for every amplifier z_k in its
    range (a, b]."""
    N = A0.size
    F, Fi = dft_matrices(N)
    w = omegas(N, T)
    K = int(round((z_to - z_from) / dz))

    def lin(X, a, b):
        b2 = integral(fib, a, b, lambda s: s.beta2_ps2_per_km)
        b3 = integral(fib, a, b, lambda s: s.beta3_ps3_per_km)
        G = integral(fib, a, b, lambda s: s.gain_per_km - fib.gamma_per_km)
        n_amp = sum(1 for k in range(1, 10 * fib.n_periods + 2) if a < k * fib.z_a_km <= b + 1e-12)
        return X * np.exp(1j * (w ** 2 / 2 * b2 + w ** 3 / 6 * b3) + G + n_amp * fib.z_a_km * fib.gamma_per_km)

    X = F @ A0
    a, b = z_from, z_from + dz / 2
    X = lin(X, a, b)
    for k in range(K):
        A = Fi @ X
        S = integral(fib, z_from + k * dz, z_from + (k + 1) * dz, lambda s: s.sigma_per_W_km)
        A = A * np.exp(1j * S * np.abs(A) ** 2)
        X = F @ A
        a, b = b, (z_to if k == K - 1 else b + dz)
        X = lin(X, a, b)
    return Fi @ X


SS_CASES = {
    # a segment boundary inside a step (sigma differs), distributed gain, an
    # amplifier inside a linear step (z = 2) and one at the end (z = 4)
    "two_spans": (FiberMap((Segment(1.3, -1.0, 0.1, 1.2), Segment(0.7, 2.0, -0.05, 0.8, 0.03)), 0.07, 2.0, 2),
                  16, 8.0, 0.0, 4.0, 0.5),
    # a later stretch that ends between amplifiers, one segment type
    "inside_a_span": (FiberMap((Segment(3.0, 0.8, 0.0, 0.9),), 0.05, 3.0, 2), 8, 6.0, 1.5, 4.5, 0.25),
}


@pytest.mark.parametrize("case", sorted(SS_CASES))
def test_oracle_ss_equals_literal_eq4(case):
    fib, N, T, z0, z1, dz = SS_CASES[case]
    rng = np.random.default_rng(11)
    A0 = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * 0.6
    ref = brute_ss(A0, fib, T, z0, z1, dz)
    got = oracle.ss(A0, fib, T, z0, z1, dz)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
