"""Pins of the oracle's reverse-mode gradients (MPA and split-step).

The adjoints are checked against things they do not compute themselves:
central finite differences of the forward methods, the closed-form
gradient of the exact linear flow (sigma = 0, where both methods reduce to
the Fourier multiplier exp(i beta + int G) of the text after Eq. (2)),
the exact zero gradients of a conserved quantity (the split-step of Eq. (4)
is unitary for gamma = 0), and the scaling identity of the cubic term
(sigma -> c sigma, A -> A / sqrt(c) maps every output to output / sqrt(c),
in Eq. (1) and in both discretisations).
"""
import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import FiberMap, Segment

N, T = 64, 16.0
Z = 2.0
MPA_ARGS = dict(L=0.5, M=10, n_tot=3)
SS_DZ = 0.05


def _segments(sig=(1.0, 0.7)):
    return [Segment(0.6, -1.0, 0.1, sig[0]), Segment(0.4, 2.0, 0.05, sig[1])]


def _fiber(flat=False, sig=(1.0, 0.7), gamma=0.05, z_a=1.0):
    segs = _segments(sig)
    if flat:
        return FiberMap(tuple(segs * 2), gamma, z_a, 1)
    return FiberMap(tuple(segs), gamma, z_a, 2)


def _field():
    t = (np.arange(N) - N / 2) * T / N
    return 0.6 * np.exp(-t ** 2 / 2) * np.exp(0.3j * t) + 0.4 * np.exp(-(t - 3) ** 2 / 2)


def _target():
    rng = np.random.default_rng(11)
    return 0.1 * (rng.normal(size=N) + 1j * rng.normal(size=N))


def _forward(meth, A, fib):
    if meth == "mpa":
        return oracle.mpa(A, fib, T, 0.0, Z, **MPA_ARGS)
    return oracle.ss(A, fib, T, 0.0, Z, SS_DZ)


def _adjoint(meth, A, g, fib):
    if meth == "mpa":
        return oracle.mpa_adjoint(A, g, fib, T, 0.0, Z, **MPA_ARGS)
    return oracle.ss_adjoint(A, g, fib, T, 0.0, Z, SS_DZ)


def _perturbed(P, which, d):
    segs = list(_fiber(flat=True).segments)
    s = segs[P]
    if which == "sigma":
        segs[P] = Segment(s.length_km, s.beta2_ps2_per_km, s.beta3_ps3_per_km, s.sigma_per_W_km + d)
    else:
        segs[P] = Segment(s.length_km, s.beta2_ps2_per_km + d, s.beta3_ps3_per_km, s.sigma_per_W_km)
    return FiberMap(tuple(segs), 0.05, 1.0, 1)


@pytest.mark.parametrize("meth", ["mpa", "ss"])
def test_adjoint_matches_central_differences(meth):
    A0, tgt = _field(), _target()
    fib = _fiber()

    def loss(out):
        return float(np.sum(np.abs(out - tgt) ** 2))

    out = _forward(meth, A0, fib)
    g = _adjoint(meth, A0, 2 * (out - tgt), fib)
    assert np.abs(g.out - out).max() <= 1e-14 * np.abs(out).max()
    rng = np.random.default_rng(5)
    for _ in range(2):
        v = rng.normal(size=N) + 1j * rng.normal(size=N)
        h = 1e-6 * np.linalg.norm(A0) / np.linalg.norm(v)
        fd = (loss(_forward(meth, A0 + h * v, fib)) - loss(_forward(meth, A0 - h * v, fib))) / (2 * h)
        an = float(np.real(np.vdot(g.field, v)))
        assert abs(fd - an) <= 1e-6 * abs(fd)
    # per physical segment (the periodic map's gradient vs differences of the
    # flattened map, where each physical segment is its own row); the
    # differences carry a rounding floor of about eps * l / h
    floor = 1e-8 * max(1.0, loss(out))
    for P in range(4):
        for which in ("sigma", "beta2"):
            h = 1e-6
            fd = (loss(_forward(meth, A0, _perturbed(P, which, h)))
                  - loss(_forward(meth, A0, _perturbed(P, which, -h)))) / (2 * h)
            an = (g.sigma if which == "sigma" else g.beta2)[P]
            assert abs(fd - an) <= 1e-6 * abs(fd) + floor, (which, P, fd, an)


@pytest.mark.parametrize("meth", ["mpa", "ss"])
def test_periodic_and_flat_maps_give_the_same_gradients(meth):
    A0, tgt = _field(), _target()
    out = _forward(meth, A0, _fiber())
    a = _adjoint(meth, A0, 2 * (out - tgt), _fiber())
    b = _adjoint(meth, A0, 2 * (out - tgt), _fiber(flat=True))
    # the two maps sum their segment integrals in different orders
    assert np.allclose(a.field, b.field, rtol=0, atol=1e-12)
    assert np.allclose(a.sigma, b.sigma, rtol=1e-9, atol=0)
    assert np.allclose(a.beta2, b.beta2, rtol=1e-9, atol=0)


@pytest.mark.parametrize("meth", ["mpa", "ss"])
def test_linear_limit_closed_form(meth):
    """sigma = 0: A_out = F^-1[H F[A]], H = exp(i beta(omega, 0, Z)) * G, so
    g_A = F^-1[conj(H) F[g_out]] and dl/dbeta2_P = sum_k Re(conj(gh_k) i (omega_k^2/2) len_P X_k)
    with gh = F[g_out]/N and X = H F[A]; written here with numpy's FFT."""
    fib = _fiber(sig=(0.0, 0.0))
    A0, tgt = _field(), _target()
    out = _forward(meth, A0, fib)
    g_out = 2 * (out - tgt)
    g = _adjoint(meth, A0, g_out, fib)
    kp = np.fft.fftfreq(N, d=1.0 / N)
    w = 2 * np.pi * kp / T
    segs = list(fib.segments) * fib.n_periods
    I2 = sum(s.length_km * s.beta2_ps2_per_km for s in segs)
    I3 = sum(s.length_km * s.beta3_ps3_per_km for s in segs)
    # loss gamma Z restored by the amplifiers at 1 and 2 km
    H = np.exp(1j * (w ** 2 / 2 * I2 + w ** 3 / 6 * I3))
    F = lambda x: np.fft.ifft(x) * N  # the paper's forward transform (exp(+i omega t))
    Fi = lambda X: np.fft.fft(X) / N
    assert np.allclose(out, Fi(H * F(A0)), rtol=0, atol=1e-13)
    assert np.allclose(g.field, Fi(np.conj(H) * F(g_out)), rtol=0, atol=1e-12)
    gh = F(g_out) / N
    X = H * F(A0)
    for P, s in enumerate(segs):
        want = float(np.sum(np.real(np.conj(gh) * 1j * (w ** 2 / 2) * s.length_km * X)))
        assert abs(g.beta2[P] - want) <= 1e-10 * max(1.0, abs(want))


def test_split_step_energy_gradient_is_exact():
    """gamma = 0, no amplifiers: Eq. (4)'s steps are unitary, so
    l = sum |A_out|^2 = sum |A_in|^2 for every sigma and beta2: g_A = 2 A,
    and the parameter gradients vanish."""
    fib = _fiber(gamma=0.0, z_a=0.0)
    A0 = _field()
    out = _forward("ss", A0, fib)
    g = _adjoint("ss", A0, 2 * out, fib)
    assert np.allclose(g.field, 2 * A0, rtol=0, atol=1e-12)
    assert np.abs(g.sigma).max() <= 1e-11
    assert np.abs(g.beta2).max() <= 1e-11


@pytest.mark.parametrize("meth", ["mpa", "ss"])
def test_cubic_scaling_identity(meth):
    """out(c sigma, A / sqrt(c)) = out(sigma, A) / sqrt(c) for every c; at c = 1:
    sum_P sigma_P dl/dsigma_P - Re<g_A, A>/2 = -Re<g_out, out>/2."""
    A0, tgt = _field(), _target()
    fib = _fiber()
    out = _forward(meth, A0, fib)
    g_out = 2 * (out - tgt)
    g = _adjoint(meth, A0, g_out, fib)
    sig = np.array([s.sigma_per_W_km for s in fib.segments] * fib.n_periods)
    lhs = float(sig @ g.sigma - 0.5 * np.real(np.vdot(g.field, A0)))
    rhs = float(-0.5 * np.real(np.vdot(g_out, out)))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(rhs))
