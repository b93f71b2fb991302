"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs.  Tolerances (relative L2): 1e-10 for FP64
runs and 1e-4 for FP32 runs against the same algorithm's FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import (FiberMap, Segment, chirped_gaussian, dm_map, random_field, wdm_field,
                                             workload)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_1101_0086_gb300 import build as B
    from paper_1101_0086_gb300 import mpa
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    mpa.lib()
    return mpa


def dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64 if prec == "fp32" else np.complex128)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("logn", [8, 9, 12, 13, 14, 17, 20])
@pytest.mark.parametrize("sign", [+1, -1])
def test_fft_matches_oracle(M, prec, logn, sign):
    N = 1 << logn
    x = random_field(N, seed=logn)
    ref = oracle.fft(x, sign)
    got = host(M.fft(dev(x, prec), sign))
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert oracle.rel_l2(got, ref) < tol


# ------------------------------------------------------------- intervals
def small_map(sigma=1.3, gamma_db=0.2):
    # two segments with a dispersion jump, beta3 and loss; period 10 km
    from paper_1101_0086_gb300.workloads import gamma_from_db_per_km
    return FiberMap((Segment(8.0, -21.7, 0.1, sigma), Segment(2.0, 85.0, 0.1, sigma)),
                    gamma_from_db_per_km(gamma_db), 10.0, 10)


@pytest.mark.parametrize("prec,schedule", [("fp32", "level"), ("fp32", "wavefront"), ("fp64", "auto")])
@pytest.mark.parametrize("N,Lk,Mn,n_iter,z0", [
    (1 << 10, 10.0, 20, 3, 0.0),      # one interval = one DM period (node on the 8 km jump)
    (1 << 12, 2.0, 36, 3, 8.0),       # ragged node batch, interval in the +85 segment
    (1 << 12, 5.0, 1, 1, 5.0),        # degenerate: M = 1, one iteration
    (1 << 14, 10.0, 50, 4, 20.0),     # several tiles per node, interval type 0 of period 3
    (1 << 14, 2.0, 37, 1, 4.0),       # one iteration (wavefront: a single slot)
    (1 << 16, 5.0, 45, 5, 0.0),       # five iterations, ragged last block
])
def test_interval_matches_oracle(M, prec, schedule, N, Lk, Mn, n_iter, z0):
    fib = small_map()
    T = 800.0 * N / 1024
    A0 = wdm_field(N, T, 2, 50.0, 8 * N // 1024, 30.0, 20.0, "qpsk", seed=N + Mn)
    psi0 = oracle.fft(A0, +1)
    ref = oracle.mpa_interval(psi0, fib, T, z0, Lk, Mn, n_iter)
    if schedule == "wavefront" and N < (1 << 14):
        schedule = "level"  # the wavefront needs N >= 2^14
    plan = M.Plan(fib, N, T, Lk, Mn, n_iter, precision=prec, schedule=schedule)
    got = host(plan.interval(dev(psi0, "fp64"), z0))
    err = oracle.rel_l2(got, ref)
    assert err < TOL[prec], err
    # the nonlinear correction is what the kernels compute: compare it too
    dref = ref - psi0
    assert oracle.rel_l2(got - psi0, dref) < (1e-9 if prec == "fp64" else 3e-3)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_propagate_matches_oracle_across_amplifiers(M, prec):
    fib = small_map()
    N, T = 1 << 12, 3200.0
    A0 = wdm_field(N, T, 3, 50.0, 32, 30.0, 10.0, "qpsk", seed=5)
    ref = oracle.mpa(A0, fib, T, 0.0, 30.0, 2.0, 24, 3)
    plan = M.Plan(fib, N, T, 2.0, 24, 3, precision=prec)
    got = host(plan.propagate(dev(A0, prec), 0.0, 30.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    assert plan.status()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fine_intervals_ending_on_amplifiers(M, prec):
    # L = z_a / 1024, below the tolerance of the amplifier count: 2048
    # intervals, two of which end on an amplifier, are a valid grid
    fib = small_map()
    N, T = 1 << 10, 800.0
    A0 = wdm_field(N, T, 2, 50.0, 16, 30.0, 10.0, "qpsk", seed=7)
    L = 10.0 / 1024
    ref = oracle.mpa(A0, fib, T, 0.0, 20.0, L, 2, 2)
    plan = M.Plan(fib, N, T, L, 2, 2, precision=prec)
    got = host(plan.propagate(dev(A0, prec), 0.0, 20.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    assert plan.status()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_linear_limit_is_exact(M, prec):
    # sigma = 0: psi is constant (text after Eq. (2)); the result is the exact
    # linear flow, computed here with numpy's FFT
    fib = small_map(sigma=0.0)
    N, T = 1 << 13, 6400.0
    A0 = chirped_gaussian(N, T, 15.0, 1.0, chirp=0.3)
    plan = M.Plan(fib, N, T, 10.0, 4, 2, precision=prec)
    got = host(plan.propagate(dev(A0, prec), 0.0, 50.0))
    w = 2 * np.pi * np.fft.fftfreq(N, d=T / N)
    I2 = 5 * (8.0 * -21.7 + 2.0 * 85.0)
    I3 = 50.0 * 0.1
    g = fib.gamma_per_km
    X = np.fft.ifft(A0) * N * np.exp(1j * (0.5 * w**2 * I2 + w**3 * I3 / 6)) * math.exp(-g * 50 + 5 * 10 * g)
    ref = np.fft.fft(X) / N
    assert oracle.rel_l2(got, ref) < (1e-12 if prec == "fp64" else 5e-6)


@pytest.mark.parametrize("N,Mn,n_iter", [(1 << 14, 40, 3), (1 << 16, 71, 2), (1 << 18, 17, 4)])
def test_wavefront_schedule_equals_level_schedule(M, N, Mn, n_iter):
    # the two launch schedules compute the same Eq. (6); only the FP32
    # summation order differs
    fib = small_map()
    T = 800.0 * N / 1024
    A0 = wdm_field(N, T, 3, 50.0, 8 * N // 1024, 30.0, 10.0, "qpsk", seed=N)
    a = M.Plan(fib, N, T, 10.0, Mn, n_iter, precision="fp32", schedule="level")
    b = M.Plan(fib, N, T, 10.0, Mn, n_iter, precision="fp32", schedule="wavefront")
    fa = host(a.propagate(dev(A0, "fp32"), 0.0, 30.0))
    fb = host(b.propagate(dev(A0, "fp32"), 0.0, 30.0))
    assert oracle.rel_l2(fb, fa) < 1e-5
    assert b.status()


def test_grid_errors_are_reported(M):
    fib = small_map()
    plan = M.Plan(fib, 1 << 10, 800.0, 2.0, 4, 2, precision="fp32")
    f = dev(np.zeros(1 << 10), "fp32")
    for z0, z1 in ((1.0, 5.0), (0.0, 3.0), (0.0, 200.0)):
        with pytest.raises(M.MPAError):
            plan.propagate(f, z0, z1)
    with pytest.raises(ValueError):
        plan.propagate(dev(np.zeros(1 << 10), "fp64"), 0.0, 2.0)


# ------------------------------------------------- distributed gain
def gain_map():
    # distributed gain on the first segment and extra loss on the second
    # (G = g - gamma of Eq. (1)), a dispersion jump inside the 2-km intervals
    from paper_1101_0086_gb300.workloads import gamma_from_db_per_km
    return FiberMap((Segment(7.0, -21.7, 0.1, 1.3, 0.03), Segment(3.0, 85.0, 0.1, 1.1, -0.01)),
                    gamma_from_db_per_km(0.2), 10.0, 4)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_distributed_gain_matches_oracle(M, prec):
    fib = gain_map()
    N, T = 1 << 12, 3200.0
    A0 = wdm_field(N, T, 3, 50.0, 32, 30.0, 10.0, "qpsk", seed=7)
    ref = oracle.mpa(A0, fib, T, 0.0, 30.0, 1.0, 20, 3)
    plan = M.Plan(fib, N, T, 1.0, 20, 3, precision=prec)
    got = host(plan.propagate(dev(A0, prec), 0.0, 30.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    ref = oracle.ss(A0, fib, T, 0.0, 30.0, 0.1)
    got = host(M.ss_propagate(dev(A0, prec), fib, T, 0.1, 0.0, 30.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]


# ------------------------------------------------------------ split-step
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("logn", [10, 14])
def test_split_step_matches_oracle(M, prec, logn):
    fib = small_map()
    N = 1 << logn
    T = 800.0 * N / 1024
    A0 = wdm_field(N, T, 2, 50.0, 8 * N // 1024, 30.0, 20.0, "qpsk", seed=logn)
    ref = oracle.ss(A0, fib, T, 0.0, 20.0, 0.1)
    got = host(M.ss_propagate(dev(A0, prec), fib, T, 0.1, 0.0, 20.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]


# ------------------------------------------------- benchmark workloads
def test_small_workload_full_length_fp64(M):
    """The N = 2^14, 4-channel, 200 km link at full size: FP64 MPA (L = one
    span, M = 710, n = 3) and FP64 split-step (dz = 0.1 km) against the oracle."""
    w = workload("0")
    A0 = w.field()
    ref = oracle.mpa(A0, w.fiber, w.T_ps, 0.0, w.length_km, w.mpa_L_km, w.mpa_M, w.mpa_n_iter)
    plan = M.Plan(w.fiber, w.N, w.T_ps, w.mpa_L_km, w.mpa_M, w.mpa_n_iter, precision="fp64")
    got = host(plan.propagate(dev(A0, "fp64"), 0.0, w.length_km))
    assert oracle.rel_l2(got, ref) < TOL["fp64"]
    ref_ss = oracle.ss(A0, w.fiber, w.T_ps, 0.0, w.length_km, w.ss_dz_km)
    got_ss = host(M.ss_propagate(dev(A0, "fp64"), w.fiber, w.T_ps, w.ss_dz_km, 0.0, w.length_km))
    assert oracle.rel_l2(got_ss, ref_ss) < TOL["fp64"]


def test_small_workload_fp32(M):
    w = workload("0")
    A0 = w.field()
    ref = oracle.mpa(A0, w.fiber, w.T_ps, 0.0, 100.0, w.mpa_L_km, w.mpa_M, w.mpa_n_iter)
    plan = M.Plan(w.fiber, w.N, w.T_ps, w.mpa_L_km, w.mpa_M, w.mpa_n_iter, precision="fp32")
    got = host(plan.propagate(dev(A0, "fp32"), 0.0, 100.0))
    assert oracle.rel_l2(got, ref) < TOL["fp32"]


def test_bench_workload_sampled_interval_fp32(M):
    """The N = 2^20, 16-channel workload in the benchmark's launch
    configuration (L = 5 km, the workload's M and n_tot): one full
    interval against the oracle, starting from the seeded field's spectrum at
    z = 45 km."""
    w = workload("1")
    A0 = w.field()
    psi0 = oracle.fft(A0, +1)
    z0 = 45.0
    ref = oracle.mpa_interval(psi0, w.fiber, w.T_ps, z0, w.mpa_L_km, w.mpa_M, w.mpa_n_iter)
    plan = M.Plan(w.fiber, w.N, w.T_ps, w.mpa_L_km, w.mpa_M, w.mpa_n_iter, precision="fp32")
    plan.autotune()  # the split the benchmark times
    got = host(plan.interval(dev(psi0, "fp64"), z0))
    assert oracle.rel_l2(got, ref) < TOL["fp32"]


def test_largest_workload_sampled_interval_and_split_step(M):
    """N = 2^24 (the 64-channel 25-GHz link, beta3 = 0.08): the same kernels
    and launch shapes as a full run, on a short interval the oracle computes
    in seconds (M = 4, n_iter = 2), and two FP64 split-steps."""
    w = workload("2")
    A0 = w.field()
    psi0 = oracle.fft(A0, +1)
    ref = oracle.mpa_interval(psi0, w.fiber, w.T_ps, 0.0, 0.5, 4, 2)
    plan = M.Plan(w.fiber, w.N, w.T_ps, 0.5, 4, 2, precision="fp32")
    plan.autotune()
    got = host(plan.interval(dev(psi0, "fp64"), 0.0))
    assert oracle.rel_l2(got, ref) < TOL["fp32"]
    del plan
    ref_ss = oracle.ss(A0, w.fiber, w.T_ps, 0.0, 0.1, 0.05)
    got_ss = host(M.ss_propagate(dev(A0, "fp64"), w.fiber, w.T_ps, 0.05, 0.0, 0.1))
    assert oracle.rel_l2(got_ss, ref_ss) < TOL["fp64"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_empty_propagation_is_the_transform_round_trip(M, prec):
    """z_to = z_from: no interval runs, the field goes through F and F^-1 only."""
    fib = small_map()
    N, T = 1 << 12, 3200.0
    A0 = wdm_field(N, T, 3, 50.0, 32, 30.0, 10.0, "qpsk", seed=3)
    ref = oracle.mpa(A0, fib, T, 10.0, 10.0, 2.0, 24, 3)
    plan = M.Plan(fib, N, T, 2.0, 24, 3, precision=prec)
    got = host(plan.propagate(dev(A0, prec), 10.0, 10.0))
    assert oracle.rel_l2(got, ref) < (1e-14 if prec == "fp64" else 1e-6)
    assert oracle.rel_l2(ref, A0) < 1e-14


def test_maximum_sizes(M):
    """The largest transforms the passes support: N = 2^25 in FP32 (column
    pass 2^11 x row pass 2^14) and N = 2^24 in FP64 (2^11 x 2^13), one short
    interval each (M = 2) against the oracle."""
    from paper_1101_0086_gb300.workloads import dm_map
    fib = dm_map(1, beta3=0.08)
    for prec, logn in (("fp32", 25), ("fp64", 24)):
        N = 1 << logn
        T = 100.0 * N / 8192
        A0 = random_field(N, seed=logn, scale=0.03)  # about 2 mW per sample, every frequency occupied
        psi0 = oracle.fft(A0, +1)
        ref = oracle.mpa_interval(psi0, fib, T, 0.0, 0.5, 2, 2)
        plan = M.Plan(fib, N, T, 0.5, 2, 2, precision=prec)
        got = host(plan.interval(dev(psi0, "fp64"), 0.0))
        assert oracle.rel_l2(got, ref) < TOL[prec], (prec, logn)
        assert oracle.rel_l2(got - psi0, ref - psi0) < (1e-9 if prec == "fp64" else 3e-3)
        del plan, got


# ------------------------------------------------------ batched links
def _batch_specs():
    from paper_1101_0086_gb300.workloads import batch_links
    return batch_links(n_links=7, seed=5, log2_n=(12, 14), spans=(1, 3))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_single_link_plans(M, prec):
    # every link of a batch gets exactly what a plan of its own computes
    specs = _batch_specs()
    L, Mn, n_iter = 5.0, 20, 3
    fields = [dev(s.field(), prec) for s in specs]
    b = M.Batch([(s.fiber, s.T_ps, s.length_km, f) for s, f in zip(specs, fields)], L, Mn, n_iter, precision=prec)
    b.propagate(use_graph=False)
    for s, f in zip(specs, fields):
        plan = M.Plan(s.fiber, s.N, s.T_ps, L, Mn, n_iter, precision=prec)
        ref = host(plan.propagate(dev(s.field(), prec), 0.0, s.length_km))
        assert oracle.rel_l2(host(f), ref) < (1e-13 if prec == "fp64" else 1e-6)


def test_batch_graph_replay_and_oracle(M):
    specs = _batch_specs()
    L, Mn, n_iter = 5.0, 20, 3
    fa = [dev(s.field(), "fp32") for s in specs]
    fb = [dev(s.field(), "fp32") for s in specs]
    a = M.Batch([(s.fiber, s.T_ps, s.length_km, f) for s, f in zip(specs, fa)], L, Mn, n_iter)
    b = M.Batch([(s.fiber, s.T_ps, s.length_km, f) for s, f in zip(specs, fb)], L, Mn, n_iter)
    for _ in range(2):  # first graph call captures (and runs directly), the second replays
        a.propagate(use_graph=True)
        b.propagate(use_graph=False)
    for x, y in zip(fa, fb):
        assert oracle.rel_l2(host(x), host(y)) < 1e-6
    # one link of the batch against the oracle (one propagation)
    s = specs[0]
    f = dev(s.field(), "fp32")
    c = M.Batch([(s.fiber, s.T_ps, s.length_km, f)], L, Mn, n_iter)
    c.propagate(use_graph=True)
    ref = oracle.mpa(s.field(), s.fiber, s.T_ps, 0.0, s.length_km, L, Mn, n_iter)
    assert oracle.rel_l2(host(f), ref) < TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_split_and_the_autotuned_one_match_the_oracle(M, prec):
    """The four-step split only reorders FP32 rounding: every admissible
    column length, and the one mpa_plan_autotune picks, give the oracle's
    result within the tolerance."""
    fib = small_map()
    N, T = 1 << 14, 6400.0
    A0 = wdm_field(N, T, 3, 50.0, 64, 30.0, 10.0, "qpsk", seed=11)
    ref = oracle.mpa(A0, fib, T, 0.0, 20.0, 2.0, 24, 3)
    plan = M.Plan(fib, N, T, 2.0, 24, 3, precision=prec)
    chosen = plan.autotune()
    got = host(plan.propagate(dev(A0, prec), 0.0, 20.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    tried = 0
    for l in range(0, 12):  # 0: the on-chip node transform (N = 2^14 fits in FP32)
        try:
            plan.set_split(l)
        except M.MPAError:
            continue
        tried += 1
        got = host(plan.propagate(dev(A0, prec), 0.0, 20.0))
        assert oracle.rel_l2(got, ref) < TOL[prec], l
    assert tried >= 3 and (chosen == 0 or 4 <= chosen <= 11)


def test_autotuned_batch_matches_the_oracle(M):
    """Per-group split tuning changes only the rounding order: after
    mpa_batch_autotune every link still matches the oracle, and the fields
    were not touched by the tuning."""
    specs = _batch_specs()
    L, Mn, n_iter = 5.0, 20, 3
    fields = [dev(s.field(), "fp32") for s in specs]
    b = M.Batch([(s.fiber, s.T_ps, s.length_km, f) for s, f in zip(specs, fields)], L, Mn, n_iter)
    b.autotune()
    for s, f in zip(specs, fields):
        assert oracle.rel_l2(host(f), s.field()) < 1e-7
    b.propagate(use_graph=True)
    for s, f in list(zip(specs, fields))[:3]:
        ref = oracle.mpa(s.field(), s.fiber, s.T_ps, 0.0, s.length_km, L, Mn, n_iter)
        assert oracle.rel_l2(host(f), ref) < TOL["fp32"]


# --------------------------------- on-chip node transform (N <= 2^14 FP32)
@pytest.mark.parametrize("prec,N,Lk,Mn,n_iter,z0", [
    ("fp32", 1 << 8, 2.0, 5, 2, 8.0),     # smallest N: 32 node rows per tile, one ragged tile
    ("fp32", 1 << 12, 10.0, 20, 3, 0.0),  # node on the 8-km dispersion jump
    ("fp32", 1 << 14, 2.0, 37, 3, 4.0),   # largest FP32 size, one node per CTA
    ("fp64", 1 << 10, 10.0, 20, 3, 0.0),
    ("fp64", 1 << 13, 2.0, 11, 2, 8.0),   # largest FP64 size
])
def test_onchip_interval_matches_oracle(M, prec, N, Lk, Mn, n_iter, z0):
    """mpa_plan_set_split(0): MPA steps 2-4 and the weight of Eq. (6) of a
    node in one kernel (spectrum in shared memory), against the oracle."""
    fib = small_map()
    T = 800.0 * N / 1024
    A0 = wdm_field(N, T, 2, 50.0, max(1, 8 * N // 1024), 30.0, 20.0, "qpsk", seed=N + Mn)
    psi0 = oracle.fft(A0, +1)
    ref = oracle.mpa_interval(psi0, fib, T, z0, Lk, Mn, n_iter)
    plan = M.Plan(fib, N, T, Lk, Mn, n_iter, precision=prec)
    plan.set_split(0)
    got = host(plan.interval(dev(psi0, "fp64"), z0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    assert oracle.rel_l2(got - psi0, ref - psi0) < (1e-9 if prec == "fp64" else 3e-3)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_onchip_propagate_matches_oracle_across_amplifiers(M, prec):
    fib = small_map()
    N, T = 1 << 12, 3200.0
    A0 = wdm_field(N, T, 3, 50.0, 32, 30.0, 10.0, "qpsk", seed=5)
    ref = oracle.mpa(A0, fib, T, 0.0, 30.0, 2.0, 24, 3)
    plan = M.Plan(fib, N, T, 2.0, 24, 3, precision=prec)
    plan.set_split(0)
    got = host(plan.propagate(dev(A0, prec), 0.0, 30.0))
    assert oracle.rel_l2(got, ref) < TOL[prec]
    assert plan.status_code() == 0


def test_onchip_small_workload_fp32(M):
    """The 2^14-mode 4-channel link over two spans with the on-chip node
    transform, and the autotuner's choice for it, against the oracle."""
    w = workload("0")
    A0 = w.field()
    ref = oracle.mpa(A0, w.fiber, w.T_ps, 0.0, 100.0, w.mpa_L_km, w.mpa_M, w.mpa_n_iter)
    for mode in ("onchip", "tuned"):
        plan = M.Plan(w.fiber, w.N, w.T_ps, w.mpa_L_km, w.mpa_M, w.mpa_n_iter, precision="fp32")
        if mode == "onchip":
            plan.set_split(0)
        else:
            plan.autotune()
        got = host(plan.propagate(dev(A0, "fp32"), 0.0, 100.0))
        assert oracle.rel_l2(got, ref) < TOL["fp32"], mode


def test_onchip_split_is_rejected_where_n_does_not_fit(M):
    fib = small_map()
    with pytest.raises(M.MPAError):
        M.Plan(fib, 1 << 17, 800.0 * 128, 2.0, 4, 2, precision="fp32").set_split(0)
    with pytest.raises(M.MPAError):
        M.Plan(fib, 1 << 14, 800.0 * 16, 2.0, 4, 2, precision="fp64").set_split(0)


@pytest.mark.parametrize("logn,Lk,Mn,n_iter,z0", [
    (15, 2.0, 13, 3, 8.0),   # a cluster of 2 CTAs per node, interval in the +85 segment
    (16, 10.0, 20, 2, 0.0),  # a cluster of 4 CTAs per node, node on the 8-km jump
])
def test_cluster_onchip_interval_matches_oracle(M, logn, Lk, Mn, n_iter, z0):
    """FP32 N = 2^15 and 2^16 through the cluster form of the on-chip node
    transform (slices exchanged through distributed shared memory)."""
    fib = small_map()
    N = 1 << logn
    T = 800.0 * N / 1024
    A0 = wdm_field(N, T, 3, 50.0, 8 * N // 1024, 30.0, 20.0, "qpsk", seed=N + Mn)
    psi0 = oracle.fft(A0, +1)
    ref = oracle.mpa_interval(psi0, fib, T, z0, Lk, Mn, n_iter)
    plan = M.Plan(fib, N, T, Lk, Mn, n_iter, precision="fp32")
    plan.set_split(0)
    got = host(plan.interval(dev(psi0, "fp64"), z0))
    assert oracle.rel_l2(got, ref) < TOL["fp32"]
    assert oracle.rel_l2(got - psi0, ref - psi0) < 3e-3
    # a whole propagation across an amplifier, against the four-step passes
    a = dev(A0, "fp32")
    plan.propagate(a, 0.0, 20.0)
    four = M.Plan(fib, N, T, Lk, Mn, n_iter, precision="fp32")
    four.set_split(logn // 2)
    b = dev(A0, "fp32")
    four.propagate(b, 0.0, 20.0)
    assert oracle.rel_l2(host(a), host(b)) < 1e-5


# ------------------------------------------- persistent batch kernel
def _small_specs(n=14):
    """Links for the persistent kernel: N = 2^9 .. 2^14 (FP32 on-chip sizes),
    channels 2-16, 1-4 spans, per-link sigma and power (the seeded batch
    generator)."""
    from paper_1101_0086_gb300.workloads import batch_links
    return batch_links(n_links=n, seed=9, log2_n=(9, 14), spans=(1, 4))


def test_persistent_batch_matches_launches_and_oracle(M):
    """mpa_batch_set_persistent: every interval and iteration of the small
    links in one persistent work-queue launch per size group, against the
    per-pass launches of the same node transform and (two links) the oracle;
    directly and through the captured graph (capture, then replay)."""
    specs = _small_specs()
    A = [sp.field() for sp in specs]
    L, Mn, n_iter = 5.0, 20, 3
    fa = [dev(a, "fp32") for a in A]
    fb = [dev(a, "fp32") for a in A]
    a = M.Batch([(sp.fiber, sp.T_ps, sp.length_km, f) for sp, f in zip(specs, fa)], L, Mn, n_iter)
    b = M.Batch([(sp.fiber, sp.T_ps, sp.length_km, f) for sp, f in zip(specs, fb)], L, Mn, n_iter)
    a.set_persistent(True)
    b.set_persistent(False)
    a.propagate(use_graph=False)
    b.propagate(use_graph=False)
    assert a.status_code() == 0 and b.status_code() == 0
    for x, y in zip(fa, fb):
        assert oracle.rel_l2(host(x), host(y)) < 1e-6
    for i in (0, 5):
        sp = specs[i]
        ref = oracle.mpa(A[i], sp.fiber, sp.T_ps, 0.0, sp.length_km, L, Mn, n_iter)
        assert oracle.rel_l2(host(fa[i]), ref) < TOL["fp32"], i
    # the captured graph: the first call captures (and runs directly), the second replays
    for _ in range(2):
        for f, x in zip(fa, A):
            f.copy_(dev(x, "fp32"))
        a.propagate(use_graph=True)
    assert a.status_code() == 0
    for x, y in zip(fa, fb):
        assert oracle.rel_l2(host(x), host(y)) < 1e-6


def test_persistent_batch_wait_limit_reports_timeout(M):
    """A wait limit of one poll makes the persistent kernel's queue waits run
    out (consumers that start before their task is pushed): the kernel ends,
    mpa_batch_status reports MPA_ERR_TIMEOUT, and with the normal limit the
    next propagation is correct.  Nothing here faults or hangs: every wait is
    bounded."""
    specs = _small_specs(7)
    A = [sp.field() for sp in specs]
    L, Mn, n_iter = 5.0, 20, 2
    f = [dev(a, "fp32") for a in A]
    bt = M.Batch([(sp.fiber, sp.T_ps, sp.length_km, x) for sp, x in zip(specs, f)], L, Mn, n_iter)
    bt.set_persistent(True)
    bt.set_wait_limit(1)
    bt.propagate(use_graph=False)
    assert bt.status_code() == 9
    bt.set_wait_limit(1 << 24)
    for x, a in zip(f, A):
        x.copy_(dev(a, "fp32"))
    bt.propagate(use_graph=False)
    assert bt.status_code() == 0
    sp = specs[3]
    ref = oracle.mpa(A[3], sp.fiber, sp.T_ps, 0.0, sp.length_km, L, Mn, n_iter)
    assert oracle.rel_l2(host(f[3]), ref) < TOL["fp32"]


def test_staged_row_pass_wait_limit_reports_timeout(M):
    """Links of 2^19 and 2^20 modes take four-step node transforms whose row
    pass is the staged persistent kernel (rows of 2^10 points at the default
    split, through a shared staging buffer filled by bulk asynchronous copies).  A wait
    limit of zero polls makes each of its waits run out at once: the groups
    stop after waiting for the copies they started, mpa_batch_status reports
    MPA_ERR_TIMEOUT, and with the normal limit the next propagation matches
    the oracle.  Nothing faults or hangs: every wait is bounded."""
    from paper_1101_0086_gb300.workloads import batch_links
    specs = batch_links(n_links=2, seed=2, log2_n=(19, 20), spans=(1, 1))
    assert sorted(sp.N for sp in specs) == [1 << 19, 1 << 20]
    A = [sp.field() for sp in specs]
    L, Mn, n_iter, z = 5.0, 8, 2, 5.0
    f = [dev(a, "fp32") for a in A]
    bt = M.Batch([(sp.fiber, sp.T_ps, z, x) for sp, x in zip(specs, f)], L, Mn, n_iter)
    bt.set_wait_limit(0)
    bt.propagate(use_graph=False)
    assert bt.status_code() == 9
    bt.set_wait_limit(1 << 22)
    for x, a in zip(f, A):
        x.copy_(dev(a, "fp32"))
    bt.propagate(use_graph=False)
    assert bt.status_code() == 0
    for i, sp in enumerate(specs):
        ref = oracle.mpa(A[i], sp.fiber, sp.T_ps, 0.0, z, L, Mn, n_iter)
        assert oracle.rel_l2(host(f[i]), ref) < TOL["fp32"], i
