"""Run-time checks of the C ABI on the GPU, each made to fire from the host
(no GPU fault is involved anywhere):

* MPA_ERR_NONFINITE: a NaN placed in the host input field;
* MPA_ERR_DIVERGED: a nonlinearity so strong that L >> z_nl, where the
  Picard iteration of the text before MPA step 1 does not contract (the
  oracle shows its relative increments growing 0.84, 0.93, 0.99 while the
  values stay finite), and the contraction factor of a weakly nonlinear
  link, which must stay far below 1;
* MPA_ERR_CUDA: a launch refused on the host by mpa_debug_fail_launch in
  the middle of a propagation, after which the library keeps working;
* the per-segment coefficients of MPAFunction and the measured FMA peaks."""
import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import dm_map, wdm_field

pytestmark = pytest.mark.gpu


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


N, T = 1 << 12, 1600.0


def field(seed=3):
    return wdm_field(N, T, 2, 50.0, 16, 30.0, 2.0, "qpsk", seed=seed)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nan_in_the_input_field_is_reported(M, prec):
    fib = dm_map(2)
    plan = M.Plan(fib, N, T, 5.0, 20, 2, precision=prec)
    a = field()
    a[N // 3] = np.nan
    plan.propagate(dev(a, prec), 0.0, 50.0)
    assert plan.status_code() == 6  # MPA_ERR_NONFINITE
    assert plan.status_code() == 0  # cleared by the read
    # a clean field afterwards reports nothing and matches the oracle
    f = dev(field(), prec)
    plan.propagate(f, 0.0, 50.0)
    assert plan.status_code() == 0
    ref = oracle.mpa(field(), fib, T, 0.0, 50.0, 5.0, 20, 2)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert oracle.rel_l2(f.cpu().numpy().astype(np.complex128), ref) < tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n_iter", [2, 3])
def test_picard_divergence_is_reported(M, prec, n_iter):
    fib = dm_map(1, sigma=100.0)  # z_nl = 1/(sigma P) = 5 km = L: no contraction
    plan = M.Plan(fib, N, T, 5.0, 20, n_iter, precision=prec)
    rc, znl, zd, flags = plan.check_scales(2e-3, 18.0)
    assert rc == 8 and flags & 2  # the plan-time check already warns (L >= z_nl)
    plan.propagate(dev(field(), prec), 0.0, 5.0)
    assert plan.contraction() >= 1.0
    assert plan.status_code() == 7  # MPA_ERR_DIVERGED (the values are still finite)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_weakly_nonlinear_link_contracts(M, prec):
    fib = dm_map(2)  # sigma = 1.3: z_nl = 385 km >> L = 5 km
    plan = M.Plan(fib, N, T, 5.0, 20, 4, precision=prec)
    assert plan.check_scales(2e-3, 18.0)[0] == 0
    plan.propagate(dev(field(), prec), 0.0, 100.0)
    q = plan.contraction()
    assert 0.0 < q < 0.2, q
    assert plan.status_code() == 0


def test_batch_status_reports_a_nan_link(M):
    import torch
    fib = dm_map(2)
    good = dev(field(1), "fp32")
    bad_h = field(2)
    bad_h[7] = np.inf
    bad = dev(bad_h, "fp32")
    other = dev(wdm_field(1 << 13, 3200.0, 2, 50.0, 32, 30.0, 2.0, "qpsk", seed=4), "fp32")
    b = M.Batch([(fib, T, 50.0, good), (fib, T, 25.0, bad), (fib, 3200.0, 50.0, other)], 5.0, 20, 2, "fp32")
    b.propagate(False)
    torch.cuda.synchronize()
    assert b.status_code() == 6
    assert b.status_code() == 0
    ref = oracle.mpa(field(1), fib, T, 0.0, 50.0, 5.0, 20, 2)
    assert oracle.rel_l2(good.cpu().numpy().astype(np.complex128), ref) < 1e-4


def test_injected_launch_failure_mid_propagation(M):
    import torch
    fib = dm_map(2)
    plan = M.Plan(fib, N, T, 5.0, 20, 2, precision="fp32")
    n0 = M.kernel_launches()
    M.debug_fail_launch(5, 2)  # the sixth launch of the next call fails with cudaErrorMemoryAllocation
    with pytest.raises(M.MPAError) as e:
        plan.propagate(dev(field(), "fp32"), 0.0, 50.0)
    assert "status 4" in str(e.value) and "memory" in str(e.value)
    assert M.kernel_launches() - n0 == 5  # five launches were made, the sixth was refused
    torch.cuda.synchronize()
    # disarmed after firing: the library keeps working
    f = dev(field(), "fp32")
    plan.propagate(f, 0.0, 50.0)
    assert plan.status_code() == 0
    ref = oracle.mpa(field(), fib, T, 0.0, 50.0, 5.0, 20, 2)
    assert oracle.rel_l2(f.cpu().numpy().astype(np.complex128), ref) < 1e-4


def test_mpa_function_checks_the_plan_coefficients(M):
    import torch
    fib = dm_map(2)
    N2, T2 = 1 << 13, 3200.0
    a0 = wdm_field(N2, T2, 2, 50.0, 32, 30.0, 2.0, "qpsk", seed=5)
    plan = M.Plan(fib, N2, T2, 5.0, 20, 2, precision="fp64")
    sig0, b20 = plan.segment_coefficients()
    sig = torch.tensor(sig0, dtype=torch.float64, requires_grad=True)
    b2 = torch.tensor(b20, dtype=torch.float64, requires_grad=True)
    x = dev(a0, "fp64")
    out = M.MPAFunction.apply(x, sig, b2, plan, 0.0, 100.0)
    assert out.shape == x.shape
    # an optimiser step changes sigma: the stale plan is refused ...
    with torch.no_grad():
        sig[1] = sig[1] * 1.1  # one physical segment only: the map is no longer periodic
    with pytest.raises(ValueError):
        M.MPAFunction.apply(x, sig, b2, plan, 0.0, 100.0)
    # ... and the matching plan propagates with the new coefficients
    plan2 = plan.with_segment_coefficients(sig, b2)
    out2 = M.MPAFunction.apply(x, sig, b2, plan2, 0.0, 100.0)
    from paper_1101_0086_gb300.workloads import FiberMap, Segment
    segs = tuple(Segment(s.length_km, s.beta2_ps2_per_km, s.beta3_ps3_per_km, float(sig[i]), s.gain_per_km)
                 for i, s in enumerate(fib.segments * fib.n_periods))
    ref = oracle.mpa(a0, FiberMap(segs, fib.gamma_per_km, fib.z_a_km, 1), T2, 0.0, 100.0, 5.0, 20, 2)
    assert oracle.rel_l2(out2.detach().cpu().numpy(), ref) < 1e-10
    loss = (out2.abs() ** 2).sum()
    loss.backward()
    assert sig.grad is not None and torch.isfinite(sig.grad).all()


def test_alu_peaks_are_plausible_for_a_gb300(M):
    f64 = M.alu_peak("fp64")
    f32 = M.alu_peak("fp32")
    # 152 SMs at up to 2.07 GHz: FP32 FMA <= 128 lanes/SM (80.5 TFLOP/s); FP64 far lower on this part
    assert 1e13 < f32 < 9e13, f32
    assert 1e10 < f64 < f32, f64


def test_per_call_timing_brackets_the_kernels_of_the_call(M):
    """mpa_last_timing: the device time of the last entry point called while
    profiling is on covers the summed kernel times of that call."""
    import torch
    fib = dm_map(2)
    plan = M.Plan(fib, N, T, 5.0, 20, 2, precision="fp32")
    f = dev(field(), "fp32")
    plan.propagate(f, 0.0, 50.0)  # first launches (attributes) outside the timing
    torch.cuda.synchronize()
    M.profile(True)
    try:
        assert M.last_timing() is None  # reset by profile(True)
        plan.propagate(f, 0.0, 50.0)
        name, ms = M.last_timing()
        kern = sum(v[0] for v in M.profile_read().values())
        assert name == "mpa_propagate"
        assert kern > 0 and ms >= 0.9 * kern, (ms, kern)
        assert ms < 1e3
    finally:
        M.profile(False)
    # not timed once profiling is off: the last timed call stays
    plan.propagate(f, 0.0, 50.0)
    assert M.last_timing()[0] == "mpa_propagate"
