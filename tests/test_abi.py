"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/mpa.h; host-only argument and grid validation."""
import ctypes
import math
import os
import re

import pytest

from paper_1101_0086_gb300 import build as B
from paper_1101_0086_gb300 import mpa
from paper_1101_0086_gb300.workloads import FiberMap, Segment, dm_map

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return mpa.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mpa.h")).read()
    return sorted(set(re.findall(r"MPA_API\s+[\w\s\*]+?\b((?:mpa|ss)_\w+)\s*\(", txt)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("mpa_plan_create", "mpa_plan_workspace_size", "mpa_plan_set_workspace", "mpa_propagate",
              "ss_propagate", "mpa_plan_destroy", "mpa_status_string"):
        assert n in names
    assert set(names) == set(mpa.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for n in declared_functions():
        assert hasattr(L, n), n
    out = os.popen(f"nm -D --defined-only {mpa.library_path()}").read()
    exported = set(re.findall(r" T (\w+)", out))
    assert set(declared_functions()) <= exported
    # nothing but the C ABI is exported
    assert {s for s in exported if not s.startswith(("mpa_", "ss_"))} == set()


def test_status_strings(L):
    for s in range(0, 12):
        assert L.mpa_status_string(s) and L.mpa_status_string(s) != b"unknown status"
    assert L.mpa_status_string(99) == b"unknown status"


def test_release_build_has_no_bounds_checks(L):
    """mpa_debug_bounds_checked is 0 in the release library; the range setter
    validates its arguments on the host (a plan without workspace, lo > hi)."""
    assert L.mpa_debug_bounds_checked() == 0
    fib = dm_map(1)
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 10, 2)
    assert rc == 0
    L.mpa_debug_set_bounds.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t]
    assert L.mpa_debug_set_bounds(h, 0, 0) == 3  # no workspace yet
    assert L.mpa_debug_set_bounds(None, 0, 0) == 1
    assert L.mpa_debug_set_bounds(h, 8, 4) == 1  # lo > hi
    L.mpa_plan_destroy(h)


def test_last_timing_without_a_timed_call(L):
    """mpa_last_timing reports no call before any entry point has been timed
    (mpa_profile(1) resets it) and refuses a NULL output."""
    import ctypes as C
    L.mpa_profile(1)
    ms, name = C.c_double(-1.0), C.c_char_p()
    assert L.mpa_last_timing(C.byref(ms), C.byref(name)) == 1 and ms.value == -1.0
    assert L.mpa_last_timing(None, None) == 1
    L.mpa_profile(0)


def test_injected_launch_failure_reaches_the_caller_without_a_gpu(L):
    """mpa_debug_fail_launch: the next kernel launch is refused on the host,
    and the entry point that attempted it returns MPA_ERR_CUDA with the
    injected error as its message; the injection fires once."""
    fib = dm_map(1)
    fm, segs = mpa._fiber_struct(fib)
    N = 1 << 12
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the first launch is refused
    assert L.mpa_debug_fail_launch(0, 0) == 1  # an error code is required
    assert L.mpa_debug_fail_launch(0, 2) == 0  # cudaErrorMemoryAllocation
    rc = L.ss_propagate(ctypes.byref(fm), N, 1600.0, 0.05, 0, fake, 0.0, 0.05, fake, 1 << 20, None)
    assert rc == 4
    assert b"memory" in L.mpa_last_cuda_error()
    assert L.mpa_debug_fail_launch(0, 719) == 0  # cudaErrorLaunchFailure
    rc = L.mpa_fft(N, 1, -1, fake, fake, 1 << 20, None)
    assert rc == 4 and b"launch" in L.mpa_last_cuda_error().lower()
    assert L.mpa_debug_fail_launch(-1, 0) == 0  # disarm


def test_scale_check_follows_the_weak_nonlinearity_assumptions(L):
    """mpa_plan_check_scales: z_nl = 1/(sigma_max P), z_disp = tau^2/<|beta2|>
    (length-weighted mean over the period), flags for z_nl <= z_disp and
    L >= z_nl (errors) and L > z_disp (soft); values recomputed here from
    the map."""
    fib = dm_map(4)
    rc, h = _plan(L, fib, 1 << 20, 102400.0, 5.0, 142, 2)
    assert rc == 0
    b2 = sum(abs(s.beta2_ps2_per_km) * s.length_km for s in fib.segments) / fib.period_km
    smax = max(s.sigma_per_W_km for s in fib.segments)

    def check(P, tau):
        znl, zd, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        L.mpa_plan_check_scales.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int32)]
        r = L.mpa_plan_check_scales(h, P, tau, ctypes.byref(znl), ctypes.byref(zd), ctypes.byref(fl))
        assert znl.value == pytest.approx(1.0 / (smax * P), rel=1e-12)
        assert zd.value == pytest.approx(tau * tau / b2, rel=1e-12)
        return r, fl.value

    t0 = 30.0 / (2.0 * math.sqrt(math.log(2.0)))  # 30 ps intensity FWHM
    assert check(2e-3, t0) == (0, 0)                # the benchmark link: z_nl 385 km, z_disp 8.4 km
    assert check(1.0, t0) == (8, 1 | 2)             # 1 W: z_nl 0.77 km < z_disp and < L
    assert check(2e-3, 3.0) == (0, 4)               # short pulses: L > z_disp only (soft)
    assert check(0.5, 3.0)[0] == 8
    assert L.mpa_plan_check_scales(h, -1.0, t0, None, None, None) == 1
    L.mpa_plan_destroy(h)


def _plan(L, fiber, N, T, Lkm, M, n, prec=0, schedule=0):
    fm, segs = mpa._fiber_struct(fiber)
    prm = mpa._PlanParams(N, T, Lkm, M, n, prec, schedule)
    h = ctypes.c_void_p()
    rc = L.mpa_plan_create(ctypes.byref(fm), ctypes.byref(prm), ctypes.byref(h))
    return rc, h


def test_plan_validation_is_host_only(L):
    fib = dm_map(4)
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 710, 3, schedule=1)
    assert rc == 0
    n = ctypes.c_size_t()
    assert L.mpa_plan_workspace_size(h, ctypes.byref(n)) == 0
    # level-synchronous: (M+1) node spectra of complex64 + FP64 state + complex64 copy + tables
    assert n.value >= 711 * (1 << 14) * 8 + (1 << 14) * 24
    L.mpa_plan_destroy(h)
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 710, 3, schedule=2)
    assert rc == 0
    nw = ctypes.c_size_t()
    assert L.mpa_plan_workspace_size(h, ctypes.byref(nw)) == 0
    # wavefront: 3 slots of 16 node buffers + V_0 + 2 x 3 running-sum arrays + FP64 D and state + copy
    assert nw.value >= (3 * 16 + 1 + 6) * (1 << 14) * 8 + (1 << 14) * 40 and nw.value < n.value
    L.mpa_plan_destroy(h)
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 710, 3, schedule=0)  # AUTO: level-synchronous
    na = ctypes.c_size_t()
    assert L.mpa_plan_workspace_size(h, ctypes.byref(na)) == 0 and na.value == n.value
    L.mpa_plan_destroy(h)
    assert _plan(L, fib, 1 << 10, 800.0, 50.0, 10, 3, schedule=2)[0] == 1  # too small for whole column tiles
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, 10, 3, prec=1, schedule=2)[0] == 1  # FP32 only
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, 10, 3, schedule=3)[0] == 1
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 710, 3)
    # propagate without workspace is refused before any CUDA call
    assert L.mpa_propagate(h, ctypes.c_void_p(16), 0.0, 50.0, None) == 3
    L.mpa_plan_destroy(h)
    assert _plan(L, fib, 3000, 12800.0, 50.0, 710, 3)[0] == 2      # N not a power of two
    assert _plan(L, fib, 1 << 26, 12800.0, 50.0, 710, 3)[0] == 2   # too large
    assert _plan(L, fib, 1 << 25, 12800.0, 50.0, 7, 3, 1)[0] == 2  # FP64 limit 2^24
    assert _plan(L, fib, 1 << 14, 12800.0, 7.0, 10, 3)[0] == 5     # L neither divides nor is a multiple of 50 km
    assert _plan(L, fib, 1 << 14, -1.0, 50.0, 10, 3)[0] == 1
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, 0, 3)[0] == 1
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, 10, 0)[0] == 1
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, 10, 3, 7)[0] == 1
    bad = FiberMap((Segment(-1.0, 0.0, 0.0, 0.0),), 0.0, 0.0, 1)
    assert _plan(L, bad, 1 << 14, 12800.0, 50.0, 10, 3)[0] == 1
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 100.0, 10, 3)  # L a multiple of the period
    assert rc == 0
    L.mpa_plan_destroy(h)


def test_size_limits_and_host_allocation_failures_are_statuses(L):
    """M above 2^24 and more than 2^20 interval starts per period are
    refused before any allocation; a node table the host cannot hold comes
    back as MPA_ERR_HOST_MEMORY (11) instead of a C++ exception crossing the
    C ABI (which would end the process)."""
    fib = dm_map(4)
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0, (1 << 24) + 1, 2)[0] == 1
    assert _plan(L, fib, 1 << 14, 12800.0, 50.0 / (1 << 21), 4, 2)[0] == 5
    # 2^20 interval starts x (2^24 + 1) nodes x 48 bytes: about 8e14 bytes of node constants
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0 / (1 << 20), 1 << 24, 2)
    assert rc == 11 and not h.value
    assert L.mpa_status_string(11) == b"host memory allocation failed"
    # the same through the batch: one link of 2^14 modes over the whole map
    fm, segs = mpa._fiber_struct(fib)
    links = (mpa._Link * 1)()
    links[0] = mpa._Link(fm, 1 << 14, 12800.0, fib.length_km, ctypes.c_void_p(256))
    L.mpa_batch_create.argtypes = [ctypes.POINTER(mpa._Link), ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]
    b = ctypes.c_void_p()
    assert L.mpa_batch_create(links, 1, 50.0, (1 << 24) + 1, 2, 0, ctypes.byref(b)) == 1
    assert L.mpa_batch_create(links, 1, 50.0 / (1 << 21), 4, 2, 0, ctypes.byref(b)) == 5
    assert L.mpa_batch_create(links, 1, 50.0 / (1 << 20), 1 << 24, 2, 0, ctypes.byref(b)) == 11 and not b.value
    # intervals far below the amplifier spacing that end on the amplifiers are a valid grid
    assert L.mpa_batch_create(links, 1, 50.0 / (1 << 10), 1, 2, 0, ctypes.byref(b)) == 0 and b.value
    L.mpa_batch_destroy(b)
    # a plan of ordinary size still works after the failures
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 800, 3)
    assert rc == 0
    L.mpa_plan_destroy(h)


def test_gamma_from_db_per_km(L):
    """The dB/km helper of the ABI: |A|^2 falls by the stated dB over 1 km."""
    from paper_1101_0086_gb300.workloads import gamma_from_db_per_km
    for db in (0.0, 0.2, 0.35, 1.0):
        g = mpa.gamma_from_db_per_km(db)
        assert g == pytest.approx(gamma_from_db_per_km(db), rel=1e-15, abs=0.0)
        assert 10 * math.log10(math.exp(2 * g)) == pytest.approx(db, rel=1e-13, abs=1e-15)


def test_ss_workspace_size(L):
    n = ctypes.c_size_t()
    assert L.ss_workspace_size(1 << 20, 0, ctypes.byref(n)) == 0 and n.value == (1 << 20) * 8
    assert L.ss_workspace_size(1 << 20, 1, ctypes.byref(n)) == 0 and n.value == (1 << 20) * 16
    assert L.ss_workspace_size(100, 0, ctypes.byref(n)) == 2
    assert L.ss_workspace_size(1 << 20, 5, ctypes.byref(n)) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(mpa, "_SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mpa, "_lib", None)
    with pytest.raises(mpa.MPAError):
        mpa.lib()


def test_split_selection_is_validated_on_the_host(L):
    """mpa_plan_set_split accepts every column length both passes (and the
    reverse-mode tiling) support, and rejects the others, without a GPU."""
    fib = dm_map(4)
    L.mpa_plan_set_split.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    for prec in (0, 1):
        rc, h = _plan(L, fib, 1 << 20, 102400.0, 5.0, 142, 3, prec=prec)
        assert rc == 0
        ok = [l for l in range(2, 14) if L.mpa_plan_set_split(h, l) == 0]
        assert 10 in ok and 8 in ok           # the square split and a longer-row one
        assert min(ok) >= 4 and max(ok) <= 11  # column pass 2^4..2^11
        assert L.mpa_plan_set_split(h, 3) == 2 and L.mpa_plan_set_split(h, 12) == 2
        L.mpa_plan_destroy(h)
    rc, h = _plan(L, fib, 1 << 14, 12800.0, 50.0, 710, 3, schedule=2)  # wavefront keeps its split
    assert L.mpa_plan_set_split(h, 7) == 0 and L.mpa_plan_set_split(h, 6) == 2
    L.mpa_plan_destroy(h)
