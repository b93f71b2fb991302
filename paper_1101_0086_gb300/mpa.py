"""Thin ctypes binding of ``libmpa.so`` (the C ABI declared in ``include/mpa.h``).

Argument marshalling only: every step of the MPA and split-step paths runs in
the library's CUDA kernels.  PyTorch provides device memory (tensors whose
``data_ptr()`` is passed through) and the stream.  There is no CPU fallback:
if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# MPA_LIB selects another build of the library (e.g. the bounds-checking
# libmpa_debug.so of build(debug=True)); the default is the release build.
_SO = os.environ.get("MPA_LIB") or os.path.join(_HERE, "libmpa.so")
_lib: Optional[ctypes.CDLL] = None

FP32, FP64 = 0, 1
SCHEDULES = {"auto": 0, "level": 1, "wavefront": 2}
_STATUS_NONFINITE = 6
STATUS_DIVERGED = 7
STATUS_SCALES = 8
SCALE_FLAGS = {1: "strong nonlinearity (z_nl <= z_disp)", 2: "L >= z_nl", 4: "L > z_disp"}


class MPAError(RuntimeError):
    pass


class _Segment(ctypes.Structure):
    _fields_ = [("length_km", ctypes.c_double), ("beta2_ps2_per_km", ctypes.c_double),
                ("beta3_ps3_per_km", ctypes.c_double), ("sigma_per_W_km", ctypes.c_double),
                ("gain_per_km", ctypes.c_double)]


class _FiberMap(ctypes.Structure):
    _fields_ = [("segments", ctypes.POINTER(_Segment)), ("n_segments", ctypes.c_int32),
                ("gamma_per_km", ctypes.c_double), ("z_a_km", ctypes.c_double), ("n_periods", ctypes.c_int32)]


class _PlanParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("T_ps", ctypes.c_double), ("L_km", ctypes.c_double),
                ("M", ctypes.c_int32), ("n_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]


class _Link(ctypes.Structure):
    _fields_ = [("map", _FiberMap), ("N", ctypes.c_int64), ("T_ps", ctypes.c_double), ("z_to_km", ctypes.c_double),
                ("field", ctypes.c_void_p)]


EXPORTS = ("mpa_plan_create", "mpa_plan_workspace_size", "mpa_plan_set_workspace", "mpa_propagate",
           "mpa_interval", "mpa_plan_status", "mpa_plan_destroy", "ss_workspace_size", "ss_propagate",
           "mpa_fft", "mpa_status_string", "mpa_last_cuda_error", "mpa_kernel_launches", "mpa_profile",
           "mpa_profile_read", "mpa_profile_kind_name", "mpa_fft_noalloc", "mpa_batch_create",
           "mpa_batch_workspace_size", "mpa_batch_set_workspace", "mpa_batch_propagate", "mpa_batch_destroy",
           "mpa_plan_n_segments", "mpa_adjoint_workspace_size", "mpa_propagate_checkpointed", "mpa_adjoint",
           "ss_adjoint_workspace_size", "ss_adjoint", "mpa_plan_autotune", "mpa_plan_set_split",
           "mpa_batch_autotune", "mpa_plan_contraction", "mpa_plan_check_scales", "mpa_batch_status",
           "mpa_debug_fail_launch", "mpa_alu_peak", "mpa_batch_set_persistent", "mpa_batch_set_wait_limit",
           "mpa_last_timing", "mpa_debug_bounds_checked", "mpa_debug_set_bounds", "mpa_gamma_from_db_per_km")


def library_path() -> str:
    return _SO


def lib() -> ctypes.CDLL:
    """Load ``libmpa.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise MPAError(f"{_SO} is missing: build it with paper_1101_0086_gb300.build.build()")
        L = ctypes.CDLL(_SO)
        vp, i32, i64, dbl, szp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_size_t)
        L.mpa_plan_create.argtypes = [ctypes.POINTER(_FiberMap), ctypes.POINTER(_PlanParams), ctypes.POINTER(vp)]
        L.mpa_plan_workspace_size.argtypes = [vp, szp]
        L.mpa_plan_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
        L.mpa_propagate.argtypes = [vp, vp, dbl, dbl, vp]
        L.mpa_interval.argtypes = [vp, vp, vp, dbl, vp]
        L.mpa_plan_status.argtypes = [vp, vp]
        L.mpa_plan_destroy.argtypes = [vp]
        L.mpa_plan_destroy.restype = None
        L.ss_workspace_size.argtypes = [i64, i32, szp]
        L.ss_propagate.argtypes = [ctypes.POINTER(_FiberMap), i64, dbl, dbl, i32, vp, dbl, dbl, vp, ctypes.c_size_t, vp]
        L.mpa_fft.argtypes = [i64, i32, i32, vp, vp, ctypes.c_size_t, vp]
        L.mpa_fft_noalloc.argtypes = [i64, i32, i32, vp, vp]
        L.mpa_batch_create.argtypes = [ctypes.POINTER(_Link), i32, dbl, i32, i32, i32, ctypes.POINTER(vp)]
        L.mpa_batch_workspace_size.argtypes = [vp, szp]
        L.mpa_batch_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
        L.mpa_batch_propagate.argtypes = [vp, i32, vp]
        L.mpa_batch_destroy.argtypes = [vp]
        L.mpa_batch_destroy.restype = None
        for f in ("mpa_batch_create", "mpa_batch_workspace_size", "mpa_batch_set_workspace", "mpa_batch_propagate"):
            getattr(L, f).restype = ctypes.c_int
        L.mpa_fft_noalloc.restype = ctypes.c_int
        L.mpa_status_string.argtypes = [ctypes.c_int]
        L.mpa_status_string.restype = ctypes.c_char_p
        L.mpa_last_cuda_error.restype = ctypes.c_char_p
        L.mpa_kernel_launches.restype = i64
        L.mpa_profile.argtypes = [ctypes.c_int]
        L.mpa_profile.restype = None
        L.mpa_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                       ctypes.POINTER(ctypes.c_double)]
        L.mpa_profile_read.restype = ctypes.c_int
        L.mpa_profile_kind_name.argtypes = [ctypes.c_int]
        L.mpa_plan_n_segments.argtypes = [vp, ctypes.POINTER(i32)]
        L.mpa_adjoint_workspace_size.argtypes = [vp, dbl, dbl, szp]
        L.mpa_propagate_checkpointed.argtypes = [vp, vp, dbl, dbl, vp, ctypes.c_size_t, vp]
        dptr = ctypes.POINTER(ctypes.c_double)
        L.mpa_adjoint.argtypes = [vp, vp, vp, vp, dbl, dbl, vp, ctypes.c_size_t, dptr, dptr, vp]
        L.ss_adjoint_workspace_size.argtypes = [ctypes.POINTER(_FiberMap), i64, i32, dbl, dbl, dbl, i32, szp]
        L.ss_adjoint.argtypes = [ctypes.POINTER(_FiberMap), i64, dbl, dbl, i32, vp, vp, vp, dbl, dbl, i32, vp,
                                 ctypes.c_size_t, dptr, dptr, vp]
        L.mpa_plan_autotune.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.mpa_plan_set_split.argtypes = [vp, i32]
        L.mpa_batch_autotune.argtypes = [vp, vp]
        L.mpa_batch_autotune.restype = ctypes.c_int
        L.mpa_profile_kind_name.restype = ctypes.c_char_p
        L.mpa_plan_contraction.argtypes = [vp, vp, ctypes.POINTER(dbl)]
        L.mpa_plan_check_scales.argtypes = [vp, dbl, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                            ctypes.POINTER(i32)]
        L.mpa_batch_status.argtypes = [vp, vp]
        L.mpa_debug_fail_launch.argtypes = [i64, i32]
        L.mpa_last_timing.argtypes = [ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_char_p)]
        L.mpa_debug_bounds_checked.restype = i32
        L.mpa_gamma_from_db_per_km.argtypes = [dbl]
        L.mpa_gamma_from_db_per_km.restype = dbl
        L.mpa_debug_set_bounds.argtypes = [vp, ctypes.c_size_t, ctypes.c_size_t]
        L.mpa_alu_peak.argtypes = [i32, ctypes.POINTER(dbl), vp]
        L.mpa_batch_set_persistent.argtypes = [vp, i32]
        L.mpa_batch_set_wait_limit.argtypes = [vp, i64]
        for f in ("mpa_plan_contraction", "mpa_plan_check_scales", "mpa_batch_status", "mpa_debug_fail_launch",
                  "mpa_alu_peak", "mpa_batch_set_persistent", "mpa_batch_set_wait_limit"):
            getattr(L, f).restype = ctypes.c_int
        for f in ("mpa_plan_create", "mpa_plan_workspace_size", "mpa_plan_set_workspace", "mpa_propagate",
                  "mpa_interval", "mpa_plan_status", "ss_workspace_size", "ss_propagate", "mpa_fft",
                  "mpa_plan_n_segments", "mpa_adjoint_workspace_size", "mpa_propagate_checkpointed", "mpa_adjoint",
                  "ss_adjoint_workspace_size", "ss_adjoint", "mpa_plan_autotune", "mpa_plan_set_split"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        L = lib()
        msg = L.mpa_status_string(rc).decode()
        if rc == 4:
            msg += ": " + L.mpa_last_cuda_error().decode()
        raise MPAError(f"{what}: {msg} (status {rc})")


def _prec(precision) -> int:
    if precision in (FP32, "fp32", "f32", torch.complex64):
        return FP32
    if precision in (FP64, "fp64", "f64", torch.complex128):
        return FP64
    raise ValueError(f"unknown precision {precision!r}")


def _cdtype(prec: int) -> torch.dtype:
    return torch.complex64 if prec == FP32 else torch.complex128


def _fiber_struct(fiber):
    rows = fiber.as_rows()
    segs = (_Segment * len(rows))(*[_Segment(*map(float, r)) for r in rows])
    fm = _FiberMap(ctypes.cast(segs, ctypes.POINTER(_Segment)), len(rows), float(fiber.gamma_per_km),
                   float(fiber.z_a_km), int(fiber.n_periods))
    return fm, segs  # keep segs alive with fm


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _resolve(device) -> torch.device:
    """The CUDA device a call runs on, with its index ("cuda" = the current one)."""
    d = torch.device(device)
    if d.type == "cuda" and d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return d


def _on_device(device: torch.device, what: str) -> None:
    """The library launches on the current CUDA device, which must be the one
    the call's buffers live on (another device's pointers would be read as
    this device's)."""
    cur = torch.cuda.current_device()
    if device.type != "cuda" or device.index != cur:
        raise ValueError(f"{what}: the buffers are on {device} but the current CUDA device is cuda:{cur}; "
                         f"call it under torch.cuda.device({device.index})")


def _field_ptr(t: torch.Tensor, dtype: torch.dtype, n: int, what: str, device=None) -> ctypes.c_void_p:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{what}: expected a contiguous CUDA {dtype} tensor of {n} elements")
    if device is not None and t.device != device:
        raise ValueError(f"{what}: the tensor is on {t.device}, the call's buffers on {device}")
    return ctypes.c_void_p(t.data_ptr())


def _ws_ptr(ws: torch.Tensor, device, what: str) -> ctypes.c_void_p:
    """A workspace: a contiguous CUDA uint8 tensor on the call's device (the
    library checks its size)."""
    if not getattr(ws, "is_cuda", False) or ws.dtype != torch.uint8 or not ws.is_contiguous():
        raise ValueError(f"{what}: the workspace must be a contiguous CUDA uint8 tensor")
    if ws.device != device:
        raise ValueError(f"{what}: the workspace is on {ws.device}, the call's buffers on {device}")
    return ctypes.c_void_p(ws.data_ptr())


class Plan:
    """An MPA plan (``mpa_plan_create``) with its caller-owned workspace."""

    def __init__(self, fiber, N: int, T_ps: float, L_km: float, M: int, n_iter: int,
                 precision="fp32", device="cuda", workspace: Optional[torch.Tensor] = None, schedule="auto"):
        L = lib()
        self.prec = _prec(precision)
        self.N = int(N)
        self.dtype = _cdtype(self.prec)
        self.fiber = fiber
        self._args = (float(T_ps), float(L_km), int(M), int(n_iter), schedule)
        self._fm, self._segs = _fiber_struct(fiber)
        prm = _PlanParams(self.N, float(T_ps), float(L_km), int(M), int(n_iter), self.prec, SCHEDULES[schedule])
        h = ctypes.c_void_p()
        _check(L.mpa_plan_create(ctypes.byref(self._fm), ctypes.byref(prm), ctypes.byref(h)), "mpa_plan_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(L.mpa_plan_workspace_size(h, ctypes.byref(nbytes)), "mpa_plan_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=_resolve(device))
        self.workspace = workspace
        self.device = workspace.device
        _check(L.mpa_plan_set_workspace(h, _ws_ptr(workspace, self.device, "Plan"), workspace.numel()),
               "mpa_plan_set_workspace")
        self._split = min(max((self.N.bit_length() - 1) // 2, 4), 11)  # split_n's default column length

    def propagate(self, field: torch.Tensor, z_from_km: float, z_to_km: float, stream=None) -> torch.Tensor:
        """In-place MPA propagation of the time-domain field (``mpa_propagate``)."""
        ptr = _field_ptr(field, self.dtype, self.N, "propagate", self.device)
        _on_device(self.device, "propagate")
        _check(lib().mpa_propagate(self._h, ptr, float(z_from_km), float(z_to_km), _stream(stream)), "mpa_propagate")
        return field

    def interval(self, psi0: torch.Tensor, z0_km: float, stream=None) -> torch.Tensor:
        """psi^{(n_iter)} at the last node of one interval (``mpa_interval``)."""
        p0 = _field_ptr(psi0, torch.complex128, self.N, "interval", self.device)
        _on_device(self.device, "interval")
        out = torch.empty_like(psi0)
        _check(lib().mpa_interval(self._h, p0, ctypes.c_void_p(out.data_ptr()), float(z0_km), _stream(stream)),
               "mpa_interval")
        return out

    def autotune(self, stream=None) -> int:
        """``mpa_plan_autotune``: time every admissible four-step split on the
        GPU and keep the fastest; returns log2 of the chosen column length."""
        l2 = ctypes.c_int32()
        _on_device(self.device, "autotune")
        _check(lib().mpa_plan_autotune(self._h, _stream(stream), ctypes.byref(l2)), "mpa_plan_autotune")
        self._split = int(l2.value)
        return int(l2.value)

    def debug_set_bounds(self, lo: int = 0, hi: int = 0) -> None:
        """``mpa_debug_set_bounds``: in a bounds-checking build, accept only
        accesses within workspace bytes [lo, hi) (0, 0: all of it)."""
        _check(lib().mpa_debug_set_bounds(self._h, int(lo), int(hi)), "mpa_debug_set_bounds")

    def set_split(self, log2_n2: int) -> None:
        """``mpa_plan_set_split``: use column length 2^log2_n2 (no timing)."""
        _check(lib().mpa_plan_set_split(self._h, int(log2_n2)), "mpa_plan_set_split")
        self._split = int(log2_n2)

    @property
    def n_segments(self) -> int:
        """Physical segments of the link (n_periods x segments per period)."""
        n = ctypes.c_int32()
        _check(lib().mpa_plan_n_segments(self._h, ctypes.byref(n)), "mpa_plan_n_segments")
        return int(n.value)

    def adjoint_workspace_bytes(self, z_from_km: float, z_to_km: float) -> int:
        n = ctypes.c_size_t()
        _check(lib().mpa_adjoint_workspace_size(self._h, float(z_from_km), float(z_to_km), ctypes.byref(n)),
               "mpa_adjoint_workspace_size")
        return int(n.value)

    def _adj_ws(self, z_from_km, z_to_km, workspace):
        # a caller's workspace goes to the library as is (it checks the size)
        if workspace is None:
            need = self.adjoint_workspace_bytes(z_from_km, z_to_km)
            workspace = torch.empty(need, dtype=torch.uint8, device=self.workspace.device)
        return workspace

    def propagate_checkpointed(self, field: torch.Tensor, z_from_km: float, z_to_km: float,
                               adj_workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """``mpa_propagate`` that also keeps the interval checkpoints in the
        adjoint workspace (returned) for a later :meth:`adjoint` without the input."""
        ws = self._adj_ws(z_from_km, z_to_km, adj_workspace)
        ptr = _field_ptr(field, self.dtype, self.N, "propagate_checkpointed", self.device)
        wp = _ws_ptr(ws, self.device, "propagate_checkpointed")
        _on_device(self.device, "propagate_checkpointed")
        _check(lib().mpa_propagate_checkpointed(self._h, ptr, float(z_from_km), float(z_to_km), wp, ws.numel(),
                                                _stream(stream)),
               "mpa_propagate_checkpointed")
        return ws

    def adjoint(self, grad_out: torch.Tensor, z_from_km: float, z_to_km: float,
                field_in: Optional[torch.Tensor] = None, adj_workspace: Optional[torch.Tensor] = None,
                params: bool = True, stream=None):
        """Reverse mode (``mpa_adjoint``): returns (dl/dA_in, dl/dsigma, dl/dbeta2)
        for the output gradient grad_out; the last two are float64 numpy arrays
        per physical segment (None unless ``params``).  Without ``field_in`` the
        checkpoints of the last :meth:`propagate_checkpointed` in
        ``adj_workspace`` are used."""
        import numpy as np
        if field_in is None and adj_workspace is None:
            raise ValueError("adjoint: give field_in or the workspace of propagate_checkpointed")
        ws = self._adj_ws(z_from_km, z_to_km, adj_workspace)
        go = _field_ptr(grad_out, self.dtype, self.N, "adjoint grad_out", self.device)
        fi = _field_ptr(field_in, self.dtype, self.N, "adjoint field_in", self.device) if field_in is not None else None
        wp = _ws_ptr(ws, self.device, "adjoint")
        _on_device(self.device, "adjoint")
        gi = torch.empty_like(grad_out)
        gs = gb = None
        ps = pb = None
        if params:
            gs = np.zeros(self.n_segments)
            gb = np.zeros(self.n_segments)
            ps = gs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            pb = gb.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().mpa_adjoint(self._h, fi, go, ctypes.c_void_p(gi.data_ptr()), float(z_from_km), float(z_to_km),
                                 wp, ws.numel(), ps, pb, _stream(stream)), "mpa_adjoint")
        return gi, gs, gb

    def status(self, stream=None) -> bool:
        """False if a NaN/Inf was produced since the last call (synchronises);
        raises MPAError if the Picard iteration diverged (``mpa_plan_status``)."""
        rc = lib().mpa_plan_status(self._h, _stream(stream))
        if rc == _STATUS_NONFINITE:
            return False
        _check(rc, "mpa_plan_status")
        return True

    def status_code(self, stream=None) -> int:
        """The raw status of ``mpa_plan_status``: 0, 6 (non-finite), 7 (diverged),
        9 (a bounded wait ran out) or 10 (debug build: an access outside the
        checked range was skipped); clears the flags."""
        return int(lib().mpa_plan_status(self._h, _stream(stream)))

    def contraction(self, stream=None) -> float:
        """Largest Picard contraction factor since the last call (``mpa_plan_contraction``)."""
        q = ctypes.c_double()
        _check(lib().mpa_plan_contraction(self._h, _stream(stream), ctypes.byref(q)), "mpa_plan_contraction")
        return float(q.value)

    def check_scales(self, peak_power_W: float, pulse_width_ps: float):
        """``mpa_plan_check_scales``: (status, z_nl_km, z_disp_km, flags) for
        the field's typical peak power and pulse width."""
        znl, zd, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        rc = lib().mpa_plan_check_scales(self._h, float(peak_power_W), float(pulse_width_ps), ctypes.byref(znl),
                                         ctypes.byref(zd), ctypes.byref(fl))
        if rc not in (0, STATUS_SCALES):
            _check(rc, "mpa_plan_check_scales")
        return int(rc), float(znl.value), float(zd.value), int(fl.value)

    def segment_coefficients(self):
        """(sigma, beta2) per physical segment (period-major, float64 numpy)
        as the plan was created with."""
        import numpy as np
        sig = np.array([sg.sigma_per_W_km for sg in self.fiber.segments] * self.fiber.n_periods, dtype=np.float64)
        b2 = np.array([sg.beta2_ps2_per_km for sg in self.fiber.segments] * self.fiber.n_periods, dtype=np.float64)
        return sig, b2

    def with_segment_coefficients(self, sigma, beta2) -> "Plan":
        """A new plan (same N, window, discretisation, precision and four-step
        split) whose physical segments carry the given sigma and beta2
        (float64, ``n_segments`` values each, period-major).  When the values
        repeat every period the map stays periodic; otherwise it is unrolled
        into one period that spans the link.  For optimisation loops that
        update the per-segment coefficients between gradient steps."""
        import dataclasses

        import numpy as np
        sig = np.asarray(sigma.detach().cpu() if isinstance(sigma, torch.Tensor) else sigma, dtype=np.float64)
        b2 = np.asarray(beta2.detach().cpu() if isinstance(beta2, torch.Tensor) else beta2, dtype=np.float64)
        segs, P = self.fiber.segments, self.fiber.n_periods
        ns = len(segs)
        if sig.shape != (ns * P,) or b2.shape != (ns * P,):
            raise ValueError(f"expected {ns * P} values of sigma and beta2")
        periodic = np.all(sig.reshape(P, ns) == sig[:ns]) and np.all(b2.reshape(P, ns) == b2[:ns])
        if periodic:
            new_segs = tuple(dataclasses.replace(sg, sigma_per_W_km=float(sig[i]), beta2_ps2_per_km=float(b2[i]))
                             for i, sg in enumerate(segs))
            fib = dataclasses.replace(self.fiber, segments=new_segs)
        else:
            new_segs = tuple(dataclasses.replace(segs[i % ns], sigma_per_W_km=float(sig[i]),
                                                 beta2_ps2_per_km=float(b2[i])) for i in range(ns * P))
            fib = dataclasses.replace(self.fiber, segments=new_segs, n_periods=1)
        T_ps, L_km, M, n_iter, schedule = self._args
        q = Plan(fib, self.N, T_ps, L_km, M, n_iter, precision=self.prec, device=self.workspace.device,
                 schedule=schedule)
        q.set_split(self.log2_n2)
        return q

    @property
    def log2_n2(self) -> int:
        """log2 of the current four-step column length (the library's default
        split until :meth:`autotune` or :meth:`set_split` changes it)."""
        return self._split

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mpa_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPAFunction(torch.autograd.Function):
    """Differentiable MPA propagation through the hand-written reverse mode.

    ``MPAFunction.apply(field, sigma, beta2, plan, z_from_km, z_to_km)``
    returns ``plan.propagate`` of a copy of ``field``.  ``sigma`` and
    ``beta2`` are float64 tensors of the plan's per-physical-segment
    coefficients (``plan.n_segments`` values, period-major); they receive
    dl/dsigma and dl/dbeta2 when they require gradients.  The plan carries
    the coefficients the propagation uses, so the forward pass checks that
    the tensors hold exactly those values and raises ValueError otherwise:
    after an optimiser changes them, make the matching plan with
    ``plan.with_segment_coefficients(sigma, beta2)``.  The forward pass
    stores the interval checkpoints; the backward pass is ``mpa_adjoint``."""

    @staticmethod
    def forward(ctx, field, sigma, beta2, plan, z_from_km, z_to_km):
        import numpy as np
        ps, pb = plan.segment_coefficients()
        gs = sigma.detach().to("cpu", torch.float64).reshape(-1).numpy()
        gb = beta2.detach().to("cpu", torch.float64).reshape(-1).numpy()
        if gs.shape != ps.shape or gb.shape != pb.shape or not (np.array_equal(gs, ps) and np.array_equal(gb, pb)):
            raise ValueError("MPAFunction: sigma/beta2 differ from the coefficients the plan propagates with; "
                             "use plan.with_segment_coefficients(sigma, beta2) to make the matching plan")
        out = field.detach().clone()
        ws = plan.propagate_checkpointed(out, z_from_km, z_to_km)
        ctx.plan, ctx.ws, ctx.z = plan, ws, (z_from_km, z_to_km)
        ctx.param_shape = (sigma.shape, sigma.dtype, sigma.device, beta2.shape, beta2.dtype, beta2.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        want_p = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        gi, gs, gb = plan.adjoint(grad_out.contiguous(), ctx.z[0], ctx.z[1], adj_workspace=ctx.ws, params=want_p)
        ss, sd, sdev, bs, bd, bdev = ctx.param_shape
        g_sig = torch.as_tensor(gs, dtype=sd, device=sdev).reshape(ss) if (want_p and ctx.needs_input_grad[1]) else None
        g_b2 = torch.as_tensor(gb, dtype=bd, device=bdev).reshape(bs) if (want_p and ctx.needs_input_grad[2]) else None
        return gi, g_sig, g_b2, None, None, None


class Batch:
    """Independent links propagated together (``mpa_batch_*``): links of equal
    N share launches, groups of different N run as parallel branches of one
    CUDA graph.  ``links`` is a list of (fiber, T_ps, z_to_km, field) with
    CUDA fields of the batch precision, updated in place by ``propagate``."""

    def __init__(self, links, L_km: float, M: int, n_iter: int, precision="fp32", device="cuda"):
        L = lib()
        self.prec = _prec(precision)
        self.dtype = _cdtype(self.prec)
        self.device = _resolve(device)
        keep = []
        arr = (_Link * len(links))()
        for i, (fiber, T_ps, z_to, field) in enumerate(links):
            ptr = _field_ptr(field, self.dtype, field.numel(), "Batch", self.device)
            fm, segs = _fiber_struct(fiber)
            keep.append(segs)
            arr[i] = _Link(fm, field.numel(), float(T_ps), float(z_to), ptr)
        self._keep = keep
        self.fields = [l[3] for l in links]
        h = ctypes.c_void_p()
        _check(L.mpa_batch_create(arr, len(links), float(L_km), int(M), int(n_iter), self.prec, ctypes.byref(h)),
               "mpa_batch_create")
        self._h = h
        n = ctypes.c_size_t()
        _check(L.mpa_batch_workspace_size(h, ctypes.byref(n)), "mpa_batch_workspace_size")
        self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
        _check(L.mpa_batch_set_workspace(h, ctypes.c_void_p(self.workspace.data_ptr()), self.workspace.numel()),
               "mpa_batch_set_workspace")

    def autotune(self, stream=None) -> None:
        """``mpa_batch_autotune``: per-group four-step split by timing."""
        _on_device(self.device, "Batch.autotune")
        _check(lib().mpa_batch_autotune(self._h, _stream(stream)), "mpa_batch_autotune")

    def propagate(self, use_graph: bool = True, stream=None) -> None:
        _on_device(self.device, "Batch.propagate")
        _check(lib().mpa_batch_propagate(self._h, 1 if use_graph else 0, _stream(stream)), "mpa_batch_propagate")

    def status_code(self, stream=None) -> int:
        """``mpa_batch_status``: 0, 6 (a link produced NaN/Inf), 7 (a link's
        Picard iteration diverged), 9 (a bounded wait of a persistent kernel
        ran out) or 10 (debug build: an access outside the workspace was
        skipped) since the last call; clears the flags."""
        return int(lib().mpa_batch_status(self._h, _stream(stream)))

    def set_persistent(self, on: bool) -> None:
        """``mpa_batch_set_persistent``: the persistent work-queue kernel for
        every eligible group (FP32, N <= 2^14) or none."""
        _check(lib().mpa_batch_set_persistent(self._h, 1 if on else 0), "mpa_batch_set_persistent")

    def set_wait_limit(self, polls: int) -> None:
        """``mpa_batch_set_wait_limit``: polls before a wait of the batch's
        persistent kernels (work queue, staged row pass) gives up; 0 makes
        every such wait run out at once."""
        _check(lib().mpa_batch_set_wait_limit(self._h, int(polls)), "mpa_batch_set_wait_limit")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mpa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ss_workspace_bytes(N: int, precision="fp32") -> int:
    n = ctypes.c_size_t()
    _check(lib().ss_workspace_size(int(N), _prec(precision), ctypes.byref(n)), "ss_workspace_size")
    return int(n.value)


def ss_propagate(field: torch.Tensor, fiber, T_ps: float, dz_km: float, z_from_km: float, z_to_km: float,
                 workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """In-place split-step propagation of Eq. (4) (``ss_propagate``); precision from the dtype."""
    prec = _prec(field.dtype)
    N = field.numel()
    ptr = _field_ptr(field, _cdtype(prec), N, "ss_propagate")
    need = ss_workspace_bytes(N, prec)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=field.device)
    wp = _ws_ptr(workspace, field.device, "ss_propagate")
    _on_device(field.device, "ss_propagate")
    fm, segs = _fiber_struct(fiber)
    _check(lib().ss_propagate(ctypes.byref(fm), N, float(T_ps), float(dz_km), prec, ptr, float(z_from_km),
                              float(z_to_km), wp, workspace.numel(), _stream(stream)), "ss_propagate")
    return field


def propagate(field: torch.Tensor, plan: "Plan", z_from_km: float, z_to_km: float, stream=None) -> torch.Tensor:
    """Module-level form of :meth:`Plan.propagate` (``mpa_propagate``)."""
    return plan.propagate(field, z_from_km, z_to_km, stream)


ss = ss_propagate  # the split-step of Eq. (4) under its short name


def ss_adjoint(field_in: torch.Tensor, grad_out: torch.Tensor, fiber, T_ps: float, dz_km: float, z_from_km: float,
               z_to_km: float, ckpt_steps: int = 0, workspace: Optional[torch.Tensor] = None, params: bool = True,
               stream=None):
    """Reverse mode of :func:`ss_propagate` (``ss_adjoint``): returns
    (dl/dA_in, dl/dsigma, dl/dbeta2), the last two float64 numpy arrays per
    physical segment (None unless ``params``)."""
    import numpy as np
    L = lib()
    prec = _prec(field_in.dtype)
    N = field_in.numel()
    fm, segs = _fiber_struct(fiber)
    if workspace is None:
        n = ctypes.c_size_t()
        _check(L.ss_adjoint_workspace_size(ctypes.byref(fm), N, prec, float(dz_km), float(z_from_km), float(z_to_km),
                                           int(ckpt_steps), ctypes.byref(n)), "ss_adjoint_workspace_size")
        workspace = torch.empty(int(n.value), dtype=torch.uint8, device=field_in.device)
    fi = _field_ptr(field_in, _cdtype(prec), N, "ss_adjoint field_in")
    go = _field_ptr(grad_out, _cdtype(prec), N, "ss_adjoint grad_out", field_in.device)
    wp = _ws_ptr(workspace, field_in.device, "ss_adjoint")
    _on_device(field_in.device, "ss_adjoint")
    gi = torch.empty_like(grad_out)
    gs = gb = ps = pb = None
    if params:
        n_phys = len(fiber.segments) * fiber.n_periods
        gs, gb = np.zeros(n_phys), np.zeros(n_phys)
        ps = gs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        pb = gb.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(L.ss_adjoint(ctypes.byref(fm), N, float(T_ps), float(dz_km), prec, fi, go, ctypes.c_void_p(gi.data_ptr()),
                        float(z_from_km), float(z_to_km), int(ckpt_steps), wp, workspace.numel(), ps, pb,
                        _stream(stream)), "ss_adjoint")
    return gi, gs, gb


def fft(data: torch.Tensor, sign: int, workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """In-place transform in the paper's convention (``mpa_fft``): +1 = F, -1 = F^-1 (1/N)."""
    prec = _prec(data.dtype)
    N = data.numel()
    ptr = _field_ptr(data, _cdtype(prec), N, "fft")
    need = ss_workspace_bytes(N, prec)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=data.device)
    wp = _ws_ptr(workspace, data.device, "fft")
    _on_device(data.device, "fft")
    _check(lib().mpa_fft(N, prec, int(sign), ptr, wp, workspace.numel(), _stream(stream)), "mpa_fft")
    return data


def fft_noalloc(data: torch.Tensor, sign: int, stream=None) -> torch.Tensor:
    """``mpa_fft`` without a workspace (``mpa_fft_noalloc``): the library's own
    static scratch is used, so the caller allocates nothing; calls must not
    overlap on the GPU.  N x element size <= 8 MiB."""
    prec = _prec(data.dtype)
    N = data.numel()
    ptr = _field_ptr(data, _cdtype(prec), N, "fft_noalloc")
    _on_device(data.device, "fft_noalloc")
    _check(lib().mpa_fft_noalloc(N, prec, int(sign), ptr, _stream(stream)), "mpa_fft_noalloc")
    return data


def kernel_launches() -> int:
    """Kernels this library has launched since it was loaded."""
    return int(lib().mpa_kernel_launches())


def profile(enable: bool) -> None:
    """Bracket every subsequent kernel launch with CUDA events (resets totals)."""
    lib().mpa_profile(1 if enable else 0)


def profile_read() -> dict:
    """{kernel kind: (total device ms, launches, algorithmic bytes)} of the launches timed so far."""
    L = lib()
    out = {}
    k = 0
    while True:
        name = L.mpa_profile_kind_name(k)
        if not name:
            break
        ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(L.mpa_profile_read(k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)), "mpa_profile_read")
        if n.value:
            out[name.decode()] = (float(ms.value), int(n.value), float(b.value))
        k += 1
    return out


def gamma_from_db_per_km(db_per_km: float) -> float:
    """``mpa_gamma_from_db_per_km``: the amplitude loss coefficient gamma of
    Eq. (1) for a power loss in dB/km."""
    return float(lib().mpa_gamma_from_db_per_km(float(db_per_km)))


def debug_bounds_checked() -> bool:
    """Whether the loaded library checks the MPA passes' accesses
    (``mpa_debug_bounds_checked``: the debug build)."""
    return bool(lib().mpa_debug_bounds_checked())


def last_timing():
    """``mpa_last_timing``: (entry-point name, device ms) of the most recent
    entry-point call timed while ``profile(True)`` is on, or None if none was."""
    ms, name = ctypes.c_double(), ctypes.c_char_p()
    rc = lib().mpa_last_timing(ctypes.byref(ms), ctypes.byref(name))
    if rc == 1:
        return None
    _check(rc, "mpa_last_timing")
    return name.value.decode(), float(ms.value)


def debug_fail_launch(after_launches: int, cuda_error: int = 2) -> None:
    """``mpa_debug_fail_launch``: make the library's launch ``after_launches``
    from now fail on the host with ``cuda_error`` (default 2, out of memory);
    a negative count disarms.  For tests of the error paths."""
    _check(lib().mpa_debug_fail_launch(int(after_launches), int(cuda_error)), "mpa_debug_fail_launch")


def alu_peak(precision="fp64", stream=None) -> float:
    """``mpa_alu_peak``: measured FMA throughput of the current GPU in flop/s."""
    v = ctypes.c_double()
    _check(lib().mpa_alu_peak(_prec(precision), ctypes.byref(v), _stream(stream)), "mpa_alu_peak")
    return float(v.value)
