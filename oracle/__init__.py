"""FP64 CPU oracle of the MPA and split-step methods (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark -- never by the product path.  The C
source (``oracle.c``) is this package's own restatement of the paper: its own
radix-2 FFT, FP64 phases from their definition, the literal MPA steps 1-7
with the full (M+1) x N node array (Eq. (6)), and the composite split-step
of Eq. (4).  It shares no code with the CUDA library.

The adjoints (``mpa_adjoint``, ``ss_adjoint``) are the reverse mode of the
same discrete methods, for gradients of a real loss with respect to the
input field and the per-segment sigma and beta2.

Parity unpinned: none -- every function here is pinned by the CPU tests
(brute-force DFT, sigma=0 closed form, L2 conservation, the sech soliton,
the accuracy theory of Eqs. (5)-(7); the adjoints by central finite
differences of the forward methods, the sigma=0 linear adjoint, exact
gradients of a conserved quantity, and the scaling identity of the cubic
term).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import NamedTuple, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib: Optional[ctypes.CDLL] = None

_ERR = {1: "N not a power of two", 2: "inconsistent z-grid", 3: "out of memory", 4: "bad argument"}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` in-tree with gcc (OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o", _SO + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_fft.argtypes = [dp, ctypes.c_long, ctypes.c_int]
        lib.oracle_mpa.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]
        lib.oracle_ss.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp]
        lib.oracle_mpa_interval.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
        lib.oracle_mpa_adjoint.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp,
                                           ctypes.c_int]
        lib.oracle_ss_adjoint.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, dp, dp, dp, dp, dp, dp]
        for f in (lib.oracle_fft, lib.oracle_mpa, lib.oracle_ss, lib.oracle_mpa_interval, lib.oracle_mpa_adjoint,
                  lib.oracle_ss_adjoint):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"{what}: {_ERR.get(rc, rc)}")


def _cfield(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()


def _rows(fiber) -> np.ndarray:
    return np.ascontiguousarray(fiber.as_rows(), dtype=np.float64)


def fft(x, sign: int = +1) -> np.ndarray:
    """sign=+1: F[x]_k = sum_n x_n e^{+2 pi i kn/N}; sign=-1: the inverse with 1/N."""
    a = _cfield(x)
    _check(_load().oracle_fft(_dp(a.view(np.float64)), a.size, int(sign)), "fft")
    return a


def mpa(field, fiber, T_ps: float, z_from: float, z_to: float, L: float, M: int, n_tot: int,
        n_threads: int = 0, return_threads: bool = False):
    """MPA (steps 1-7, Eq. (6)) from z_from to z_to in intervals of length L."""
    a = _cfield(field)
    rows = _rows(fiber)
    used = ctypes.c_int(0)
    rc = _load().oracle_mpa(_dp(rows), rows.shape[0], fiber.gamma_per_km, fiber.z_a_km, fiber.n_periods,
                            a.size, float(T_ps), float(z_from), float(z_to), float(L), int(M), int(n_tot),
                            _dp(a.view(np.float64)), int(n_threads), ctypes.byref(used))
    _check(rc, "mpa")
    return (a, used.value) if return_threads else a


def mpa_interval(psi0, fiber, T_ps: float, z0: float, L: float, M: int, n_tot: int,
                 n_threads: int = 0) -> np.ndarray:
    """psi^{(n_tot)} at the last node of one interval, before step 7."""
    p0 = _cfield(psi0)
    out = np.empty_like(p0)
    rows = _rows(fiber)
    rc = _load().oracle_mpa_interval(_dp(rows), rows.shape[0], fiber.gamma_per_km, fiber.z_a_km,
                                     fiber.n_periods, p0.size, float(T_ps), float(z0), float(L), int(M),
                                     int(n_tot), _dp(p0.view(np.float64)), _dp(out.view(np.float64)),
                                     int(n_threads))
    _check(rc, "mpa_interval")
    return out


def ss(field, fiber, T_ps: float, z_from: float, z_to: float, dz: float) -> np.ndarray:
    """Symmetric split-step of Eq. (4) from z_from to z_to with step dz."""
    a = _cfield(field)
    rows = _rows(fiber)
    rc = _load().oracle_ss(_dp(rows), rows.shape[0], fiber.gamma_per_km, fiber.z_a_km, fiber.n_periods,
                           a.size, float(T_ps), float(z_from), float(z_to), float(dz), _dp(a.view(np.float64)))
    _check(rc, "ss")
    return a


class Gradients(NamedTuple):
    """Reverse-mode results: gradient of the input field, dl/dsigma and
    dl/dbeta2 per physical segment (period-major), and the forward output."""
    field: np.ndarray
    sigma: np.ndarray
    beta2: np.ndarray
    out: np.ndarray


def _adj_buffers(field, grad_out, fiber):
    a = _cfield(field)
    g = _cfield(grad_out)
    n_phys = fiber.n_periods * len(fiber.segments)
    return a, g, np.empty_like(a), np.empty(n_phys), np.empty(n_phys), np.empty_like(a)


def mpa_adjoint(field, grad_out, fiber, T_ps: float, z_from: float, z_to: float, L: float, M: int, n_tot: int,
                n_threads: int = 0) -> Gradients:
    """Reverse mode of :func:`mpa` for a real loss with output gradient
    grad_out (dl/dRe + i dl/dIm)."""
    a, g, gi, gs, gb, out = _adj_buffers(field, grad_out, fiber)
    rows = _rows(fiber)
    rc = _load().oracle_mpa_adjoint(_dp(rows), rows.shape[0], fiber.gamma_per_km, fiber.z_a_km, fiber.n_periods,
                                    a.size, float(T_ps), float(z_from), float(z_to), float(L), int(M), int(n_tot),
                                    _dp(a.view(np.float64)), _dp(g.view(np.float64)), _dp(gi.view(np.float64)),
                                    _dp(gs), _dp(gb), _dp(out.view(np.float64)), int(n_threads))
    _check(rc, "mpa_adjoint")
    return Gradients(gi, gs, gb, out)


def ss_adjoint(field, grad_out, fiber, T_ps: float, z_from: float, z_to: float, dz: float) -> Gradients:
    """Reverse mode of :func:`ss`."""
    a, g, gi, gs, gb, out = _adj_buffers(field, grad_out, fiber)
    rows = _rows(fiber)
    rc = _load().oracle_ss_adjoint(_dp(rows), rows.shape[0], fiber.gamma_per_km, fiber.z_a_km, fiber.n_periods,
                                   a.size, float(T_ps), float(z_from), float(z_to), float(dz),
                                   _dp(a.view(np.float64)), _dp(g.view(np.float64)), _dp(gi.view(np.float64)),
                                   _dp(gs), _dp(gb), _dp(out.view(np.float64)))
    _check(rc, "ss_adjoint")
    return Gradients(gi, gs, gb, out)


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
