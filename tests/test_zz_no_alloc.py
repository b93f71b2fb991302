"""mpa_fft_noalloc: the transform for callers that cannot allocate device
memory (no workspace argument; the library's own static scratch is used).

Called through the C ABI and compared with mpa_fft (caller-provided
workspace) on two calls in a row, within the FFT parity tolerance used by the
other GPU tests, and with the FP64 oracle's transform of the same input.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1101_0086_gb300.workloads import random_field

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-6, "fp64": 1e-13}


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1101_0086_gb300 import build as B
    from paper_1101_0086_gb300 import mpa
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch, mpa, mpa.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,logn", [("fp32", 12), ("fp32", 20), ("fp64", 14), ("fp64", 19)])
@pytest.mark.parametrize("sign", [+1, -1])
def test_noalloc_matches_workspace_transform_twice(env, prec, logn, sign):
    torch, mpa, L = env
    N = 1 << logn
    code = 0 if prec == "fp32" else 1
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = torch.empty(mpa.ss_workspace_bytes(N, prec), dtype=torch.uint8, device="cuda")
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        xh = random_field(N, seed=100 * logn + call)
        x = torch.from_numpy(xh).to(dt).cuda()
        a = x.clone()
        b = x.clone()
        rc = L.mpa_fft_noalloc(N, code, sign, ctypes.c_void_p(a.data_ptr()), stream)
        assert rc == 0, L.mpa_status_string(rc)
        rc = L.mpa_fft(N, code, sign, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                       stream)
        assert rc == 0
        torch.cuda.synchronize()
        got, ref = a.cpu().numpy(), b.cpu().numpy()
        assert rel_l2(got, ref) < TOL[prec], (call, rel_l2(got, ref))
        # the input as the GPU saw it (rounded to complex64 for FP32)
        exact = oracle.fft(x.cpu().numpy().astype(np.complex128), sign)
        assert rel_l2(got.astype(np.complex128), exact) < TOL[prec], (call, rel_l2(got, exact))


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, mpa, L = env
    big = torch.zeros(1 << 21, dtype=torch.complex64, device="cuda")  # 16 MiB > 8 MiB
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.mpa_fft_noalloc(1 << 21, 0, 1, ctypes.c_void_p(big.data_ptr()), stream)
    assert rc == 3 and b"workspace" in L.mpa_status_string(rc)
    big64 = torch.zeros(1 << 20, dtype=torch.complex128, device="cuda")
    assert L.mpa_fft_noalloc(1 << 20, 1, 1, ctypes.c_void_p(big64.data_ptr()), stream) == 3
