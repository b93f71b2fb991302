"""The bounds-checking debug build (libmpa_debug.so, MPA_DEBUG_BOUNDS=1):
every global access of the MPA passes, the scan and the on-chip node
transform is checked against the plan's workspace.  It runs in a child
process (the release library is loaded in this one).  The checks must not
fire on correct propagations (staged four-step passes with the tile layout,
the on-chip transform, FP64 per-tile passes), and narrowing the accepted
range to half of the workspace must make them fire (MPA_ERR_BOUNDS) with
no access ever leaving the workspace; afterwards the full range gives
correct results again.  Nothing here faults: a failed check skips the
access."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_1101_0086_gb300 import mpa
from paper_1101_0086_gb300.workloads import dm_map, wdm_field
assert mpa.debug_bounds_checked()

def run(N, T, prec, split, L=5.0, M=12, n=2, z=10.0):
    fib = dm_map(1)
    a = wdm_field(N, T, 4, 50.0, max(16, N // 4096), 30.0, 2.0, "qpsk", seed=7)
    plan = mpa.Plan(fib, N, T, L, M, n, precision=prec)
    if split is not None:
        plan.set_split(split)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    f = torch.from_numpy(a).to(dt).cuda()
    plan.propagate(f, 0.0, z)
    st = plan.status_code()
    ref = oracle.mpa(a, fib, T, 0.0, z, L, M, n)
    err = oracle.rel_l2(f.cpu().numpy().astype(np.complex128), ref)
    return plan, a, st, err

# staged four-step passes: 2^10-point rows, 2^8-point columns, tile layout
plan, a, st, err = run(1 << 18, 102400.0, "fp32", 8)
assert st == 0 and err < 1e-4, (st, err)
# the accepted range narrowed to the first half of the workspace: the checks fire
plan.debug_set_bounds(0, plan.workspace_bytes // 2)
f = torch.from_numpy(a).to(torch.complex64).cuda()
plan.propagate(f, 0.0, 10.0)
assert plan.status_code() == 10, "MPA_ERR_BOUNDS expected"
plan.debug_set_bounds(0, 0)
f = torch.from_numpy(a).to(torch.complex64).cuda()
plan.propagate(f, 0.0, 10.0)
assert plan.status_code() == 0
# the on-chip node transform and the FP64 per-tile passes
for N, T, prec, split in ((1 << 12, 1600.0, "fp32", None), (1 << 14, 6400.0, "fp64", None)):
    _, _, st, err = run(N, T, prec, split)
    assert st == 0 and err < (1e-4 if prec == "fp32" else 1e-10), (N, prec, st, err)
print("debug-bounds ok")
"""


def test_debug_build_checks_accesses_without_false_alarms():
    import torch
    from paper_1101_0086_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    so = B.build(debug=True)
    env = dict(os.environ, MPA_LIB=so, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "debug-bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
