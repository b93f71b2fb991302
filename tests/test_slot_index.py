"""The split shared-memory slot form of the transforms (per-thread base plus
compile-time offset) equals the padded slot everywhere a pass uses it: the
real device.cuh helpers compiled as host code by nvcc and checked over every
layout, padding, transform length and tile width (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_slots_equal_padded_slots(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "slot_check")
    src = os.path.join(ROOT, "tests", "native", "slot_check.cu")
    inc = os.path.join(ROOT, "paper_1101_0086_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", inc, src, "-o", exe],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 10_000_000


def test_staged_pass_layouts(tmp_path):
    """Shared-memory layouts and copy ranges of the staged row and column
    passes (krs.cuh, kcs.cuh) for every supported length, checked on the
    host: disjoint regions within 227 KB, aligned copy destinations covering
    the stage exactly once, in-range stage reads and exchange slots."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "staged_layout_check")
    src = os.path.join(ROOT, "tests", "native", "staged_layout_check.cu")
    inc = os.path.join(ROOT, "paper_1101_0086_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", inc, src, "-o", exe],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 100_000
