"""Host-side sanitizer run of the FP64 oracle.

``tests/native/oracle_sanitize_check.c`` links ``oracle/oracle.c`` and calls
every exported entry point (FFT, MPA, the single-interval MPA, split-step and
both adjoints) on small cases and on each argument error.  Built with
AddressSanitizer and UndefinedBehaviorSanitizer, any out-of-bounds access,
use after free, leak or undefined arithmetic in the oracle fails this test.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "oracle_sanitize_check.c")
ORACLE_DIR = os.path.join(ROOT, "oracle")
FLAGS = ["-std=c11", "-O1", "-g", "-fopenmp", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
         "-fno-omit-frame-pointer"]


def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "oracle_sanitize_check")
    cmd = [gcc, *FLAGS, "-I", ORACLE_DIR, SRC, os.path.join(ORACLE_DIR, "oracle.c"), "-lm", "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "asan" in (build.stderr or "").lower():
        pytest.skip("this gcc has no sanitizer runtime: " + build.stderr.strip().splitlines()[-1])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1",
               OMP_NUM_THREADS="2")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "oracle sanitizer checks passed" in run.stdout
