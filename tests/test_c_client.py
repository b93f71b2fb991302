"""The C ABI from plain C: ``include/mpa.h`` compiles as C99 with warnings
as errors, and ``tests/native/c_client.c`` links ``libmpa.so`` and runs its
host-only calls (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_1101_0086_gb300 import mpa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_is_plain_c99():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    r = subprocess.run([gcc, "-x", "c", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        os.path.join(ROOT, "include", "mpa.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_client_links_and_runs(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    so = mpa.library_path()
    if not os.path.exists(so):
        pytest.skip("libmpa.so is not built")
    exe = str(tmp_path / "c_client")
    libdir = os.path.dirname(so)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "native", "c_client.c"), "-L", libdir, "-l:" + os.path.basename(so),
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "checks passed" in run.stdout
