"""Host-side ordering of the spike raster (no GPU): compiles a small C++ check
against the library's header and runs it; see tests/raster_order_check.cpp."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_raster_order_matches_std_sort():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "raster_order_check")
        subprocess.check_call([cxx, "-O2", "-std=c++17", "-pthread",
                               "-I", os.path.join(ROOT, "paper_1902_08410_gb300", "csrc"),
                               os.path.join(ROOT, "tests", "raster_order_check.cpp"), "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stdout + out.stderr
        assert out.stdout.strip().endswith("ok")
