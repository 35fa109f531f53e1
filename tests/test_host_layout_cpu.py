"""Host layouts of the sparse kernels (SELL form, warp partition, the direct projection's
factor arrays), checked on the CPU by a small C++ driver over seeded random matrices:
tests/host_layout_check.cpp includes the same headers the library is built from."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_host_layout_invariants(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "host_layout_check"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-o", str(exe), os.path.join(HERE, "host_layout_check.cpp")],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
