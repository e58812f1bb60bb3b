"""Host-only unit tests of the library's C++ bookkeeping, compiled with the
host compiler (no GPU, no CUDA runtime call)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    return os.path.join(home, "include")


def test_per_device_state_is_kept_per_device(tmp_path):
    """Device tables and one-time set-up flags are kept per CUDA device: an
    entry written for device 0 is not the entry of device 1, and device
    indexes beyond the table are refused (the caller turns that into an
    error) instead of aliasing another device's entry."""
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(_cuda_include()):
        pytest.skip("no host compiler or CUDA headers")
    exe = str(tmp_path / "per_device_test")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", _cuda_include(),
                           os.path.join(ROOT, "tests", "host", "per_device_test.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
