"""Per-device launch set-up cache (CPU only).

Kernel shared-memory attributes, occupancy and SM counts are per device; the
library caches them per device id (csrc/tfft_device_cache.h).  Compiles
tests/native/device_cache_check.cpp against that header with the host
compiler and checks the keying, the once-per-device construction and its
thread safety.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "native", "device_cache_check.cpp")
CSRC = os.path.join(ROOT, "paper_1804_09536_gb300", "csrc")


def test_per_device_cache(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path / "libcache.so")
    subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", CSRC, SRC, "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    assert lib.check_device_cache() == 0


def test_no_process_wide_static_setup_left():
    """No launcher keeps a kernel attribute or a grid size in a plain function-local
    static (which would hold the first device's value for every device)."""
    import re
    bad = []
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith(".cu"):
            continue
        text = open(os.path.join(CSRC, name)).read()
        for m in re.finditer(r"static\s+(const\s+)?(cudaError_t|int|int64_t)\s+\w+\s*=", text):
            bad.append(f"{name}: {m.group(0)}")
    assert not bad, bad
