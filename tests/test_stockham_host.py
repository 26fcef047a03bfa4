"""Host emulation of the kernels' Stockham schedule and butterflies (CPU only).

Compiles tests/native/stockham_emu.cpp (which includes the kernels' own
butterfly and index code from tfft_common.cuh) with the host compiler and
checks every radix combination against the oracle's per-axis DFT.
"""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dft

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "native", "stockham_emu.cpp")
CSRC = os.path.join(ROOT, "paper_1804_09536_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "vector_types.h")):
        pytest.skip("CUDA headers not found")
    out = str(tmp_path_factory.mktemp("emu") / "libemu.so")
    subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", cuda_inc,
                    SRC, "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.emulate_fft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.emulate_fft.restype = ctypes.c_int
    return lib


def _run(lib, L, E, radices, x, sign):
    r = (ctypes.c_int * len(radices))(*radices)
    xin = np.ascontiguousarray(x.astype(np.complex64))
    out = np.zeros(L, np.complex64)
    rc = lib.emulate_fft(L, E, r, len(radices), xin.ctypes.data, out.ctypes.data, sign)
    assert rc == 0
    return out


CASES = []
for radices in [(2,), (3,), (4,), (5,), (8,), (16,), (8, 8, 8), (16, 16, 2), (8, 4, 2), (4, 4, 3, 2),
                (5, 4, 4, 2), (16, 8), (8, 16), (3, 5), (5, 3), (2, 2, 2, 2), (16, 16, 16), (4, 3),
                (8, 3, 4), (16, 5, 2), (32,), (32, 16), (16, 32), (32, 32), (32, 2)]:
    L = int(np.prod(radices))
    lcm = int(np.lcm.reduce(radices))
    for E in (2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 32):
        if E % lcm == 0 and L % E == 0:
            CASES.append((L, E, radices))


@pytest.mark.parametrize("L,E,radices", CASES)
def test_schedule_matches_dft(emu, L, E, radices):
    rng = np.random.default_rng(L * 31 + E)
    x = (rng.standard_normal(L) + 1j * rng.standard_normal(L)).astype(np.complex64)
    ref_f = dft.partial_dft(x.astype(np.complex128), 0, -1) * L     # unnormalised forward
    ref_b = dft.partial_dft(x.astype(np.complex128), 0, +1)
    got_f = _run(emu, L, E, radices, x, -1)
    got_b = _run(emu, L, E, radices, x, +1)
    tol = 1e-6 * np.sqrt(L) * np.log2(max(L, 2)) * np.linalg.norm(ref_f)
    assert np.linalg.norm(got_f - ref_f) <= tol
    assert np.linalg.norm(got_b - ref_b) <= tol
