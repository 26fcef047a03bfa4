"""tfft_execute_noalloc(): the fused transform with its scratch in the library's
fixed device array, for callers that may not allocate device memory (needs a GPU).

Called straight through the C ABI (ctypes) and compared with the existing
entry point, tfft_execute() in fused mode with a caller-allocated workspace,
on two calls in a row (the array keeps the previous call's contents).  Both
run the same kernels on the same scratch layout, so the outputs must agree
bit for bit.  The inputs are kept, except by the complex-to-real backward of
a real-to-complex plan, which uses its input as scratch with either entry
point.
"""
import ctypes

import numpy as np
import pytest
import torch


pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09536_gb300 import build, _lib
    build.build()
    return _lib.load()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _same_bits(a, b):
    """Equal bit patterns (torch.equal on the 32-bit words of the two tensors)."""
    return torch.equal(a.contiguous().view(torch.float32).view(torch.int32),
                       b.contiguous().view(torch.float32).view(torch.int32))


@pytest.mark.parametrize("shape,grid,kind", [((32, 32, 32), (2, 2), "c2c"),
                                             ((64, 64, 64), (2, 4), "c2c"),
                                             ((16, 32, 64), (4,), "r2c"),
                                             ((16, 64, 256), (2, 4), "r2c")])   # padded stage 0, column window
def test_noalloc_matches_execute(cuda_device, lib, shape, grid, kind):
    from paper_1804_09536_gb300 import inputs
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, kind=kind, device=cuda_device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if kind == "r2c":
        x = p.scatter(inputs.normal_real(shape, seed=11).to(cuda_device), 0, real=True)
    else:
        x = p.scatter(inputs.uniform_complex(shape, seed=11).to(cuda_device), 0)
    x_keep = x.clone()
    ref_f = p.forward(x)                            # existing entry point, caller workspace
    ref_b = p.inverse(ref_f.clone())
    torch.cuda.synchronize()
    for call in range(2):
        y = torch.full_like(ref_f, float("nan"))
        rc = lib.tfft_execute_noalloc(p.handle, -1, _vp(x), _vp(y), stream)
        assert rc == 0, lib.tfft_last_error()
        yin = y.clone()
        z = torch.full_like(ref_b, float("nan"))
        rc = lib.tfft_execute_noalloc(p.handle, 1, _vp(yin), _vp(z), stream)
        assert rc == 0, lib.tfft_last_error()
        torch.cuda.synchronize()
        assert _same_bits(x, x_keep), "the input is kept"
        if kind == "c2c":
            assert _same_bits(yin, y), "a complex-to-complex backward keeps its input too"
        assert _same_bits(y, ref_f), call
        assert _same_bits(z, ref_b), call


def test_noalloc_rejects_plans_beyond_the_array(cuda_device, lib):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan((128, 128, 256), (2, 2), device=cuda_device)   # 32 MiB stage buffer > 16 MiB
    x = p.empty_stage(0)
    y = p.empty_stage(2)
    rc = lib.tfft_execute_noalloc(p.handle, -1, _vp(x), _vp(y), None)
    assert rc == 4                                             # TFFT_EWORKSPACE
    assert b"fixed device array" in lib.tfft_last_error()
