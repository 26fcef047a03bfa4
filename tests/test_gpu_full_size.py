"""GPU parity at the full benchmark sizes, whole array against the FP64 oracle (needs a GPU).

The workloads bench.py times, in the launch configuration it times them
(fused path, TMA-staged passes, workspace kept), compared element by element
over the whole global array with the oracle's rank-by-rank transform
(Eqs. pencil0-pencil2 / slab0-slab1 and their reverse):

  * 512^3 c2c on the 4 x 8 pencil grid: forward and inverse, rel-L2 <= 1e-5;
    the tensor-core modes' forward error against the same oracle output;
  * 256^3 r2c on the 8-rank slab and 512^3 r2c on the 4 x 8 pencil grid:
    forward and complex-to-real inverse, rel-L2 <= 1e-5;
  * 128^4 c2c on the 4 x 4 x 2 grid: forward, rel-L2 <= 1e-5.

The oracle runs in FP64 on the host cores (seconds to a minute per transform).
"""
import os

import numpy as np
import pytest
import torch

from oracle import dft, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# Measured bars of the tensor-core modes (test_gpu_tc.py), whole array at 512^3
TC_BARS = {"bf16x3": 2e-5, "fp16x3": 1e-6}


def _host_gib() -> float:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES") / 2**30
    except (ValueError, OSError):
        return 0.0


def rel_l2_chunked(got, ref, chunks: int = 64) -> float:
    """||got - ref|| / ||ref|| over whole arrays, in float64, a chunk at a time."""
    got = np.asarray(got).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    assert got.shape == ref.shape
    num = den = 0.0
    for a, b in zip(np.array_split(got, chunks), np.array_split(ref, chunks)):
        b2 = b.astype(np.complex128) if np.iscomplexobj(b) else b.astype(np.float64)
        d = a.astype(b2.dtype) - b2
        num += float(np.vdot(d, d).real)
        den += float(np.vdot(b2, b2).real)
    return float(np.sqrt(num / den))


@pytest.fixture(scope="module")
def pencil512():
    """The 512^3 input (complex N(0,1), seed 0), its stage buffers and the oracle's
    forward of stage 0 and backward of the same values placed in stage 2."""
    if _host_gib() < 24:
        pytest.skip("the 512^3 oracle needs ~16 GiB of host memory")
    shape, grid = (512, 512, 512), (4, 8)
    x = inputs.normal_complex(shape, seed=0).numpy()
    b0 = R.scatter(x, grid, 0)
    b2 = R.scatter(x, grid, 2)
    del x
    want_f = dft.distributed_forward(b0, shape, grid)
    want_b = dft.distributed_backward(b2, shape, grid)
    return shape, grid, b0, b2, want_f, want_b


def test_full_size_512_pencil_whole_array(cuda_device, pencil512):
    from paper_1804_09536_gb300.plan import Plan
    shape, grid, b0, b2, want_f, want_b = pencil512
    p = Plan(shape, grid, device=cuda_device)
    assert any("tma" in n for n, _ in p.launch_info(-1))
    x = torch.from_numpy(b0).to(cuda_device)
    y = p.forward(x)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    err_f = rel_l2_chunked(y.cpu().numpy(), want_f)
    assert err_f <= RTOL_FP32, err_f
    del y
    z = p.inverse(torch.from_numpy(b2).to(cuda_device))
    torch.cuda.synchronize()
    err_b = rel_l2_chunked(z.cpu().numpy(), want_b)
    assert err_b <= RTOL_FP32, err_b


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_full_size_512_tensor_core_whole_array(cuda_device, pencil512, precision):
    """The tensor-core modes at the size bench.py reports them: forward error against
    the FP64 oracle over the whole array, within the modes' measured bars."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid, b0, _, want_f, _ = pencil512
    p = Plan(shape, grid, device=cuda_device, precision=precision)
    assert any("_tc_" in n for n, _ in p.launch_info(-1))
    y = p.forward(torch.from_numpy(b0).to(cuda_device))
    torch.cuda.synchronize()
    assert p.device_status() == 0
    err = rel_l2_chunked(y.cpu().numpy(), want_f)
    assert err <= TC_BARS[precision], (precision, err)


def test_full_size_r2c_256_slab_whole_array(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (256, 256, 256), (8,)
    x = inputs.normal_real(shape, seed=0).numpy()
    b0 = R.scatter(x, grid, 0)
    want = dft.distributed_rfft_forward(b0, shape, grid)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    y = p.forward(torch.from_numpy(b0).to(cuda_device))
    torch.cuda.synchronize()
    assert rel_l2_chunked(y.cpu().numpy(), want) <= RTOL_FP32
    want_b = dft.distributed_irfft_backward(want, shape, grid)
    z = p.inverse(y)
    torch.cuda.synchronize()
    assert rel_l2_chunked(z.cpu().numpy(), want_b) <= RTOL_FP32


def test_full_size_r2c_512_pencil_whole_array(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    if _host_gib() < 24:
        pytest.skip("the 512^3 oracle needs ~16 GiB of host memory")
    shape, grid = (512, 512, 512), (4, 8)
    x = inputs.normal_real(shape, seed=0).numpy()
    b0 = R.scatter(x, grid, 0)
    del x
    want = dft.distributed_rfft_forward(b0, shape, grid)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    y = p.forward(torch.from_numpy(b0).to(cuda_device))
    torch.cuda.synchronize()
    assert rel_l2_chunked(y.cpu().numpy(), want) <= RTOL_FP32
    want_b = dft.distributed_irfft_backward(want, shape, grid)
    del want
    z = p.inverse(y)
    torch.cuda.synchronize()
    assert rel_l2_chunked(z.cpu().numpy(), want_b) <= RTOL_FP32


def test_full_size_128_4d_whole_array(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    if _host_gib() < 48:
        pytest.skip("the 128^4 oracle needs ~32 GiB of host memory")
    shape, grid = (128, 128, 128, 128), (4, 4, 2)
    x = inputs.normal_complex(shape, seed=0).numpy()
    b0 = R.scatter(x, grid, 0)
    del x
    want = dft.distributed_forward(b0, shape, grid)
    p = Plan(shape, grid, device=cuda_device)
    y = p.forward(torch.from_numpy(b0).to(cuda_device))
    torch.cuda.synchronize()
    assert rel_l2_chunked(y.cpu().numpy(), want) <= RTOL_FP32
