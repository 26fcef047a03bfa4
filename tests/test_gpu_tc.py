"""GPU: tensor-core radix-16 stage (split hi/lo BF16 / FP16, FP32 accumulate) (needs a GPU).

The error of these modes is reported against the FP64 oracle; the bars below
are the measured error with headroom (BF16 x3 keeps about 16 mantissa bits,
FP16 x3 about 22), not the FP32 1e-5 bar.
"""
import numpy as np
import pytest
import torch

from oracle import dft, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, rel_l2, to_dev

pytestmark = pytest.mark.gpu

BARS = {"bf16x3": 2e-5, "fp16x3": 1e-6}   # measured on 8 x 16 x 512: 3.1e-6, 2.7e-7


TC_CASES = [
    ((8, 16, 512), (2, 2)),         # contiguous 512 pass on the tensor cores
    ((32, 24, 512), (4, 8)),
    ((4, 4, 512), ()),
    ((512, 64, 64), (4, 2)),        # strided TMA 512 pass on the tensor cores (axis 0)
    ((256, 128, 256), (2, 4)),      # strided TMA 256 pass (axis 0) and contiguous 256 (FP32)
    ((64, 512, 512), (2, 4)),       # strided 512 on axis 1 and contiguous 512, both on the tensor cores
    ((96, 256, 128), (2, 2)),       # strided 256 on axis 1 between FP32 passes
]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("shape,grid", TC_CASES)
def test_tc_forward_inverse_vs_oracle(cuda_device, precision, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    x = inputs.normal_complex(shape, seed=0).numpy()
    p = Plan(shape, grid, device=cuda_device, precision=precision)
    names = [n for n, _ in p.launch_info(-1)]
    assert any("_tc_" in n for n in names), names
    if 512 in shape[:-1] or 256 in shape[:-1]:
        assert any(n.startswith("fft_strided_tma_tc_") for n in names), names
    b0 = R.scatter(x, grid, 0)
    y = p.forward(to_dev(b0, cuda_device))
    torch.cuda.synchronize()
    assert p.device_status() == 0
    want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    err_f = rel_l2(y.cpu().numpy(), want)
    z = p.inverse(y.clone())
    err_b = rel_l2(z.cpu().numpy(), b0)
    assert err_f <= BARS[precision], err_f
    assert err_b <= 2 * BARS[precision], err_b
    # the FP32 path on the same input for comparison
    yf = Plan(shape, grid, device=cuda_device).forward(to_dev(b0, cuda_device))
    assert rel_l2(yf.cpu().numpy(), want) <= RTOL_FP32


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("scale", [1e-6, 1e4])
@pytest.mark.parametrize("shape,grid", [((8, 16, 512), (2, 2)), ((512, 32, 32), (2, 2))])
def test_tc_range_of_the_operands(cuda_device, precision, scale, shape, grid):
    """Inputs far from O(1): x 1e4 drives the radix-16 operands past FP16's maximum
    (65504) and x 1e-6 into its subnormals unless each line is range-scaled; the
    error relative to the oracle stays within the same bar (contiguous and strided
    tensor-core passes)."""
    from paper_1804_09536_gb300.plan import Plan
    x = (inputs.normal_complex(shape, seed=1) * scale).numpy()
    b0 = R.scatter(x, grid, 0)
    p = Plan(shape, grid, device=cuda_device, precision=precision)
    y = p.forward(to_dev(b0, cuda_device))
    torch.cuda.synchronize()
    want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    assert np.all(np.isfinite(y.cpu().numpy()))
    assert rel_l2(y.cpu().numpy(), want) <= BARS[precision]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_tc_inverse_of_an_o1_spectrum(cuda_device, precision):
    """The backward transform is unscaled (Eq. 2): an O(1) spectrum concentrated at
    k = 0 (ones plus 1 % noise) grows to 64 x 64 x 32 = 131072 on the radix-16
    operands of the last, contiguous pass -- twice the FP16 maximum."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (64, 64, 512), (2, 2)
    yhat = (1.0 + 0.01 * inputs.normal_complex(shape, seed=2)).numpy().astype(np.complex64)
    b2 = R.scatter(yhat, grid, 2)
    p = Plan(shape, grid, device=cuda_device, precision=precision)
    z = p.inverse(to_dev(b2, cuda_device))
    torch.cuda.synchronize()
    want = dft.distributed_backward(b2.astype(np.complex128), shape, grid)
    assert np.all(np.isfinite(z.cpu().numpy()))
    assert rel_l2(z.cpu().numpy(), want) <= 2 * BARS[precision]


def test_tc_partial_tiles(cuda_device):
    """Lines that do not fill the last 8-line tile."""
    from paper_1804_09536_gb300.plan import Plan
    shape = (3, 5, 512)
    x = inputs.normal_complex(shape, seed=3).numpy()
    p = Plan(shape, (), device=cuda_device, precision="fp16x3")
    y = p.forward(to_dev(x.reshape(-1), cuda_device))
    assert rel_l2(y.cpu().numpy(), dft.fftn_forward(x.astype(np.complex128)).reshape(-1)) <= BARS["fp16x3"]


def test_tc_wait_expiry_reports_status(cuda_device):
    """A one-poll limit on the MMA-completion wait expires: status word set, TMEM
    released, the context stays usable and a normal run afterwards is correct."""
    from paper_1804_09536_gb300.plan import Plan
    shape = (16, 16, 512)
    x = to_dev(inputs.normal_complex(shape, seed=4).numpy().reshape(-1), cuda_device)
    p = Plan(shape, (), device=cuda_device, precision="bf16x3")
    p.set_wait_limit(1)
    p.forward(x)
    torch.cuda.synchronize()
    assert p.device_status(reset=True) == 1
    p.set_wait_limit(0)
    y = p.forward(x)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    want = dft.fftn_forward(x.cpu().numpy().reshape(shape).astype(np.complex128)).reshape(-1)
    assert rel_l2(y.cpu().numpy(), want) <= BARS["bf16x3"]


def test_tc_strided_wait_expiry_reports_status(cuda_device):
    """The strided tensor-core pass with a one-poll limit on its copy and MMA waits:
    the status word is set, tensor memory is released, the context stays usable and
    a normal run afterwards is correct."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (512, 32, 32), (2, 2)
    x = inputs.normal_complex(shape, seed=6).numpy()
    b0 = R.scatter(x, grid, 0)
    p = Plan(shape, grid, device=cuda_device, precision="bf16x3")
    assert any(n.startswith("fft_strided_tma_tc_") for n, _ in p.launch_info(-1))
    xd = to_dev(b0, cuda_device)
    p.set_wait_limit(1)
    p.forward(xd)
    torch.cuda.synchronize()
    assert p.device_status(reset=True) & 1
    p.set_wait_limit(0)
    y = p.forward(xd)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    assert rel_l2(y.cpu().numpy(), want) <= BARS["bf16x3"]


@pytest.mark.slow
def test_tc_full_size_512_sampled(cuda_device):
    """The tensor-core workload of bench.py (512^3, 4 x 8): sampled outputs of both split
    modes against the oracle's definition (error relative to the spectrum's rms), and the
    round trip."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (512, 512, 512), (4, 8)
    x = inputs.normal_complex(shape, seed=0)
    rng = np.random.default_rng(3)
    ks = [(0, 0, 0), (511, 511, 511), (5, 6, 7)] + [tuple(int(v) for v in rng.integers(0, 512, 3))
                                                   for _ in range(3)]
    want = dft.forward_at(x.numpy(), ks)
    for precision in ("bf16x3", "fp16x3"):
        p = Plan(shape, grid, device=cuda_device, precision=precision)
        b0 = p.scatter(x.to(cuda_device), 0)
        y = p.forward(b0)
        torch.cuda.synchronize()
        assert p.device_status() == 0
        yg = p.gather(y, 2).cpu().numpy()
        rms = float(np.sqrt(np.mean(np.abs(yg.astype(np.complex128)) ** 2)))
        got = np.array([yg[k] for k in ks])
        assert np.max(np.abs(got - want)) <= 20 * BARS[precision] * rms, precision
        back = p.inverse(y)
        d = torch.linalg.vector_norm((back - b0).to(torch.complex128)) / torch.linalg.vector_norm(b0.to(torch.complex128))
        assert float(d) <= 2 * BARS[precision], precision
        del p, b0, y, back
