"""GPU: tfft_execute_host -- arrays in page-locked host memory, copies overlapped with the
transforms on two buffer sets; results must equal the device-resident path bit for bit."""
import pytest
import torch

from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, rel_l2

pytestmark = pytest.mark.gpu


def _pinned(t):
    return t.contiguous().pin_memory()


@pytest.mark.parametrize("signs", [[-1], [-1, +1], [+1], [-1, +1, -1]])
def test_execute_host_c2c_matches_device_path(cuda_device, signs):
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (32, 48, 40), (2, 4)
    p = Plan(shape, grid, device=cuda_device)
    first = 0 if signs[0] == -1 else p.g
    last = p.g if signs[-1] == -1 else 0
    xs = [p.scatter(inputs.normal_complex(shape, seed=20 + k).to(cuda_device), first) for k in range(5)]
    h_in = [_pinned(x.cpu()) for x in xs]
    h_out = [torch.empty(p.stage_elems(last), dtype=torch.complex64).pin_memory() for _ in xs]
    p.execute_host(signs, h_in, h_out)
    torch.cuda.synchronize()
    for k, x in enumerate(xs):
        y = x
        for sg in signs:
            y = p.execute(sg, y, p.empty_stage(p.g if sg == -1 else 0), "fused", p.workspace("fused"))
        assert torch.equal(h_out[k], y.cpu()), k
        assert torch.equal(h_in[k], x.cpu())  # inputs untouched
    if signs == [-1, +1]:
        assert rel_l2(h_out[0].numpy(), h_in[0].numpy()) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid", [((16, 32, 64), (4,)),
                                        ((16, 64, 256), (2, 4))])   # padded stage 0, column window
def test_execute_host_r2c(cuda_device, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    xs = [p.scatter(inputs.normal_real(shape, seed=30 + k).to(cuda_device), 0, real=True) for k in range(3)]
    h_in = [_pinned(x.cpu()) for x in xs]
    h_spec = [torch.empty(p.stage_elems(p.g), dtype=torch.complex64).pin_memory() for _ in xs]
    h_back = [torch.empty(p.stage_elems(0, True), dtype=torch.float32).pin_memory() for _ in xs]
    p.execute_host([-1], h_in, h_spec)
    p.execute_host([-1, +1], h_in, h_back)
    torch.cuda.synchronize()
    for k, x in enumerate(xs):
        y = p.execute(-1, x, p.empty_stage(p.g), "fused", p.workspace("fused"))
        assert torch.equal(h_spec[k], y.cpu())
        assert rel_l2(h_back[k].numpy(), h_in[k].numpy()) <= RTOL_FP32


def test_execute_host_rejects_pageable_and_small_space(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    from paper_1804_09536_gb300._lib import TfftError
    shape, grid = (16, 16, 16), (2, 2)
    p = Plan(shape, grid, device=cuda_device)
    pin = torch.zeros(p.stage_elems(0), dtype=torch.complex64).pin_memory()
    pageable = torch.zeros(p.stage_elems(0), dtype=torch.complex64)
    with pytest.raises(TfftError) as e:
        p.execute_host([-1], [pageable], [pin])
    assert e.value.status == 1
    small = torch.empty(p.host_space_bytes() // 2, dtype=torch.uint8, device=cuda_device)
    with pytest.raises(TfftError) as e:
        p.execute_host([-1], [pin], [pin.clone().pin_memory()], space=small)
    assert e.value.status == 4
    with pytest.raises(TfftError):
        p.execute_host([-1, -1], [pin], [pin.clone().pin_memory()])
