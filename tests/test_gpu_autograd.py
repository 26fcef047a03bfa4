"""GPU: adjoint transform, spectral-weight loss and its autograd gradient (needs a GPU).

Pinned against the oracle's loss / gradient (itself pinned to FP64 central
differences and the adjoint identity in tests/test_oracle_loss.py) and against
FP64 central differences of the oracle loss directly, on 32^3.
"""
import numpy as np
import pytest
import torch

from oracle import dft, loss as oloss, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,grid", [((32, 32, 32), (2, 2)), ((64, 32, 16), (4, 8)),
                                        ((16, 24, 20), (2, 3))])
def test_adjoint_identity_and_oracle(cuda_device, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, device=cuda_device)
    g = len(grid)
    x = inputs.normal_complex(shape, seed=1).numpy()
    y = inputs.normal_complex(shape, seed=2).numpy()
    fx = p.forward(to_dev(R.scatter(x, grid, 0), cuda_device)).cpu().numpy()
    fhy = p.adjoint(to_dev(R.scatter(y, grid, g), cuda_device)).cpu().numpy()
    lhs = np.vdot(fx.astype(np.complex128), R.scatter(y, grid, g).astype(np.complex128))
    rhs = np.vdot(R.scatter(x, grid, 0).astype(np.complex128), fhy.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    want = R.scatter(oloss.adjoint(y.astype(np.complex128)), grid, 0)
    assert rel_l2(fhy, want) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid", [((32, 32, 32), (2, 2)), ((32, 32, 32), (4, 8))])
def test_loss_and_gradient(cuda_device, shape, grid):
    """The 32^3 instance of the 512^3 spectral-weight loss: value, gradient vs the oracle,
    and directional derivatives vs FP64 central differences (h = 1e-6)."""
    from paper_1804_09536_gb300.autograd import spectral_weight_loss
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    p = Plan(shape, grid, device=cuda_device)
    x = inputs.normal_complex(shape, seed=0).numpy()
    w = inputs.uniform01_real(shape, seed=1).numpy()
    xd = to_dev(R.scatter(x, grid, 0), cuda_device).requires_grad_(True)
    wd = to_dev(R.scatter(w, grid, g), cuda_device)
    L = spectral_weight_loss(xd, wd, p)
    L.backward()
    x64, w64 = x.astype(np.complex128), w.astype(np.float64)
    want_L = oloss.loss(x64, w64)
    assert abs(float(L.detach()) - want_L) <= 1e-5 * want_L
    gx = xd.grad.detach().cpu().numpy()
    want_g = R.scatter(oloss.grad(x64, w64), grid, 0)
    assert rel_l2(gx, want_g) <= RTOL_FP32
    gglob = R.gather(gx.astype(np.complex128), shape, grid, 0)
    rng = np.random.default_rng(5)
    for k in range(4):
        d = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        fd = oloss.central_difference(x64, w64, d, h=1e-6)
        an = float(np.sum(gglob.real * d.real + gglob.imag * d.imag))
        assert abs(fd - an) <= 1e-4 * max(1.0, abs(fd)), (k, fd, an)


def test_loss_gradient_scales_with_upstream(cuda_device):
    """backward with an upstream gradient g: d(g * loss)/dx = g * d loss/dx (seed read on device)."""
    from paper_1804_09536_gb300.autograd import spectral_weight_loss
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (16, 16, 16), (2, 2)
    p = Plan(shape, grid, device=cuda_device)
    x = to_dev(R.scatter(inputs.normal_complex(shape, seed=3).numpy(), grid, 0), cuda_device)
    w = to_dev(R.scatter(inputs.uniform01_real(shape, seed=4).numpy(), grid, 2), cuda_device)
    a = x.clone().requires_grad_(True)
    spectral_weight_loss(a, w, p).backward()
    b = x.clone().requires_grad_(True)
    (3.5 * spectral_weight_loss(b, w, p)).backward()
    assert rel_l2(b.grad.cpu().numpy(), 3.5 * a.grad.cpu().numpy()) <= 1e-6


def test_weighted_energy_is_deterministic(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (64, 64, 64), (2, 2)
    p = Plan(shape, grid, device=cuda_device)
    y = to_dev(inputs.normal_complex(shape, seed=6).numpy().reshape(-1), cuda_device)
    w = to_dev(inputs.uniform01_real(shape, seed=7).numpy().reshape(-1), cuda_device)
    vals = [float(p.weighted_energy(2, y, w)) for _ in range(3)]
    assert vals[0] == vals[1] == vals[2]
    ref = float(np.sum(np.abs(y.cpu().numpy().astype(np.complex128)) ** 2 * w.cpu().numpy().astype(np.float64) ** 2))
    assert abs(vals[0] - ref) <= 1e-12 * ref


def test_weighted_energy_writes_u(cuda_device):
    """The loss sweep's second output u = w^2 y (also in place over y), the loss unchanged."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (32, 48, 40), (2, 4)
    p = Plan(shape, grid, device=cuda_device)
    y = to_dev(inputs.normal_complex(shape, seed=8).numpy().reshape(-1), cuda_device)
    w = to_dev(inputs.uniform01_real(shape, seed=9).numpy().reshape(-1), cuda_device)
    l0 = float(p.weighted_energy(2, y, w))
    u = torch.empty_like(y)
    l1 = float(p.weighted_energy(2, y, w, u=u))
    assert l0 == l1
    want = (w.double() ** 2) * y.to(torch.complex128)
    assert float(torch.linalg.vector_norm(u.to(torch.complex128) - want) / torch.linalg.vector_norm(want)) <= 1e-7
    y2 = y.clone()
    l2 = float(p.weighted_energy(2, y2, w, u=y2))
    assert l2 == l0 and torch.equal(y2, u)


@pytest.mark.parametrize("mode", ["fused", "unfused", "packed"])
def test_adjoint_device_coefficient(cuda_device, mode):
    """adjoint(y, coef=c) = c * adjoint(y): the factor is read on the device by the last pass."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (32, 32, 32), (2, 2)
    p = Plan(shape, grid, device=cuda_device)
    y = to_dev(R.scatter(inputs.normal_complex(shape, seed=10).numpy(), grid, 2), cuda_device)
    c = torch.tensor(-2.75, dtype=torch.float64, device=cuda_device)
    a = p.adjoint(y, mode=mode)
    b = p.adjoint(y, mode=mode, coef=c)
    assert rel_l2(b.cpu().numpy(), -2.75 * a.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("mode", ["fused", "unfused", "packed"])
@pytest.mark.parametrize("norm", ["forward", "backward"])
def test_weighted_energy_grad_is_twice_g_times_the_adjoint(cuda_device, mode, norm):
    """tfft_weighted_energy_grad(u, g) = 2 g F^H u with g read on the device (and g = 1
    when none is given), under both normalisations."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (32, 32, 32), (2, 2)
    p = Plan(shape, grid, norm=norm, device=cuda_device)
    u = to_dev(R.scatter(inputs.normal_complex(shape, seed=12).numpy(), grid, 2), cuda_device)
    g = torch.tensor(0.375, dtype=torch.float64, device=cuda_device)
    a = p.adjoint(u, mode=mode).cpu().numpy()
    assert rel_l2(p.weighted_energy_grad(u, g, mode=mode).cpu().numpy(), 0.75 * a) <= 1e-6
    assert rel_l2(p.weighted_energy_grad(u, None, mode=mode).cpu().numpy(), 2.0 * a) <= 1e-6


@pytest.mark.slow
def test_full_size_512_loss_and_gradient_properties(cuda_device):
    """The differentiable workload of bench.py (512^3, 4 x 8), through the properties that
    hold at any size: the loss equals sum w^2 |F x|^2 formed in double from the forward
    output (whose samples the FFT tests pin to the oracle); the gradient equals
    2 F^H(w^2 F x) assembled from the separate calls; the adjoint identity
    <F x, z> = <x, F^H z> for a random z."""
    from paper_1804_09536_gb300.autograd import spectral_weight_loss
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (512, 512, 512), (4, 8)
    p = Plan(shape, grid, device=cuda_device)
    x = p.scatter(inputs.normal_complex(shape, seed=0).to(cuda_device), 0)
    w = p.scatter(inputs.uniform01_real(shape, seed=1).to(cuda_device), 2)
    xr = x.clone().requires_grad_(True)
    L = spectral_weight_loss(xr, w, p)
    L.backward()
    y = p.forward(x)
    want_L = float(torch.sum(w.double() ** 2 * torch.abs(y.to(torch.complex128)) ** 2))
    assert abs(float(L.detach()) - want_L) <= 1e-9 * want_L
    z = p.adjoint(((w * w) * y).contiguous())
    g = xr.grad.detach()
    assert float(torch.linalg.vector_norm((g - 2 * z).to(torch.complex128)) /
                 torch.linalg.vector_norm((2 * z).to(torch.complex128))) <= 1e-6
    zr = p.scatter(inputs.normal_complex(shape, seed=2).to(cuda_device), 2)
    lhs = torch.vdot(y.to(torch.complex128), zr.to(torch.complex128))
    rhs = torch.vdot(x.to(torch.complex128), p.adjoint(zr).to(torch.complex128))
    assert float(torch.abs(lhs - rhs)) <= 1e-5 * float(torch.abs(lhs))
