"""GPU parity over a seeded sweep of (shape, grid, kind) draws (needs a GPU).

Each draw picks a 2-D or 3-D shape from the specialised lengths, a slab or
pencil grid whose extents need not divide the axes (uneven blocks and, for
real-to-complex plans with an odd Hermitian half, the padded stage 0 and its
column window), and checks the fused forward and inverse against the FP64
oracle and the unfused path bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import dft, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, bits, rel_l2, to_dev

pytestmark = pytest.mark.gpu

C2C_LENGTHS = [8, 12, 16, 24, 32, 48, 60, 64, 80, 96, 120, 128, 160, 192, 240, 256]
R2C_LENGTHS = [64, 96, 120, 128, 160, 192, 240, 256, 320, 384, 512]   # real innermost extents
GRID_EXTENTS = [1, 2, 3, 4, 5, 8]


def _draws(n, seed=2024, max_elems=1 << 20):
    rng = np.random.RandomState(seed)
    out = []
    while len(out) < n:
        kind = "r2c" if rng.rand() < 0.4 else "c2c"
        d = 3 if rng.rand() < 0.8 else 2
        shape = [int(rng.choice(C2C_LENGTHS)) for _ in range(d - 1)]
        shape.append(int(rng.choice(R2C_LENGTHS if kind == "r2c" else C2C_LENGTHS)))
        if math.prod(shape) > max_elems:
            continue
        g = 1 if (d == 2 or rng.rand() < 0.3) else 2
        grid = tuple(int(rng.choice(GRID_EXTENTS)) for _ in range(g))
        out.append((tuple(shape), grid, kind))
    return out


DRAWS = _draws(24)


@pytest.mark.parametrize("shape,grid,kind", DRAWS)
def test_sweep_vs_oracle(cuda_device, shape, grid, kind):
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    p = Plan(shape, grid, kind=kind, device=cuda_device)
    if kind == "r2c":
        x = inputs.normal_real(shape, seed=7).numpy()
        b0 = R.scatter(x, grid, 0)
        want = dft.distributed_rfft_forward(b0.astype(np.float64), shape, grid)
    else:
        x = inputs.uniform_complex(shape, seed=7).numpy()
        b0 = R.scatter(x, grid, 0)
        want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    y = p.forward(to_dev(b0, cuda_device))
    yu = p.forward(to_dev(b0, cuda_device), mode="unfused")
    assert p.device_status() == 0
    assert rel_l2(y.cpu().numpy(), want) <= RTOL_FP32
    assert np.array_equal(bits(y), bits(yu))
    z = p.inverse(y.clone())
    back = z.cpu().numpy()
    if kind == "r2c":
        assert rel_l2(back, dft.distributed_irfft_backward(want, shape, grid)) <= RTOL_FP32
    assert rel_l2(back, b0) <= RTOL_FP32
