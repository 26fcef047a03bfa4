"""GPU parity: the subarray exchange kernel (Alg. 3) is a bit-exact copy (needs a GPU)."""
import numpy as np
import pytest
import torch

from oracle import redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import bits, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    ((32, 32, 32), (2, 2)),
    ((12, 12, 12), (3, 4)),          # the paper's Fig. 4 example
    ((42, 127, 256), (3, 4)),        # App. A's uneven extents
    ((42, 127, 256), (2, 3)),
    ((3, 2, 5), (4, 3)),             # zero-size ranks
    ((64, 64, 33), (8,)),            # slab, odd innermost extent (no pair copies)
    ((256, 256, 129), (8,)),         # the r2c slab's complex array
    ((16, 17, 18, 19), (2, 3, 2)),   # App. B's 4-D shape on a 3-D grid
    ((7,), ()),                      # no grid: nothing to exchange
]


@pytest.mark.parametrize("shape,grid", CASES)
def test_exchange_bit_exact(cuda_device, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    x = inputs.uniform_complex(shape, seed=0).numpy()
    g = len(grid)
    if g == 0:
        return
    p = Plan(shape, grid, device=cuda_device)
    bufs = [R.scatter(x, grid, 0)]
    for s in range(g):
        bufs.append(R.exchange_subarray(bufs[-1], shape, grid, s, s + 1))
    for s in range(g):
        v, w = g - s, g - s - 1          # stage s holds axis g-s whole, stage s+1 axis g-s-1
        dev_in = to_dev(bufs[s], cuda_device)
        out = torch.full((bufs[s + 1].size,), float("nan"), dtype=torch.complex64, device=cuda_device)
        p.redistribute(v, w, dev_in, out)
        torch.cuda.synchronize()
        assert np.array_equal(bits(out), bufs[s + 1].view(np.uint8)), (s, v, w)
        # and back: w -> v restores stage s bit for bit
        back = torch.full_like(dev_in, float("nan"))
        p.redistribute(w, v, out, back)
        torch.cuda.synchronize()
        assert np.array_equal(bits(back), bufs[s].view(np.uint8))


def test_exchange_rejects_bad_axes(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    from paper_1804_09536_gb300._lib import TfftError
    p = Plan((8, 8, 8), (2, 2), device=cuda_device)
    a = p.empty_stage(0)
    b = p.empty_stage(2)
    with pytest.raises(TfftError):
        p.redistribute(2, 0, a, b)       # stages 0 and 2 are not adjacent
    with pytest.raises(TfftError):
        p.redistribute(2, 1, a, a)       # in and out overlap
