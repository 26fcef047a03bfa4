"""Pins for oracle.redistribute: three constructions agree bit for bit (CPU only)."""
import numpy as np
import pytest

from oracle import decomp, redistribute as R

CASES = [
    ((6, 8, 4), (2, 2)),
    ((8, 8, 8), (2, 4)),
    ((12, 12, 12), (3, 4)),     # the paper's Fig. 4 example: 12^3 on 3 x 4
    ((8, 16, 8), (8,)),         # slab
    ((5, 7, 9), (2, 3)),        # uneven
    ((3, 2, 5), (4, 3)),        # zero-size ranks (M > N_m)
    ((42, 127, 4), (3, 4)),     # App. A's uneven extents on axes 0-1
    ((4, 6, 6, 5), (2, 3, 2)),  # 4-D on a 3-D grid
]


def _rand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


@pytest.mark.parametrize("shape,grid", CASES)
def test_three_constructions_agree_bitwise(shape, grid):
    x = _rand(shape)
    g = len(grid)
    bufs = [R.scatter(x, grid, 0)]
    ntrad = 0
    for s in range(g):
        a = R.redistribute(bufs[-1], shape, grid, s, s + 1)
        b = R.exchange_subarray(bufs[-1], shape, grid, s, s + 1)
        assert np.array_equal(_bits(a), _bits(b))
        i, v, w = decomp.exchange_between(len(shape), grid, s, s + 1)
        if shape[v] % grid[i] == 0 and shape[w] % grid[i] == 0:
            ntrad += 1
            c = R.exchange_traditional(bufs[-1], shape, grid, s, s + 1)
            assert np.array_equal(_bits(a), _bits(c))
        bufs.append(b)
    # chunks keep their global position (Fig. 2c caption): gather is stage independent
    for s, b in enumerate(bufs):
        assert np.array_equal(_bits(R.gather(b, shape, grid, s)), _bits(x))
    # v -> w -> v is the identity
    for s in range(g):
        back = R.exchange_subarray(bufs[s + 1], shape, grid, s + 1, s)
        assert np.array_equal(_bits(back), _bits(bufs[s]))


def test_scatter_places_blocks_by_rank():
    """Tiny explicit example: 4 x 2 x 2 on a 2 x 1 grid, values = global linear index."""
    shape, grid = (4, 2, 2), (2, 1)
    x = np.arange(16, dtype=np.complex64).reshape(shape)
    b0 = R.scatter(x, grid, 0)
    # stage 0: rank 0 holds rows 0-1, rank 1 rows 2-3 -> the buffer is x in C order
    assert np.array_equal(b0.real, np.arange(16))
    b1 = R.exchange_subarray(b0, shape, grid, 0, 1)
    # stage 1: direction 1 (size 1) now cuts axis 2, nothing moves
    assert np.array_equal(b1.real, np.arange(16))
    b2 = R.exchange_subarray(b1, shape, grid, 1, 2)
    # stage 2: axis 1 cut in two by direction 0: rank 0 = x[:, 0, :], rank 1 = x[:, 1, :]
    want = np.concatenate([x[:, 0, :].reshape(-1), x[:, 1, :].reshape(-1)])
    assert np.array_equal(b2, want)


def test_traditional_rejects_uneven():
    x = _rand((5, 7, 9))
    b = R.scatter(x, (2, 3), 0)
    with pytest.raises(ValueError):
        R.exchange_traditional(b, x.shape, (2, 3), 0, 1)


def test_buffer_size_checked():
    with pytest.raises(ValueError):
        R.gather(np.zeros(5, np.complex64), (2, 3), (2,), 0)
