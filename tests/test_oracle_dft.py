"""Pins for oracle.dft: brute force, closed forms, invariants, library cross-check (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import dft, redistribute as R

TINY = [(2, 3, 5), (4, 6, 5), (1, 7, 3), (3, 4, 8)]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _crand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def check_brute_force(fwd=None, bwd=None):
    fwd = fwd or dft.fftn_forward
    bwd = bwd or dft.fftn_backward
    for shape in TINY:
        x = _crand(shape, 1)
        assert np.allclose(fwd(x), dft.brute_force_dft(x, -1), rtol=0, atol=1e-13)
        assert np.allclose(bwd(x), dft.brute_force_dft(x, +1), rtol=0, atol=1e-12)


def test_brute_force_matches_eq_multifft():
    check_brute_force()


def test_brute_force_single_entries():
    """Brute force itself: one entry written out as the explicit triple sum."""
    x = _crand((2, 3, 4), 3)
    k = (1, 2, 3)
    acc = 0j
    for j0 in range(2):
        for j1 in range(3):
            for j2 in range(4):
                acc += x[j0, j1, j2] * np.exp(-2j * np.pi * (k[0] * j0 / 2 + k[1] * j1 / 3 + k[2] * j2 / 4))
    acc /= 24
    assert abs(dft.brute_force_dft(x, -1)[k] - acc) < 1e-14


def check_closed_forms(fwd=None, bwd=None):
    fwd = fwd or dft.fftn_forward
    bwd = bwd or dft.fftn_backward
    shape = (6, 10, 8)
    N = math.prod(shape)
    # delta at the origin -> constant 1/N (paper normalisation: 1/N on the forward)
    x = np.zeros(shape, complex)
    x[0, 0, 0] = 1
    assert np.allclose(fwd(x), np.full(shape, 1.0 / N), rtol=0, atol=1e-15)
    # plane wave exp(+2 pi i sum k'_m j_m / N_m) -> a spike of height exactly 1 at k'
    kp = (2, 7, 3)
    j = np.indices(shape)
    pw = np.exp(2j * np.pi * sum(kp[m] * j[m] / shape[m] for m in range(3)))
    y = fwd(pw)
    spike = np.zeros(shape, complex)
    spike[kp] = 1.0
    assert np.allclose(y, spike, rtol=0, atol=1e-13)
    # delta at j' -> (1/N) exp(-2 pi i k . j' / N)
    jp = (4, 1, 5)
    x = np.zeros(shape, complex)
    x[jp] = 1
    k = np.indices(shape)
    want = np.exp(-2j * np.pi * sum(k[m] * jp[m] / shape[m] for m in range(3))) / N
    assert np.allclose(fwd(x), want, rtol=0, atol=1e-15)
    # backward of a spike of height 1 is the plane wave (Eq. 2: no scale)
    assert np.allclose(bwd(spike), pw, rtol=0, atol=1e-12)


def test_closed_forms():
    check_closed_forms()


def check_invariants(fwd=None, bwd=None):
    fwd = fwd or dft.fftn_forward
    bwd = bwd or dft.fftn_backward
    shape = (5, 6, 8)
    N = math.prod(shape)
    x, z = _crand(shape, 4), _crand(shape, 5)
    X = fwd(x)
    # Parseval with the paper's normalisation: sum |X|^2 = (1/N) sum |x|^2
    assert np.isclose(np.sum(abs(X) ** 2), np.sum(abs(x) ** 2) / N, rtol=1e-12)
    # linearity
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    assert np.allclose(fwd(a * x + b * z), a * X + b * fwd(z), rtol=0, atol=1e-13)
    # shift theorem along each axis: x[j - t] -> X[k] exp(-2 pi i k t / N_m)
    for m in range(3):
        t = 2
        k = np.indices(shape)[m]
        assert np.allclose(fwd(np.roll(x, t, axis=m)),
                           X * np.exp(-2j * np.pi * k * t / shape[m]), rtol=0, atol=1e-13)
    # backward o forward = identity
    assert np.allclose(bwd(X), x, rtol=0, atol=1e-12)


def test_invariants():
    check_invariants()


def test_numpy_library_crosscheck():
    """Special case that reduces to a textbook routine: numpy.fft.fftn(norm="forward")."""
    for shape in [(8, 8, 8), (16, 12, 10), (64, 64, 64), (3, 5, 96)]:
        x = _crand(shape, 7)
        assert np.allclose(dft.fftn_forward(x), np.fft.fftn(x, norm="forward"), rtol=0, atol=1e-12)
        assert np.allclose(dft.fftn_backward(x), np.fft.ifftn(x, norm="forward"), rtol=0, atol=1e-9)


def test_partial_dft_order_and_axes():
    """Eq. fftn_forward applies F_{d-1} first; each F_i touches only axis i."""
    x = _crand((4, 5, 6), 8)
    y = dft.partial_dft(x, 1, -1)
    want = np.fft.fft(x, axis=1, norm="forward")
    assert np.allclose(y, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape,grid", [((8, 8, 8), (2, 2)), ((6, 10, 12), (3, 2)),
                                        ((12, 12, 12), (3, 4)), ((8, 16, 4), (4,)),
                                        ((5, 7, 9), (2, 3)), ((4, 6, 6, 5), (2, 3, 2))])
def test_distributed_is_grid_independent(shape, grid):
    x = _crand(shape, 9)
    y = dft.distributed_forward(R.scatter(x, grid, 0), shape, grid)
    assert np.allclose(R.gather(y, shape, grid, len(grid)), dft.fftn_forward(x), rtol=0, atol=1e-13)
    xb = dft.distributed_backward(y, shape, grid)
    assert np.allclose(R.gather(xb, shape, grid, 0), x, rtol=0, atol=1e-12)
    # the traditional exchange (divisible shapes) gives the same bits
    if shape == (12, 12, 12):
        y2 = dft.distributed_forward(R.scatter(x, grid, 0), shape, grid,
                                     exchange=R.exchange_traditional)
        assert np.array_equal(y2, y)


@pytest.mark.slow
def test_appendix_a_round_trip():
    """App. A: 42 x 127 x 256 on a 2-D grid, fill j + j i per local array, forward then
    backward, |Re - j| and |Im - j| < 1e-8 (tests/golden/appendix_a_shapes.txt)."""
    shape, grid = (42, 127, 256), (2, 3)
    from oracle import decomp
    layout, total = decomp.stage_layout(shape, grid, 0)
    buf = np.empty(total, complex)
    for starts, sizes, off in layout:
        n = math.prod(sizes)
        j = np.arange(n, dtype=np.float64)
        buf[off:off + n] = j + 1j * j
    y = dft.distributed_forward(buf, shape, grid)
    back = dft.distributed_backward(y, shape, grid)
    for starts, sizes, off in layout:
        n = math.prod(sizes)
        j = np.arange(n, dtype=np.float64)
        assert np.max(np.abs(back[off:off + n].real - j)) < 1e-8
        assert np.max(np.abs(back[off:off + n].imag - j)) < 1e-8


def test_real_transforms():
    """Footnote to Eq. multifft: real input -> Hermitian; r2c = first N/2 + 1 of c2c."""
    for shape in [(4, 6, 8), (3, 5, 10), (2, 2, 6)]:
        rng = np.random.default_rng(11)
        x = rng.standard_normal(shape)
        full = dft.fftn_forward(x.astype(complex))
        half = dft.rfftn_forward(x)
        assert np.array_equal(half, full[..., : shape[-1] // 2 + 1])
        # Hermitian symmetry X[-k] = conj X[k]
        neg = np.conj(full[(-np.arange(shape[0])) % shape[0]][:, (-np.arange(shape[1])) % shape[1]]
                      [:, :, (-np.arange(shape[2])) % shape[2]])
        assert np.allclose(full, neg, rtol=0, atol=1e-14)
        assert np.allclose(half, np.fft.rfftn(x, norm="forward"), rtol=0, atol=1e-14)
        back = dft.irfftn_backward(half, shape[-1])
        assert np.allclose(back, x, rtol=0, atol=1e-12)
        # c2r ignores the imaginary parts of k = 0 and k = n/2 on the last axis
        pert = half.copy()
        pert[..., 0] += 0.25j
        pert[..., -1] += 0.5j
        assert np.allclose(dft.irfftn_backward(pert, shape[-1]),
                           np.fft.irfftn(pert, s=shape, axes=(0, 1, 2), norm="forward"), rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,grid", [((8, 8, 8), (4,)), ((6, 6, 10), (2, 3)),
                                        ((16, 16, 16), (8,))])
def test_distributed_real(shape, grid):
    rng = np.random.default_rng(12)
    x = rng.standard_normal(shape)
    cshape = shape[:-1] + (shape[-1] // 2 + 1,)
    y = dft.distributed_rfft_forward(R.scatter(x, grid, 0), shape, grid)
    assert np.allclose(R.gather(y, cshape, grid, len(grid)), dft.rfftn_forward(x), rtol=0, atol=1e-14)
    xb = dft.distributed_irfft_backward(y, shape, grid)
    assert np.allclose(R.gather(xb, shape, grid, 0), x, rtol=0, atol=1e-12)


def test_forward_at_matches_full_transform():
    x = _crand((6, 10, 8), 21)
    full = dft.fftn_forward(x)
    ks = [(0, 0, 0), (5, 9, 7), (3, 2, 1), (1, 0, 6)]
    got = dft.forward_at(x, ks, chunk=4)
    assert np.allclose(got, [full[k] for k in ks], rtol=0, atol=1e-14)
