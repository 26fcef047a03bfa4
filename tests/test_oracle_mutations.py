"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case monkeypatches one oracle function with a plausible bug (a dropped
term, a wrong sign, index or axis) and checks that at least one pin fails.
"""
import numpy as np
import pytest

from oracle import decomp, dft, loss, redistribute as R

import test_oracle_decomp as tdec
import test_oracle_dft as tdft
import test_oracle_loss as tloss


def _wrong_sign_matrix(L, sign):
    j = np.arange(L)
    return np.exp(-sign * 2j * np.pi * ((np.outer(j, j) % L) / L))


def _partial_no_scale(x, axis, sign):
    y = np.moveaxis(np.tensordot(dft.dft_matrix(x.shape[axis], sign), np.asarray(x, complex),
                                 axes=([1], [axis])), 0, axis)
    return y


def _partial_wrong_index(x, axis, sign):
    L = x.shape[axis]
    j = np.arange(L)
    W = np.exp(sign * 2j * np.pi * ((np.outer(j, j + 1) % L) / L))   # off-by-one in j
    y = np.moveaxis(np.tensordot(W, np.asarray(x, complex), axes=([1], [axis])), 0, axis)
    return y / L if sign == -1 else y


def _fwd_wrong_axis_order(x):
    y = np.asarray(x, complex)
    for axis in range(y.ndim):           # harmless for a full transform, so also drop one axis
        if axis == 1:
            continue
        y = dft.partial_dft(y, axis, -1)
    return y


def _decompose_bad_start(N, M, p):
    q, r = divmod(N, M)
    return q + (r > p), q * p + r


def test_wrong_sign_caught(monkeypatch):
    monkeypatch.setattr(dft, "dft_matrix", _wrong_sign_matrix)
    with pytest.raises(AssertionError):
        tdft.check_closed_forms()


def test_missing_scale_caught(monkeypatch):
    monkeypatch.setattr(dft, "partial_dft", _partial_no_scale)
    with pytest.raises(AssertionError):
        tdft.check_closed_forms()


def test_wrong_index_caught(monkeypatch):
    monkeypatch.setattr(dft, "partial_dft", _partial_wrong_index)
    with pytest.raises(AssertionError):
        tdft.check_brute_force()


def test_dropped_axis_caught():
    with pytest.raises(AssertionError):
        tdft.check_brute_force(fwd=_fwd_wrong_axis_order)


def test_bad_decompose_start_caught():
    with pytest.raises(AssertionError):
        tdec.check_decompose_closed_form(_decompose_bad_start)


def test_swapped_pencil_axes_caught():
    def swapped(shape, grid, stage, rank):
        starts, sizes = decomp.local_box(shape, grid, stage, rank)
        return starts, (sizes[1], sizes[0], sizes[2])
    with pytest.raises(AssertionError):
        tdec.check_pencil_shapes(swapped)


def test_wrong_exchange_box_caught(monkeypatch):
    orig = decomp.subarray_boxes

    def rotated(sizes, axis, nparts):
        b = orig(sizes, axis, nparts)
        return b[1:] + b[:1]
    monkeypatch.setattr(decomp, "subarray_boxes", rotated)
    x = np.arange(8 * 8 * 8, dtype=np.complex64).reshape(8, 8, 8)
    b0 = R.scatter(x, (2, 2), 0)
    with pytest.raises(AssertionError):
        a = R.redistribute(b0, x.shape, (2, 2), 0, 1)
        b = R.exchange_subarray(b0, x.shape, (2, 2), 0, 1)
        assert np.array_equal(a, b)


def test_gradient_missing_factor_caught():
    with pytest.raises(AssertionError):
        tloss.check_gradient_fd(shape=(8, 8, 8), ndirs=3, grad_fn=lambda x, w: loss.grad(x, w) / 2)


def test_gradient_missing_weight_square_caught():
    def g(x, w):
        return 2.0 * loss.adjoint(w * dft.fftn_forward(x))
    with pytest.raises(AssertionError):
        tloss.check_gradient_fd(shape=(8, 8, 8), ndirs=3, grad_fn=g)
