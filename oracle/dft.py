"""Discrete Fourier transforms for the oracle (test infrastructure only).

Sec. 2, Eqs. 1-2: forward  u^_k = (1/N) sum_j u_j exp(-i k x_j),
                  backward u_j  =       sum_k u^_k exp(+i k x_j),  x_j = 2 pi j / N.
Eq. multifft: the d-D forward DFT applies omega_m^{k_m j_m} / N_m along every
axis m, omega_m = exp(-2 pi i / N_m), with k_m = 0 .. N_m - 1 (not centred).
Eq. fftn_forward: forward = F_0(F_1(... F_{d-1}(u))) -- axis d-1 first;
Eq. fftn_backward: backward = F^-1_{d-1}(... F^-1_0(u^)) -- axis 0 first.
Sign convention of the appendix listings: FORWARD = -1, BACKWARD = +1.

Each partial transform F_i is a matrix product with the L x L matrix
W[k, j] = exp(sign * 2 pi i * ((j k) mod L) / L); reducing j k modulo L in
integers keeps every angle in [0, 2 pi) before the float64 exponential.
"""
from __future__ import annotations

import math

import numpy as np

from . import decomp, redistribute

FORWARD = -1
BACKWARD = +1


def dft_matrix(L: int, sign: int) -> np.ndarray:
    """W[k, j] = exp(sign * 2 pi i (j k mod L) / L), complex128."""
    j = np.arange(L, dtype=np.int64)
    jk = np.outer(j, j) % L
    return np.exp(sign * 2j * np.pi * jk.astype(np.float64) / L)


def partial_dft(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """F_axis (sign -1, includes the 1/N_axis of Eq. multifft) or F^-1_axis (sign +1)."""
    if sign not in (FORWARD, BACKWARD):
        raise ValueError("sign must be -1 (forward) or +1 (backward)")
    x = np.asarray(x, dtype=np.complex128)
    L = x.shape[axis]
    if L == 0:
        return x.copy()
    W = dft_matrix(L, sign)
    y = np.tensordot(W, x, axes=([1], [axis]))   # y[k, ...] = sum_j W[k, j] x[..., j, ...]
    y = np.moveaxis(y, 0, axis)
    if sign == FORWARD:
        y = y / L
    return np.ascontiguousarray(y)


def fftn_forward(x: np.ndarray) -> np.ndarray:
    """Eq. fftn_forward on a whole (undistributed) array: axes d-1, ..., 0."""
    y = np.asarray(x, dtype=np.complex128)
    for axis in reversed(range(y.ndim)):
        y = partial_dft(y, axis, FORWARD)
    return y


def fftn_backward(xhat: np.ndarray) -> np.ndarray:
    """Eq. fftn_backward on a whole array: axes 0, ..., d-1, unscaled."""
    y = np.asarray(xhat, dtype=np.complex128)
    for axis in range(y.ndim):
        y = partial_dft(y, axis, BACKWARD)
    return y


def brute_force_dft(x: np.ndarray, sign: int) -> np.ndarray:
    """Eq. multifft as one (prod N) x (prod N) matrix (tiny shapes only)."""
    x = np.asarray(x, dtype=np.complex128)
    shape = x.shape
    N = math.prod(shape)
    idx = np.array(list(np.ndindex(*shape)), dtype=np.int64).reshape(N, len(shape))
    phase = np.zeros((N, N), dtype=np.float64)
    for m, Nm in enumerate(shape):
        km = idx[:, m][:, None]
        jm = idx[:, m][None, :]
        phase += ((km * jm) % Nm) / Nm
    mat = np.exp(sign * 2j * np.pi * phase)
    y = mat @ x.reshape(N)
    if sign == FORWARD:
        y = y / N
    return y.reshape(shape)


# ------------------------------------------------------------ distributed form

def _transform_ranks(buf, shape, grid, stage, axis, sign):
    """Apply F_axis (or its inverse) to every rank's local array of ``stage``."""
    layout, total = decomp.stage_layout(shape, grid, stage)
    out = np.empty(total, dtype=np.complex128)
    for starts, sizes, offset in layout:
        n = math.prod(sizes)
        if sizes[axis] != shape[axis]:
            raise ValueError(f"axis {axis} is not aligned in stage {stage}")
        loc = buf[offset:offset + n].reshape(sizes)
        out[offset:offset + n] = partial_dft(loc, axis, sign).reshape(-1)
    return out


def distributed_forward(buf, shape, grid, exchange=redistribute.exchange_subarray):
    """Forward transform rank by rank on the virtual grid (Secs. 3.3-3.6).

    ``buf``: stage-0 buffer.  Stage 0 transforms axes d-1 .. g locally
    (Eq. pencil0 / slab0); then for s = 1 .. g: exchange (g-s+1) -> (g-s) in
    P_{g-s} (Eqs. gtp1, gtp2, gt_slab) and transform axis g - s.  Returns the
    stage-g buffer (output aligned in axis 0, axes not permuted).
    """
    d, g = len(shape), len(grid)
    y = np.asarray(buf, dtype=np.complex128)
    for axis in reversed(range(g, d)):
        y = _transform_ranks(y, shape, grid, 0, axis, FORWARD)
    for s in range(1, g + 1):
        y = exchange(y, shape, grid, s - 1, s)
        y = _transform_ranks(y, shape, grid, s, g - s, FORWARD)
    return y


def distributed_backward(buf, shape, grid, exchange=redistribute.exchange_subarray):
    """Backward transform: the forward steps in reverse order with sign +1 (App. A)."""
    d, g = len(shape), len(grid)
    y = np.asarray(buf, dtype=np.complex128)
    for s in range(g, 0, -1):
        y = _transform_ranks(y, shape, grid, s, g - s, BACKWARD)
        y = exchange(y, shape, grid, s, s - 1)
    for axis in range(g, d):
        y = _transform_ranks(y, shape, grid, 0, axis, BACKWARD)
    return y


# ------------------------------------------------------------ real transforms

def rfftn_forward(x: np.ndarray) -> np.ndarray:
    """Real-input forward: the complex forward restricted to k_{d-1} = 0 .. N_{d-1}/2
    (footnote to Eq. multifft, Hermitian symmetry)."""
    x = np.asarray(x, dtype=np.float64)
    full = fftn_forward(x.astype(np.complex128))
    half = x.shape[-1] // 2 + 1
    return np.ascontiguousarray(full[..., :half])


def hermitian_extend_last(xh: np.ndarray, n_last: int) -> np.ndarray:
    """Rebuild k = 0 .. n_last-1 on the last axis from k = 0 .. n_last//2 with
    X[n - k] = conj(X[k]) (the array must already be back-transformed on the
    other axes, where each last-axis line of a real array is Hermitian)."""
    half = n_last // 2 + 1
    if xh.shape[-1] != half:
        raise ValueError("last axis must hold n//2 + 1 coefficients")
    full = np.empty(xh.shape[:-1] + (n_last,), dtype=np.complex128)
    full[..., :half] = xh
    for k in range(half, n_last):
        full[..., k] = np.conj(xh[..., n_last - k])
    return full


def irfftn_backward(xh: np.ndarray, n_last: int) -> np.ndarray:
    """Complex-to-real backward: inverse on axes 0 .. d-2, then Hermitian extension
    and inverse on the last axis, real part kept (imaginary parts of the k = 0 and
    k = n/2 coefficients therefore drop out)."""
    y = np.asarray(xh, dtype=np.complex128)
    for axis in range(y.ndim - 1):
        y = partial_dft(y, axis, BACKWARD)
    y = hermitian_extend_last(y, n_last)
    y = partial_dft(y, y.ndim - 1, BACKWARD)
    return np.ascontiguousarray(y.real)


def distributed_rfft_forward(buf_real, shape, grid, exchange=redistribute.exchange_subarray):
    """r2c on the virtual grid: stage 0 real buffer -> stage g complex buffer of the
    global shape shape[:-1] + (shape[-1]//2 + 1,)."""
    d, g = len(shape), len(grid)
    cshape = tuple(shape[:-1]) + (shape[-1] // 2 + 1,)
    # Real stage-0 local arrays have the full last axis: transform each rank.
    layout_r, _ = decomp.stage_layout(shape, grid, 0)
    layout_c, total_c = decomp.stage_layout(cshape, grid, 0)
    y = np.empty(total_c, dtype=np.complex128)
    for (st, sz, off), (stc, szc, offc) in zip(layout_r, layout_c):
        loc = np.asarray(buf_real[off:off + math.prod(sz)], dtype=np.float64).reshape(sz)
        full = partial_dft(loc.astype(np.complex128), d - 1, FORWARD)
        y[offc:offc + math.prod(szc)] = full[..., :cshape[-1]].reshape(-1)
    for axis in reversed(range(g, d - 1)):
        y = _transform_ranks(y, cshape, grid, 0, axis, FORWARD)
    for s in range(1, g + 1):
        y = exchange(y, cshape, grid, s - 1, s)
        y = _transform_ranks(y, cshape, grid, s, g - s, FORWARD)
    return y


def distributed_irfft_backward(buf_c, shape, grid, exchange=redistribute.exchange_subarray):
    """c2r on the virtual grid: stage g complex buffer -> stage 0 real buffer."""
    d, g = len(shape), len(grid)
    cshape = tuple(shape[:-1]) + (shape[-1] // 2 + 1,)
    y = np.asarray(buf_c, dtype=np.complex128)
    for s in range(g, 0, -1):
        y = _transform_ranks(y, cshape, grid, s, g - s, BACKWARD)
        y = exchange(y, cshape, grid, s, s - 1)
    for axis in range(g, d - 1):
        y = _transform_ranks(y, cshape, grid, 0, axis, BACKWARD)
    layout_r, total_r = decomp.stage_layout(shape, grid, 0)
    layout_c, _ = decomp.stage_layout(cshape, grid, 0)
    out = np.empty(total_r, dtype=np.float64)
    for (st, sz, off), (stc, szc, offc) in zip(layout_r, layout_c):
        loc = y[offc:offc + math.prod(szc)].reshape(szc)
        full = hermitian_extend_last(loc, shape[-1])
        out[off:off + math.prod(sz)] = partial_dft(full, d - 1, BACKWARD).real.reshape(-1)
    return out


def forward_at(x: np.ndarray, ks, chunk: int = 32) -> np.ndarray:
    """Selected outputs of the d-D forward transform (Eq. multifft), one index at a time.

    X[k] = sum_{j_0} (w_0^{k_0 j_0} / N_0) ... sum_{j_{d-1}} (w_{d-1}^{k_{d-1} j_{d-1}} / N_{d-1}) x[j]
    evaluated by contracting the last axis first, ``chunk`` slices of axis 0 at a
    time so that large arrays (e.g. 512^3) need little extra memory.
    """
    x = np.asarray(x)
    shape = x.shape
    d = x.ndim
    out = np.empty(len(ks), dtype=np.complex128)
    for n, k in enumerate(ks):
        vecs = []
        for m in range(d):
            j = np.arange(shape[m], dtype=np.int64)
            vecs.append(np.exp(-2j * np.pi * ((k[m] * j) % shape[m]) / shape[m]) / shape[m])
        acc = np.zeros((), dtype=np.complex128)
        for a in range(0, shape[0], chunk):
            blk = x[a:a + chunk].astype(np.complex128)
            for m in range(d - 1, 0, -1):
                blk = blk @ vecs[m]
            acc = acc + blk @ vecs[0][a:a + chunk]
        out[n] = acc
    return out
