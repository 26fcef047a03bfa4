"""Index-level global redistribution on the virtual grid (oracle; test infrastructure only).

Three independent constructions of the same permutation of elements:

1. ``redistribute``: gather the whole global array from the stage buffer by
   explicit slicing, then scatter it into the target stage (the definition:
   every element keeps its global position, only its owner changes; Fig. 2c
   caption).
2. ``exchange_subarray``: the paper's method, Alg. 3 / Eq. gt.  Within each
   one-dimensional subgroup P_i, each rank a cuts its input A along its aligned
   axis v into M boxes (Alg. 2); box q goes to peer q, which stores it in the
   a-th box of its output B cut along axis w.  All pairs are one all-to-all-w.
3. ``exchange_traditional``: Sec. 3.3.1, Eq. transpose: reshape the aligned
   axis v into (M, N_v / M), move the M-axis to the front (the local transpose),
   all-to-all contiguous chunks, then place the received chunks along axis w.
   Divisible shapes only (the paper notes all-to-all-v is needed otherwise).

All three copy values unchanged, so they must agree bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

from . import decomp


def _local_view(buf, layout_entry):
    starts, sizes, offset = layout_entry
    n = math.prod(sizes)
    return buf[offset:offset + n].reshape(sizes)


def local_arrays(buf, shape, grid, stage):
    """Views of every rank's local array inside the concatenated stage buffer."""
    layout, total = decomp.stage_layout(shape, grid, stage)
    if buf.size != total:
        raise ValueError(f"buffer has {buf.size} elements, stage {stage} needs {total}")
    return [_local_view(buf, e) for e in layout]


def scatter(x, grid, stage):
    """Global array -> concatenated stage buffer (each rank's block, rank order)."""
    layout, total = decomp.stage_layout(x.shape, grid, stage)
    buf = np.empty(total, dtype=x.dtype)
    for starts, sizes, offset in layout:
        sl = tuple(slice(s, s + n) for s, n in zip(starts, sizes))
        buf[offset:offset + math.prod(sizes)] = x[sl].reshape(-1)
    return buf


def gather(buf, shape, grid, stage):
    """Concatenated stage buffer -> global array."""
    layout, total = decomp.stage_layout(shape, grid, stage)
    if buf.size != total:
        raise ValueError("buffer size does not match the stage layout")
    x = np.empty(shape, dtype=buf.dtype)
    for starts, sizes, offset in layout:
        sl = tuple(slice(s, s + n) for s, n in zip(starts, sizes))
        x[sl] = buf[offset:offset + math.prod(sizes)].reshape(sizes)
    return x


def redistribute(buf, shape, grid, s_from, s_to):
    """Construction 1: scatter(gather(buf, s_from), s_to); any pair of stages."""
    return scatter(gather(buf, shape, grid, s_from), grid, s_to)


def exchange_subarray(buf, shape, grid, s_from, s_to):
    """Construction 2 (Alg. 3, Eq. gt): subarray boxes + all-to-all-w, per subgroup."""
    d = len(shape)
    i, v, w = decomp.exchange_between(d, grid, s_from, s_to)
    A = local_arrays(buf, shape, grid, s_from)
    out_layout, total = decomp.stage_layout(shape, grid, s_to)
    out = np.empty(total, dtype=buf.dtype)
    B = [_local_view(out, e) for e in out_layout]
    M = grid[i]
    for group in decomp.subgroups(grid, i):        # concurrent exchanges on subslabs
        for a_idx, a in enumerate(group):
            send = decomp.subarray_boxes(A[a].shape, v, M)      # S_A: cut aligned axis v
            for q_idx, q in enumerate(group):
                recv = decomp.subarray_boxes(B[q].shape, w, M)  # S_B: cut axis w
                ssz, sst = send[q_idx]
                rsz, rst = recv[a_idx]
                assert ssz == rsz, (ssz, rsz)
                src = tuple(slice(s, s + n) for s, n in zip(sst, ssz))
                dst = tuple(slice(s, s + n) for s, n in zip(rst, rsz))
                B[q][dst] = A[a][src]
    return out


def exchange_traditional(buf, shape, grid, s_from, s_to):
    """Construction 3 (Sec. 3.3.1, Eq. transpose): local transpose + contiguous all-to-all.

    Requires N_v and N_w divisible by the subgroup size.
    """
    d = len(shape)
    i, v, w = decomp.exchange_between(d, grid, s_from, s_to)
    M = grid[i]
    if shape[v] % M or shape[w] % M:
        raise ValueError("traditional exchange needs divisible shapes")
    A = local_arrays(buf, shape, grid, s_from)
    out_layout, total = decomp.stage_layout(shape, grid, s_to)
    out = np.empty(total, dtype=buf.dtype)
    B = [_local_view(out, e) for e in out_layout]
    for group in decomp.subgroups(grid, i):
        # Local transpose (pack): axis v of extent N_v -> (M, N_v/M), M-axis first.
        packed = []
        for a in group:
            x = A[a]
            sh = list(x.shape)
            split = sh[:v] + [M, sh[v] // M] + sh[v + 1:]
            y = np.moveaxis(x.reshape(split), v, 0)          # (M, ..., N_v/M, ...)
            packed.append(np.ascontiguousarray(y))
        # All-to-all of contiguous chunks: rank q receives chunk q from every a.
        for q_idx, q in enumerate(group):
            recv = np.stack([packed[a_idx][q_idx] for a_idx in range(M)])  # (M, ...)
            # Unpack: the received M-axis becomes the high part of axis w.
            z = np.moveaxis(recv, 0, w)                        # (..., M, n_w, ...)
            zs = list(z.shape)
            merged = zs[:w] + [zs[w] * zs[w + 1]] + zs[w + 2:]
            B[q][...] = z.reshape(merged)
    return out
