"""Decomposition, virtual process grid and stage layouts (oracle; test infrastructure only).

Sec. 3.1 (Eq. decompose, Alg. 1): a balanced block-contiguous decomposition of
N elements in M parts gives part p the length n_p = q + 1 if r > p else q
(q = N // M, r = N mod M) and the start s_p = n_0 + ... + n_{p-1}.

Sec. 3.4 (Fig. 3): an M_0 x M_1 (x ...) Cartesian grid of processes; process
coordinates (p_0, p_1, ...) are in C row-major order of the rank.  The grid
splits into one-dimensional subgroups P_i: the processes that share every
coordinate except p_i.

Stage layouts (Eqs. slab0-slab1, pencil0-pencil2, 4d_fft0-4d_fft3): a d-D
array on a g-D grid (g <= d - 1, Sec. 3.6) passes through g + 1 alignments.
In stage 0 grid direction i distributes axis i (i < g); every exchange moves
one direction i, from i = g - 1 down to 0, from axis i to axis i + 1.  So in
stage s direction i distributes axis i when i < g - s and axis i + 1 otherwise,
and the axis that stage s newly holds in full is g - s.

The virtual grid lives in one buffer: each rank's local array in C order,
concatenated in rank order (a convention of this build; the paper's processes
have separate memories).
"""
from __future__ import annotations

import itertools
import math


def decompose(N: int, M: int, p: int):
    """Local length and start of part p (Eq. decompose; s_p by the recursion of Sec. 3.1).

    N >= 0 elements, M > 0 parts, 0 <= p < M (Alg. 1 input contract).
    """
    if N < 0 or M <= 0 or not (0 <= p < M):
        raise ValueError(f"decompose: bad arguments N={N} M={M} p={p}")
    q, r = N // M, N % M
    lengths = [q + 1 if r > k else q for k in range(M)]
    start = 0
    for k in range(p):          # s_0 = 0, s_k = s_{k-1} + n_{k-1}
        start += lengths[k]
    return lengths[p], start


def decompose_alg1(N: int, M: int, p: int):
    """Alg. 1 in its two-branch form (used as a cross-check of ``decompose``)."""
    q = N // M
    r = N % M
    if r > p:
        n = q + 1
        s = n * p
    else:
        n = q
        s = n * p + r
    return n, s


def subarray_boxes(sizes, axis: int, nparts: int):
    """Alg. 2: for each part p, the box (subsizes, substarts) that cuts ``axis``.

    Every axis keeps its full extent and zero start except ``axis``, which gets
    the p-th block of the balanced decomposition of ``sizes[axis]``.
    """
    boxes = []
    for p in range(nparts):
        subsizes = list(sizes)
        substarts = [0] * len(sizes)
        n, s = decompose(sizes[axis], nparts, p)
        subsizes[axis] = n
        substarts[axis] = s
        boxes.append((tuple(subsizes), tuple(substarts)))
    return boxes


# ---------------------------------------------------------------- process grid

def rank_to_coords(rank: int, grid):
    """Row-major Cartesian coordinates of ``rank`` on ``grid`` (Sec. 3.4)."""
    coords = []
    for m in reversed(grid):
        coords.append(rank % m)
        rank //= m
    return tuple(reversed(coords))


def coords_to_rank(coords, grid) -> int:
    r = 0
    for c, m in zip(coords, grid):
        r = r * m + c
    return r


def nranks(grid) -> int:
    return math.prod(grid)


def subgroups(grid, direction: int):
    """The one-dimensional subgroups P_direction: lists of ranks, ordered by p_direction."""
    groups = {}
    for r in range(nranks(grid)):
        c = rank_to_coords(r, grid)
        key = c[:direction] + c[direction + 1:]
        groups.setdefault(key, []).append(r)
    return [groups[k] for k in sorted(groups)]


# ---------------------------------------------------------------- stage layouts

def num_stages(grid) -> int:
    return len(grid) + 1


def axis_owner(d: int, grid, stage: int):
    """owner[m] = grid direction that distributes axis m in ``stage``, or None."""
    g = len(grid)
    if not (0 <= stage <= g) or g > d - 1:
        raise ValueError("bad stage or grid dimensionality")
    owner = [None] * d
    for i in range(g):
        axis = i if i < g - stage else i + 1
        owner[axis] = i
    return owner


def aligned_axis(d: int, grid, stage: int) -> int:
    """The axis stage ``stage`` newly holds in full (the one its FFT pass transforms)."""
    return len(grid) - stage


def local_box(shape, grid, stage: int, rank: int):
    """(starts, sizes) of ``rank``'s block of the global array in ``stage``."""
    d = len(shape)
    owner = axis_owner(d, grid, stage)
    coords = rank_to_coords(rank, grid)
    starts, sizes = [], []
    for m in range(d):
        if owner[m] is None:
            starts.append(0)
            sizes.append(shape[m])
        else:
            i = owner[m]
            n, s = decompose(shape[m], grid[i], coords[i])
            starts.append(s)
            sizes.append(n)
    return tuple(starts), tuple(sizes)


def stage_layout(shape, grid, stage: int):
    """Per rank (starts, sizes, offset) in the concatenated buffer, and the total length."""
    out = []
    offset = 0
    for r in range(nranks(grid)):
        starts, sizes = local_box(shape, grid, stage, r)
        out.append((starts, sizes, offset))
        offset += math.prod(sizes)
    return out, offset


def exchange_between(d: int, grid, s_from: int, s_to: int):
    """For adjacent stages: (direction i, v, w) of the exchange Exchange(P_i, A, v, B, w).

    A (stage s_from) holds axis v in full and has axis w cut by direction i;
    B (stage s_to) holds axis w in full and has axis v cut by direction i.
    """
    if abs(s_from - s_to) != 1:
        raise ValueError("exchange only between adjacent stages")
    g = len(grid)
    i = g - max(s_from, s_to)
    own_from = axis_owner(d, grid, s_from)
    own_to = axis_owner(d, grid, s_to)
    w = own_from.index(i)
    v = own_to.index(i)
    return i, v, w


def all_local_boxes(shape, grid, stage: int):
    return [local_box(shape, grid, stage, r) for r in range(nranks(grid))]


def iter_global_index(shape):
    return itertools.product(*[range(n) for n in shape])
