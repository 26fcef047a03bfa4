"""Pins for oracle.decomp: decomposition, process grid, stage layouts (CPU only)."""
import math
import os

import pytest

from oracle import decomp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def check_decompose_closed_form(fn=None):
    """Eq. decompose / Alg. 1: n_p = q + [r > p]; parts tile 0..N-1 contiguously."""
    fn = fn or decomp.decompose
    for N in range(0, 65):
        for M in range(1, 17):
            q, r = divmod(N, M)
            nxt = 0
            total = 0
            for p in range(M):
                n, s = fn(N, M, p)
                assert n == (q + 1 if p < r else q), (N, M, p, n)
                assert s == nxt, (N, M, p, s)          # s_p = s_{p-1} + n_{p-1}
                nxt = s + n
                total += n
            assert total == N                            # sum_p n_p = N
            # balanced: lengths differ by at most one
            lens = [fn(N, M, p)[0] for p in range(M)]
            assert max(lens) - min(lens) <= 1


def test_decompose_closed_form():
    check_decompose_closed_form()


def test_decompose_alg1_agrees():
    for N in range(0, 65):
        for M in range(1, 17):
            for p in range(M):
                assert decomp.decompose(N, M, p) == decomp.decompose_alg1(N, M, p)


def test_decompose_rejects_bad_args():
    for args in [(-1, 2, 0), (4, 0, 0), (4, 2, 2), (4, 2, -1)]:
        with pytest.raises(ValueError):
            decomp.decompose(*args)


def test_subarray_boxes_partition_axis():
    sizes = (5, 7, 3)
    for axis in range(3):
        for M in (1, 2, 3, 4, 9):
            boxes = decomp.subarray_boxes(sizes, axis, M)
            covered = []
            for subsizes, substarts in boxes:
                for m in range(3):
                    if m != axis:
                        assert subsizes[m] == sizes[m] and substarts[m] == 0
                covered.extend(range(substarts[axis], substarts[axis] + subsizes[axis]))
            assert covered == list(range(sizes[axis]))


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_grid_matches_paper_example():
    """Sec. 3.4-3.5 worked example on a 3 x 4 grid (tests/golden/subgroups_3x4.txt)."""
    lines = _golden_lines("subgroups_3x4.txt")
    grid = tuple(int(v) for v in lines[0][1:])
    assert grid == (3, 4)
    for ln in lines:
        if ln[0] == "coords":
            c = (int(ln[1]), int(ln[2]))
            r = int(ln[4])
            assert decomp.coords_to_rank(c, grid) == r
            assert decomp.rank_to_coords(r, grid) == c
        if ln[0] == "subgroup_P0_containing":
            want = [int(v) for v in ln[3:]]
            groups = decomp.subgroups(grid, 0)
            assert want in groups
        if ln[0] == "count_P0":
            assert len(decomp.subgroups(grid, 0)) == int(ln[1])
            assert all(len(g) == int(ln[3]) for g in decomp.subgroups(grid, 0))
        if ln[0] == "count_P1":
            assert len(decomp.subgroups(grid, 1)) == int(ln[1])
            assert all(len(g) == int(ln[3]) for g in decomp.subgroups(grid, 1))


def check_pencil_shapes(local_box=None):
    """Local shapes of the appendix's sizesA / sizesB / sizesC for App. A's array."""
    local_box = local_box or decomp.local_box
    shape = (42, 127, 256)
    for grid in [(2, 3), (3, 4), (4, 8), (1, 5)]:
        for r in range(math.prod(grid)):
            p0, p1 = decomp.rank_to_coords(r, grid)
            n0 = decomp.decompose(42, grid[0], p0)[0]
            n1 = decomp.decompose(127, grid[1], p1)[0]
            n2 = decomp.decompose(256, grid[1], p1)[0]
            m1 = decomp.decompose(127, grid[0], p0)[0]
            assert local_box(shape, grid, 0, r)[1] == (n0, n1, 256)     # sizesA
            assert local_box(shape, grid, 1, r)[1] == (n0, 127, n2)     # sizesB
            assert local_box(shape, grid, 2, r)[1] == (42, m1, n2)      # sizesC


def test_pencil_stage_shapes_appendix_a():
    check_pencil_shapes()


def test_pencil_512_4x8_shapes():
    shape, grid = (512, 512, 512), (4, 8)
    assert decomp.local_box(shape, grid, 0, 0)[1] == (128, 64, 512)
    assert decomp.local_box(shape, grid, 1, 0)[1] == (128, 512, 64)
    assert decomp.local_box(shape, grid, 2, 0)[1] == (512, 128, 64)


def test_slab_and_4d_stage_owners():
    # Slab (Eqs. slab0-slab1): stage 0 cuts axis 0, stage 1 cuts axis 1.
    assert decomp.axis_owner(3, (8,), 0) == [0, None, None]
    assert decomp.axis_owner(3, (8,), 1) == [None, 0, None]
    # 4-D on a 3-D grid (Eqs. 4d_fft0 - 4d_fft3).
    assert decomp.axis_owner(4, (2, 2, 2), 0) == [0, 1, 2, None]
    assert decomp.axis_owner(4, (2, 2, 2), 1) == [0, 1, None, 2]
    assert decomp.axis_owner(4, (2, 2, 2), 2) == [0, None, 1, 2]
    assert decomp.axis_owner(4, (2, 2, 2), 3) == [None, 0, 1, 2]
    # exchanges of the pencil method: 2 -> 1 in P_1, then 1 -> 0 in P_0
    assert decomp.exchange_between(3, (4, 8), 0, 1) == (1, 2, 1)
    assert decomp.exchange_between(3, (4, 8), 1, 2) == (0, 1, 0)


def test_stage_layout_covers_every_element_once():
    for shape, grid in [((5, 7, 6), (2, 3)), ((3, 2, 4), (4, 2)), ((6, 5, 4, 3), (2, 2, 1)),
                        ((7, 9, 10), (5,))]:
        for s in range(len(grid) + 1):
            layout, total = decomp.stage_layout(shape, grid, s)
            assert total == math.prod(shape)
            seen = set()
            for starts, sizes, off in layout:
                for idx in decomp.iter_global_index(sizes):
                    g = tuple(a + b for a, b in zip(starts, idx))
                    assert g not in seen
                    seen.add(g)
            assert len(seen) == math.prod(shape)
