"""Copy tasks of the subarray exchange kernel, emulated on the CPU (no GPU).

The planner cuts every box of Alg. 3's exchange (and of the traditional
pack -> all-to-all -> unpack of Sec. 3.3.1) into 2-D copy tasks.  Here each
box-copy launch of the unfused and packed step lists is replayed with NumPy
from the tasks the library reports (tfft_plan_copy_tasks): the tasks must
stay inside their buffers, write every element exactly once, and compose to
the oracle's exchange between the same stages, bit for bit.
"""
import ctypes

import numpy as np
import pytest

from oracle import redistribute as R

SHAPES = [
    ((32, 32, 32), (2, 2)),
    ((64, 64, 64), (4, 8)),
    ((6, 10, 12), (3, 2)),
    ((5, 6, 8), (4, 3)),            # zero-size ranks
    ((42, 127, 256), (3, 4)),       # App. A shape, uneven blocks
    ((12, 10, 8, 6), (2, 3, 2)),    # 4-D on a 3-D grid
    ((16, 17, 18, 19), (2, 3, 2)),
    ((64, 96), (4,)),
    ((1, 16, 8), (1, 2)),
    ((16, 8, 1), (2, 2)),           # unit innermost axis: strided rows of one element
    ((512, 64, 64), (4, 8)),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09536_gb300 import build, _lib
    build.build()
    return _lib.load()


def _tasks(lib, handle, sign, mode, index):
    n = ctypes.c_int64()
    assert lib.tfft_plan_copy_tasks(handle, sign, mode, index, None, 0, ctypes.byref(n)) == 0
    buf = (ctypes.c_int64 * (6 * max(1, n.value)))()
    assert lib.tfft_plan_copy_tasks(handle, sign, mode, index, buf, n.value, ctypes.byref(n)) == 0
    return np.frombuffer(buf, dtype=np.int64)[:6 * n.value].reshape(-1, 6)


def _replay(tasks, src, n_out):
    """out[dst + r ds + c] = src[src + r ss + c]; checks bounds and single writes."""
    out = np.full(n_out, np.nan + 1j * np.nan, dtype=np.complex128)
    hits = np.zeros(n_out, dtype=np.int64)
    for s0, d0, ss, ds, nrows, rowlen in tasks:
        assert nrows >= 1 and rowlen >= 1
        r = np.arange(nrows, dtype=np.int64)[:, None]
        c = np.arange(rowlen, dtype=np.int64)[None, :]
        si = (s0 + r * ss + c).ravel()
        di = (d0 + r * ds + c).ravel()
        assert si.min() >= 0 and si.max() < src.size, "source index out of the buffer"
        assert di.min() >= 0 and di.max() < n_out, "destination index out of the buffer"
        out[di] = src[si]
        np.add.at(hits, di, 1)
    assert np.all(hits == 1), "every element written exactly once"
    return out


@pytest.mark.parametrize("shape,grid", SHAPES)
def test_copy_tasks_compose_to_the_exchange(lib, shape, grid):
    from paper_1804_09536_gb300 import _lib
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, bind=False)
    g = len(grid)
    n = p.stage_elems(0)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for mode in (_lib.TFFT_MODE_UNFUSED, _lib.TFFT_MODE_PACKED):
        for sign in (-1, 1):
            names = [nm for nm, _ in p.launch_info(sign, {1: "unfused", 2: "packed"}[mode])]
            # consecutive box copies form one exchange; forward: stage k-1 -> k,
            # backward: stage g-k+1 -> g-k (k = 1, 2, ...)
            groups, cur = [], []
            for i, nm in enumerate(names):
                if nm == "box_copy":
                    cur.append(i)
                elif cur:
                    groups.append(cur)
                    cur = []
            if cur:
                groups.append(cur)
            assert len(groups) == g
            for k, grp in enumerate(groups, start=1):
                s_from, s_to = (k - 1, k) if sign < 0 else (g - k + 1, g - k)
                buf = R.scatter(x, grid, s_from)
                want = R.exchange_subarray(buf, shape, grid, s_from, s_to)
                cur_buf = buf
                for idx in grp:
                    cur_buf = _replay(_tasks(lib, p.handle, sign, mode, idx), cur_buf, n)
                assert np.array_equal(cur_buf.view(np.uint8), want.view(np.uint8)), (mode, sign, k)


def test_copy_tasks_rejects_fft_launches(lib):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan((16, 16, 16), (2, 2), bind=False)
    n = ctypes.c_int64()
    assert lib.tfft_plan_copy_tasks(p.handle, -1, 0, 0, None, 0, ctypes.byref(n)) == 1
