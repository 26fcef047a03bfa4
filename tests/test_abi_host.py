"""C-ABI library: loads, exports every declared symbol, host-side plan queries (CPU only).

No compute call is made here: plan creation and layout queries are host code.
"""
import ctypes
import math
import os
import re

import pytest

from oracle import decomp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tfft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09536_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tfft_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_functions():
    names = declared_functions()
    assert "tfft_execute" in names and "tfft_redistribute" in names and len(names) >= 15


def test_every_declared_symbol_exported(lib):
    from paper_1804_09536_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no binding"


def test_decompose_abi_matches_oracle(lib):
    n = ctypes.c_int64()
    s = ctypes.c_int64()
    for N in range(0, 40):
        for M in range(1, 9):
            for p in range(M):
                assert lib.tfft_decompose(N, M, p, ctypes.byref(n), ctypes.byref(s)) == 0
                assert (n.value, s.value) == decomp.decompose(N, M, p)
    assert lib.tfft_decompose(4, 0, 0, ctypes.byref(n), ctypes.byref(s)) == 1
    assert lib.tfft_decompose(4, 2, 2, ctypes.byref(n), ctypes.byref(s)) == 1


@pytest.mark.parametrize("shape,grid", [((32, 32, 32), (2, 2)), ((512, 512, 512), (4, 8)),
                                        ((42, 127, 256), (3, 4)), ((256, 256, 256), (8,)),
                                        ((3, 2, 5), (4, 3)), ((16, 17, 18, 20), (2, 3, 2)),
                                        ((64, 128, 256), (2, 4)), ((8,), ())])
def test_plan_layouts_match_oracle(lib, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, bind=False)
    assert p.num_stages == len(grid) + 1
    assert p.num_ranks == math.prod(grid)
    for s in range(len(grid) + 1):
        layout, total = decomp.stage_layout(shape, grid, s)
        assert p.stage_elems(s) == total
        assert p.stage_axis(s) == decomp.aligned_axis(len(shape), grid, s)
        for r, (st, sz, off) in enumerate(layout):
            assert p.local_box(s, r) == (st, sz, off)


def test_unsupported_and_invalid(lib):
    from paper_1804_09536_gb300.plan import Plan
    from paper_1804_09536_gb300._lib import TfftError
    p = Plan((4099, 8, 8), (2, 2), bind=False)  # prime length above 2048: plans and redistributes ...
    with pytest.raises(TfftError) as e:
        p.num_launches(-1)                        # ... but does not transform
    assert e.value.status == 2
    assert Plan((7, 127, 8), (2, 2), bind=False).num_launches(-1) == 3  # Bluestein lengths do
    with pytest.raises(TfftError) as e:
        Plan((8, 8, 8), (2, 2, 2), bind=False)
    assert e.value.status == 1  # grid_ndims > ndims - 1 (Sec. 3.6)
    with pytest.raises(TfftError):
        Plan((8, 8, 8), (0, 2), bind=False)
    with pytest.raises(TfftError):
        Plan((0, 8, 8), (2, 2), bind=False)


def test_calls_validate_before_launch(lib):
    """Unbound plan and bad pointers are rejected without touching a GPU."""
    from paper_1804_09536_gb300.plan import Plan
    p = Plan((8, 8, 8), (2, 2), bind=False)
    rc = lib.tfft_execute(p.handle, -1, 0, ctypes.c_void_p(16), ctypes.c_void_p(4096),
                          None, 0, None)
    assert rc == 6  # TFFT_ESTATE: not bound
    rc = lib.tfft_redistribute(p.handle, 2, 1, ctypes.c_void_p(16), ctypes.c_void_p(4096), None)
    assert rc == 6
    rc = lib.tfft_plan_bind(p.handle, ctypes.c_void_p(8), 1 << 20, None)
    assert rc == 3  # TFFT_EALIGN
    rc = lib.tfft_plan_bind(p.handle, None, 1 << 20, None)
    assert rc == 1


def test_launch_counts(lib):
    from paper_1804_09536_gb300.plan import Plan
    p = Plan((32, 32, 32), (2, 2), bind=False)
    assert p.num_launches(-1, "fused") == 3
    assert p.num_launches(1, "fused") == 3
    assert p.num_launches(-1, "unfused") == 5
    # packed: the 2 -> 1 exchange needs pack + all-to-all + unpack, 1 -> 0 needs pack + all-to-all
    assert p.num_launches(-1, "packed") >= 7


def _batch_order(lib, problems):
    from paper_1804_09536_gb300.plan import Plan
    plans = [Plan(sh, gr, bind=False) for sh, gr in problems]
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    b = ctypes.c_void_p()
    assert lib.tfft_batch_create(ctypes.byref(b), len(plans), arr, -1) == 0
    try:
        items, segs = ctypes.c_int64(), ctypes.c_int()
        assert lib.tfft_batch_num_items(b, ctypes.byref(items), ctypes.byref(segs)) == 0
        t, k = ctypes.c_int(), ctypes.c_int()
        order = []
        for i in range(segs.value):
            assert lib.tfft_batch_segment(b, i, ctypes.byref(t), ctypes.byref(k)) == 0
            order.append((t.value, k.value))
        assert lib.tfft_batch_segment(b, segs.value, ctypes.byref(t), ctypes.byref(k)) == 1
        npass = [p.num_launches(-1, "fused") for p in plans]
    finally:
        lib.tfft_batch_destroy(b)
    return order, npass


@pytest.mark.parametrize("which", ["bench48", "mixed"])
def test_batch_issue_order(lib, which):
    """Every pass of every transform exactly once, pass-major: all first
    passes (transform order), then all second passes, ..."""
    from paper_1804_09536_gb300 import inputs
    if which == "bench48":
        problems = inputs.batch_problems(48, seed=0)
    else:
        problems = [((256, 256, 256), (2, 4)), ((64, 96), (4,)), ((128, 128, 128), (2, 2)),
                    ((128,), ()), ((96, 96, 96), (2, 2))]
    order, npass = _batch_order(lib, problems)
    want = [(t, k) for k in range(max(npass)) for t in range(len(problems)) if k < npass[t]]
    assert order == want


def test_batch_executor_choice(lib):
    """The stream executor is chosen and queried on the host (no GPU work):
    stream counts are clipped to the transform count, bad values rejected,
    and the persistent kernel stays the default."""
    from paper_1804_09536_gb300.plan import Plan
    plans = [Plan(sh, gr, bind=False) for sh, gr in [((64, 64, 64), (2, 2)), ((96, 96, 96), (2, 2)),
                                                      ((128, 128, 128), (2, 4))]]
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    b = ctypes.c_void_p()
    assert lib.tfft_batch_create(ctypes.byref(b), len(plans), arr, -1) == 0
    e, k = ctypes.c_int(), ctypes.c_int()
    try:
        assert lib.tfft_batch_executor(b, ctypes.byref(e), ctypes.byref(k)) == 0
        assert (e.value, k.value) == (0, 0)
        assert lib.tfft_batch_set_executor(b, 1, 2) == 0
        assert lib.tfft_batch_executor(b, ctypes.byref(e), ctypes.byref(k)) == 0
        assert (e.value, k.value) == (1, 2)
        assert lib.tfft_batch_set_executor(b, 1, 8) == 0     # more streams than transforms
        assert lib.tfft_batch_executor(b, ctypes.byref(e), ctypes.byref(k)) == 0
        assert (e.value, k.value) == (1, 3)
        assert lib.tfft_batch_set_executor(b, 1, 0) == 1
        assert lib.tfft_batch_set_executor(b, 1, 17) == 1
        assert lib.tfft_batch_set_executor(b, 2, 1) == 1
        assert lib.tfft_batch_set_executor(b, 0, 0) == 0
        assert lib.tfft_batch_executor(b, ctypes.byref(e), ctypes.byref(k)) == 0
        assert (e.value, k.value) == (0, 0)
        # executing an unbound batch is refused before any GPU work
        assert lib.tfft_batch_set_executor(b, 1, 2) == 0
        assert lib.tfft_batch_execute(b, None) == 6
    finally:
        lib.tfft_batch_destroy(b)


@pytest.mark.parametrize("shape,grid,c0,nc", [((512, 512, 512), (4, 8), 33, 224),
                                               ((64, 128, 512), (4, 8), 33, 224),
                                               ((128, 64, 256), (2, 4), 33, 96),
                                               ((16, 512, 120), (2, 4), 0, 16)])
def test_r2c_column_window_plan(lib, shape, grid, c0, nc):
    """Real-to-complex plans with odd stage-0 rows: the fused gathering pass
    along axis 1 is one TMA step over the column window plus the plain kernel
    over the other columns; their algorithmic bytes add up to one whole pass,
    and the fused workspace is the padded stage-0 buffer (rows of an even
    pitch, the window's first column on a 16-byte boundary).  Unfused, packed
    and no-TMA plans keep the plain layouts."""
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, kind="r2c", bind=False)
    n2 = shape[-1] // 2 + 1
    rows = math.prod(shape[:-1])
    # rows padded so that the window's first column starts a 128-byte line,
    # unless that costs over 1/16 more memory (then a 16-byte boundary)
    lead = (16 - c0 % 16) % 16
    pitch = (lead + n2 + 15) // 16 * 16
    if 16 * (pitch - n2) > n2:
        lead = c0 % 2
        pitch = (lead + n2 + 1) // 2 * 2
    assert (lead + c0) * 8 % 16 == 0 and pitch * 8 % 16 == 0
    assert p.workspace_bytes("fused") == 8 * rows * pitch
    assert p.workspace_bytes("unfused") == 2 * 8 * rows * n2
    whole = 2 * 8 * rows * n2
    for sign in (-1, 1):
        info = p.launch_info(sign)
        win = [b for n, b in info if "tma_window" in n]
        rest = [b for n, b in info if n.startswith("fft_strided_L")]
        assert len(win) == 1 and len(rest) == 1, info
        assert win[0] == 2 * 8 * rows * nc
        assert win[0] + rest[0] == whole
        assert p.num_launches(sign, "fused") == len(info) == 4
        assert not any("window" in n for n, _ in p.launch_info(sign, "unfused"))
    q = Plan(shape, grid, kind="r2c", bind=False, tma=False)
    assert q.workspace_bytes("fused") == 8 * rows * n2
    assert not any("window" in n for n, _ in q.launch_info(-1))
    c = Plan(shape, grid, kind="r2c", bind=False, precision="bf16x3")
    assert not any("window" in n for n, _ in c.launch_info(-1))


def test_launch_bytes_account_for_every_pass(lib):
    """Host-side roofline accounting over a seeded sweep of plans: the fused
    path's launches report one read and one write of every element per pass
    (a real-to-complex pass: the real array plus the complex half), whatever
    the column splits (windows, rank groups, plain remainders); the fused
    workspace is at least one complex stage and at most 1/16 larger."""
    import random
    from paper_1804_09536_gb300.plan import Plan
    from paper_1804_09536_gb300._lib import TfftError
    rng = random.Random(5)
    lens = [8, 16, 24, 32, 48, 60, 64, 96, 120, 128, 160, 192, 240, 256, 512]
    checked = 0
    while checked < 60:
        d = rng.choice([2, 3, 3])
        shape = tuple(rng.choice(lens) for _ in range(d))
        grid = tuple(rng.choice([1, 2, 3, 4, 8]) for _ in range(rng.randint(1, d - 1)))
        kind = rng.choice(["c2c", "r2c"])
        try:
            p = Plan(shape, grid, kind=kind, bind=False)
            info = p.launch_info(-1) + p.launch_info(1)
        except TfftError:
            continue
        n = math.prod(shape)
        nc = n if kind == "c2c" else n // shape[-1] * (shape[-1] // 2 + 1)
        want = 2 * d * 16 * nc
        if kind == "r2c":
            want += 2 * (4 * n + 8 * nc) - 2 * 16 * nc
        assert sum(b for _, b in info) == want, (shape, grid, kind, info)
        ws = p.workspace_bytes("fused")
        if kind == "r2c":
            assert 8 * nc <= ws <= 8 * nc + 8 * nc // 16 + 64, (shape, grid, ws)
        checked += 1


def test_plan_flags(lib):
    """Known flag bits are accepted together; any other bit is rejected."""
    from paper_1804_09536_gb300 import _lib
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 3)(16, 16, 16)
    grd = (ctypes.c_int * 2)(2, 2)
    every = _lib.TFFT_NORM_BACKWARD | _lib.TFFT_NO_TMA | _lib.TFFT_NO_GRAPH
    assert lib.tfft_plan_create(ctypes.byref(h), 3, shp, 2, grd, _lib.TFFT_C2C, _lib.TFFT_FP32, every) == 0
    lib.tfft_plan_destroy(h)
    for bad in (1, 2, 32, 1 << 20):
        assert lib.tfft_plan_create(ctypes.byref(h), 3, shp, 2, grd, _lib.TFFT_C2C, _lib.TFFT_FP32, bad) == 1
