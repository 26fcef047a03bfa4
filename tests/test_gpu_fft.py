"""GPU parity: whole transforms vs the FP64 oracle (needs a GPU).

rel-L2 <= 1e-5 against the oracle for the fused path and both comparison
paths; the three paths run the same butterflies on every line, so their
outputs must also agree bit for bit.
"""
import math

import numpy as np
import pytest
import torch

from oracle import dft, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, bits, rel_l2, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    ((32, 32, 32), (2, 2)),          # the 32^3 pencil 2 x 2 parity workload
    ((8, 8, 8), (2, 2)),
    ((6, 10, 12), (3, 2)),           # mixed radix 2/3/5, uneven decomposition
    ((12, 12, 12), (3, 4)),
    ((64, 128, 256), (2, 4)),        # batch shape, several tiles per pass
    ((96, 40, 160), (2, 2)),         # radix 3 and 5 lengths
    ((16, 32, 64), (4,)),            # slab
    ((5, 6, 8), (4, 3)),             # zero-size ranks on axis 0
    ((12, 10, 8, 6), (2, 3, 2)),     # 4-D on a 3-D grid
    ((32, 32, 32, 32), (2, 2, 2)),   # 4-D, several tiles per pass
    ((64, 96), (4,)),                # 2-D slab
    ((128,), ()),                    # 1-D, no grid
    ((1, 16, 8), (1, 2)),            # length-1 axis
    ((256, 128, 256), (2, 4)),       # TMA-staged passes (equal blocks, lengths 128/256)
    ((512, 64, 64), (4, 2)),         # TMA-staged passes, a 512-row axis split in two tensor dimensions
    ((96, 160, 64), (2, 2)),         # TMA-staged passes of lengths 96 and 160
    ((60, 120, 240), (2, 4)),        # 2.3.5 lengths: threads with uneven butterfly counts
    ((480, 60, 120), (3, 2)),
    ((192, 320, 48), (2, 2)),        # specialised lengths 48, 192, 320
    ((640, 48, 80), (4, 2)),
    ((768, 4, 384), (2, 2)),
    ((1024, 8, 64), (2, 2)),
    ((8, 2048, 8), (2, 2)),
    ((4096, 4, 8), (4, 2)),          # the longest specialised line, strided
    ((384, 32, 64), (2, 4)),         # TMA-staged 384 (uncut rows viewed as 192 x 2)
    ((1024, 16, 32), (2, 2)),        # TMA-staged 1024 (256 x 4), 8-column tiles
    ((42, 127, 256), (3, 4)),        # the paper's App. A shape: 42 = 2.3.7 and 127 (prime) by Bluestein
    ((7, 11, 26), (2, 3)),           # Bluestein on every axis (26 = 2.13), uneven blocks
    ((2047,), ()),                   # the longest Bluestein line (convolution length 4096)
    ((16, 17, 18, 19), (2, 3, 2)),   # App. B's 4-D shape on a 3-D grid (17, 19 by Bluestein)
    ((32, 32, 64), (48, 2)),         # more parts than rows on both specialised strided axes (empty parts)
]


def _run(p, x_dev, mode, sign, keep=True):
    if sign < 0:
        return p.forward(x_dev, mode=mode, keep_input=keep)
    return p.inverse(x_dev, mode=mode, keep_input=keep)


@pytest.mark.parametrize("shape,grid", CASES)
def test_forward_inverse_vs_oracle(cuda_device, shape, grid):
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    x = inputs.uniform_complex(shape, seed=0).numpy()
    b0 = R.scatter(x, grid, 0)
    want_f = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    want_b = dft.distributed_backward(R.scatter(x, grid, g).astype(np.complex128), shape, grid)
    p = Plan(shape, grid, device=cuda_device)
    outs_f, outs_b = {}, {}
    for mode in ("fused", "unfused", "packed"):
        xin = to_dev(b0, cuda_device)
        y = _run(p, xin, mode, -1)
        torch.cuda.synchronize()
        assert np.array_equal(bits(xin), b0.view(np.uint8)), "input must be kept"
        err = rel_l2(y.cpu().numpy(), want_f)
        assert err <= RTOL_FP32, (mode, err)
        outs_f[mode] = bits(y)
        yin = to_dev(R.scatter(x, grid, g), cuda_device)
        z = _run(p, yin, mode, +1)
        torch.cuda.synchronize()
        err = rel_l2(z.cpu().numpy(), want_b)
        assert err <= RTOL_FP32, (mode, err)
        outs_b[mode] = bits(z)
    assert np.array_equal(outs_f["fused"], outs_f["unfused"])
    assert np.array_equal(outs_f["fused"], outs_f["packed"])
    assert np.array_equal(outs_b["fused"], outs_b["unfused"])
    assert np.array_equal(outs_b["fused"], outs_b["packed"])


@pytest.mark.parametrize("shape,grid", [((256, 128, 256), (2, 4)), ((512, 64, 64), (4, 2)),
                                        ((64, 64, 64), (2, 2)), ((128, 512, 64), (2, 2)),
                                        ((384, 32, 64), (2, 4)), ((1024, 16, 32), (2, 2))])
def test_tma_and_plain_passes_agree(cuda_device, shape, grid):
    """The TMA-staged passes and the plain load/store passes move every line
    the same way.  Where both run the same radices the outputs are
    bit-identical; the plain 512-long strided pass runs 8 x 8 x 8 (16 values
    per thread, twice the resident warps) where the TMA kernel runs 32 x 16,
    so there the two agree to rounding (a misplaced line or element would
    show as an error of order 1e-3 or more)."""
    from paper_1804_09536_gb300.plan import Plan
    x = inputs.normal_complex(shape, seed=7).numpy()
    b0 = R.scatter(x, grid, 0)
    pt = Plan(shape, grid, device=cuda_device)
    pp = Plan(shape, grid, device=cuda_device, tma=False)
    names = [n for n, _ in pt.launch_info(-1)]
    assert any("tma" in n for n in names), names
    assert not any("tma" in n for n, _ in pp.launch_info(-1))
    yt = pt.forward(to_dev(b0, cuda_device))
    yp = pp.forward(to_dev(b0, cuda_device))
    zt = pt.inverse(yt.clone())
    zp = pp.inverse(yp.clone())
    torch.cuda.synchronize()
    assert pt.device_status() == 0
    if 512 not in shape[:-1]:
        assert np.array_equal(bits(yt), bits(yp))
        assert np.array_equal(bits(zt), bits(zp))
    else:
        assert rel_l2(yt.cpu().numpy(), yp.cpu().numpy()) <= 2e-6
        assert rel_l2(zt.cpu().numpy(), zp.cpu().numpy()) <= 2e-6
    want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    assert rel_l2(yt.cpu().numpy(), want) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid,kind", [((512, 64, 100), (2, 3), "c2c"),   # axis 2 split 34/33/33
                                             ((64, 64, 64), (2, 4), "c2c"),    # equal blocks, 16-column ranks
                                             ((96, 96, 96), (2, 4), "c2c"),
                                             ((128, 64, 256), (2, 4), "r2c"),  # 129 complex split 33/32/32/32
                                             ((64, 128, 512), (4, 8), "r2c"),  # the r2c pencil kind, 257 = 33 + 7 x 32
                                             ((256, 32, 256), (8,), "r2c")])   # r2c slab, rows of 129
def test_rank_group_tma_passes(cuda_device, shape, grid, kind):
    """In-place passes along axis 0 of layouts without the equal-block 5-D view
    (uneven splits, odd row lengths, ranks narrower than a tile) run TMA-staged
    tiles over the layout's rank groups: same bits as the plain passes (equal
    radices), and the oracle's result."""
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    pt = Plan(shape, grid, kind=kind, device=cuda_device)
    pp = Plan(shape, grid, kind=kind, device=cuda_device, tma=False)
    names = [n for n, _ in pt.launch_info(-1)] + [n for n, _ in pt.launch_info(+1)]
    assert sum("tma_groups" in n for n in names) == 2, names
    if kind == "r2c":
        x = inputs.normal_real(shape, seed=9).numpy()
        want = dft.distributed_rfft_forward(R.scatter(x, grid, 0).astype(np.float64), shape, grid)
        b0 = R.scatter(x, grid, 0)
    else:
        x = inputs.normal_complex(shape, seed=9).numpy()
        b0 = R.scatter(x, grid, 0)
        want = dft.distributed_forward(b0.astype(np.complex128), shape, grid)
    yt = pt.forward(to_dev(b0, cuda_device))
    yp = pp.forward(to_dev(b0, cuda_device))
    zt = pt.inverse(yt.clone())
    zp = pp.inverse(yp.clone())
    torch.cuda.synchronize()
    assert pt.device_status() == 0
    assert rel_l2(yt.cpu().numpy(), want) <= RTOL_FP32
    if 512 not in shape[:1]:
        assert np.array_equal(bits(yt), bits(yp))
        assert np.array_equal(bits(zt), bits(zp))
    else:
        assert rel_l2(yt.cpu().numpy(), yp.cpu().numpy()) <= 2e-6
        assert rel_l2(zt.cpu().numpy(), zp.cpu().numpy()) <= 2e-6
    assert rel_l2(zt.cpu().numpy(), b0) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid", [((32, 32, 32), (2, 2)), ((40, 48, 60), (3, 4))])
def test_round_trip_and_destroyed_input(cuda_device, shape, grid):
    """App. A: backward(forward(x)) = x; without a workspace the input is scratch."""
    from paper_1804_09536_gb300.plan import Plan
    x = inputs.uniform_complex(shape, seed=3).numpy()
    p = Plan(shape, grid, device=cuda_device)
    b0 = R.scatter(x, grid, 0)
    xin = to_dev(b0, cuda_device)
    y = p.forward(xin, keep_input=False)
    back = p.inverse(y.clone(), keep_input=False)
    torch.cuda.synchronize()
    assert rel_l2(back.cpu().numpy(), b0) <= RTOL_FP32


def test_appendix_a_fill_round_trip(cuda_device):
    """App. A's fill arrayA[j] = j + j i on every local array (scaled to O(1) for FP32),
    forward then backward on a 2-D grid; FP32 tolerance instead of the paper's FP64 1e-8."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (40, 120, 256), (2, 3)
    p = Plan(shape, grid, device=cuda_device)
    buf = np.empty(p.stage_elems(0), np.complex64)
    for r in range(p.num_ranks):
        st, sz, off = p.local_box(0, r)
        n = math.prod(sz)
        j = np.arange(n, dtype=np.float64) / n
        buf[off:off + n] = (j + 1j * j).astype(np.complex64)
    y = p.forward(to_dev(buf, cuda_device))
    back = p.inverse(y).cpu().numpy()
    assert np.max(np.abs(back - buf)) < 1e-6


@pytest.mark.parametrize("shape,grid", [((16, 24, 32), (2, 2)), ((16, 32, 20), (4,))])
def test_partial_transforms(cuda_device, shape, grid):
    """F_axis on every rank's local array (the appendix's sequential routine)."""
    from paper_1804_09536_gb300.plan import Plan
    p = Plan(shape, grid, device=cuda_device)
    x = inputs.normal_complex(shape, seed=5).numpy()
    g = len(grid)
    for s in range(g + 1):
        b = R.scatter(x, grid, s)
        layout_axes = [a for a in range(len(shape)) if all(
            p.local_box(s, r)[1][a] == shape[a] for r in range(p.num_ranks))]
        for axis in layout_axes:
            for sign in (-1, 1):
                t = to_dev(b, cuda_device)
                p.partial(s, axis, sign, t)
                want = dft._transform_ranks(b.astype(np.complex128), shape, grid, s, axis, sign)
                assert rel_l2(t.cpu().numpy(), want) <= RTOL_FP32, (s, axis, sign)


def test_norm_backward_flag(cuda_device):
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (16, 16, 16), (2, 2)
    x = inputs.uniform_complex(shape, seed=4).numpy()
    p = Plan(shape, grid, norm="backward", device=cuda_device)
    y = p.forward(to_dev(R.scatter(x, grid, 0), cuda_device)).cpu().numpy()
    want = dft.distributed_forward(R.scatter(x, grid, 0).astype(np.complex128), shape, grid) * 4096
    assert rel_l2(y, want) <= RTOL_FP32


def test_norm_backward_r2c_window_plan(cuda_device):
    """TFFT_NORM_BACKWARD on a real-to-complex plan with a column window: the
    unscaled forward, and the 1/N of the inverse on its complex-to-real pass
    after the two column ranges of the gathering pass."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (16, 512, 120), (2, 4)
    p = Plan(shape, grid, kind="r2c", norm="backward", device=cuda_device)
    assert sum("tma_window" in n for n, _ in p.launch_info(+1)) == 1
    x = inputs.normal_real(shape, seed=6).numpy()
    b0 = R.scatter(x, grid, 0)
    y = p.forward(to_dev(b0, cuda_device))
    want = dft.distributed_rfft_forward(b0.astype(np.float64), shape, grid) * math.prod(shape)
    assert rel_l2(y.cpu().numpy(), want) <= RTOL_FP32
    z = p.inverse(y.clone())
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert rel_l2(z.cpu().numpy(), b0) <= RTOL_FP32


@pytest.mark.slow
def test_full_size_512_pencil_sampled(cuda_device):
    """The bench workload (512^3, 4 x 8, launch configuration of bench.py): sampled
    outputs against the oracle's definition, plus round trip and Parseval."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (512, 512, 512), (4, 8)
    x = inputs.normal_complex(shape, seed=0)
    p = Plan(shape, grid, device=cuda_device)
    b0 = p.scatter(x.to(cuda_device), 0)
    y = p.forward(b0)
    yg = p.gather(y, 2).cpu().numpy()
    rng = np.random.default_rng(0)
    ks = [(0, 0, 0), (511, 511, 511), (1, 2, 3)] + [tuple(int(v) for v in rng.integers(0, 512, 3))
                                                   for _ in range(5)]
    want = dft.forward_at(x.numpy(), ks)
    got = np.array([yg[k] for k in ks])
    rms = float(np.sqrt(np.mean(np.abs(yg.astype(np.complex128)) ** 2)))
    assert np.max(np.abs(got - want)) <= 1e-4 * rms
    # Parseval (paper normalisation) and round trip hold at any size
    n = x.numel()
    e_in = float(torch.sum(torch.abs(x.to(torch.complex128)) ** 2)) / n
    e_out = float(np.sum(np.abs(yg.astype(np.complex128)) ** 2))
    assert abs(e_out - e_in) <= 1e-5 * e_in
    back = p.inverse(y)
    diff = torch.linalg.vector_norm((back - b0).to(torch.complex128)) / torch.linalg.vector_norm(b0.to(torch.complex128))
    assert float(diff) <= RTOL_FP32


@pytest.mark.slow
def test_full_size_128_4d_sampled(cuda_device):
    """The 4-D workload of bench.py (128^4 on a 4 x 4 x 2 grid): sampled outputs
    against the oracle's definition, Parseval and round trip."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (128, 128, 128, 128), (4, 4, 2)
    x = inputs.normal_complex(shape, seed=0)
    p = Plan(shape, grid, device=cuda_device)
    b0 = p.scatter(x.to(cuda_device), 0)
    y = p.forward(b0)
    yg = p.gather(y, p.g).cpu().numpy()
    rng = np.random.default_rng(1)
    ks = [(0, 0, 0, 0), (127, 127, 127, 127), (1, 2, 3, 4)] + [
        tuple(int(v) for v in rng.integers(0, 128, 4)) for _ in range(3)]
    want = dft.forward_at(x.numpy(), ks, chunk=8)
    got = np.array([yg[k] for k in ks])
    rms = float(np.sqrt(np.mean(np.abs(yg.astype(np.complex128)) ** 2)))
    assert np.max(np.abs(got - want)) <= 1e-4 * rms
    n = x.numel()
    e_in = float(torch.sum(torch.abs(x.to(torch.complex128)) ** 2)) / n
    e_out = float(np.sum(np.abs(yg.astype(np.complex128)) ** 2))
    assert abs(e_out - e_in) <= 1e-5 * e_in
    back = p.inverse(y)
    diff = torch.linalg.vector_norm((back - b0).to(torch.complex128)) / torch.linalg.vector_norm(b0.to(torch.complex128))
    assert float(diff) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid", [((64, 128, 512), (4, 8)),    # 257 = 33 + 7 x 32: window over ranks 1..7, lead 1
                                         ((128, 64, 256), (2, 4)),    # 129 = 33 + 3 x 32
                                         ((32, 512, 512), (4, 8)),    # the pencil workload's axis-1 length
                                         ((16, 512, 120), (2, 4)),    # 61 = 16 + 3 x 15: window over rank 0, no lead
                                         ((8, 160, 120), (2, 4))])    # a 5-smooth length, window over rank 0
def test_r2c_column_window_passes(cuda_device, shape, grid):
    """Real-to-complex plans whose stage-0 rows are odd: the fused path keeps its
    complex stage-0 buffer with padded rows and runs the gathering pass along
    axis 1 TMA-staged over the column window of the ranks of one even width,
    the other columns with the plain kernel.  Forward and inverse against the
    oracle and against the plan without TMA passes (same bits where the two
    kernels use the same radices)."""
    from paper_1804_09536_gb300.plan import Plan
    pt = Plan(shape, grid, kind="r2c", device=cuda_device)
    pp = Plan(shape, grid, kind="r2c", device=cuda_device, tma=False)
    for sign in (-1, +1):
        names = [n for n, _ in pt.launch_info(sign)]
        assert sum("tma_window" in n for n in names) == 1, names
    assert pt.workspace_bytes("fused") > pp.workspace_bytes("fused")
    x = inputs.normal_real(shape, seed=21).numpy()
    b0 = R.scatter(x, grid, 0)
    want = dft.distributed_rfft_forward(b0.astype(np.float64), shape, grid)
    xin = to_dev(b0, cuda_device)
    yt = pt.forward(xin)
    yp = pp.forward(to_dev(b0, cuda_device))
    zt = pt.inverse(yt.clone())
    zp = pp.inverse(yp.clone())
    torch.cuda.synchronize()
    assert pt.device_status() == 0
    assert np.array_equal(bits(xin), b0.view(np.uint8)), "r2c keeps its input"
    assert rel_l2(yt.cpu().numpy(), want) <= RTOL_FP32
    want_b = dft.distributed_irfft_backward(want, shape, grid)
    assert rel_l2(zt.cpu().numpy(), want_b) <= RTOL_FP32
    if shape[1] != 512:
        assert np.array_equal(bits(yt), bits(yp))
        assert np.array_equal(bits(zt), bits(zp))
    else:
        assert rel_l2(yt.cpu().numpy(), yp.cpu().numpy()) <= 2e-6
        assert rel_l2(zt.cpu().numpy(), zp.cpu().numpy()) <= 2e-6
    # unfused and packed paths (plain layouts) give the same transform
    yu = pt.forward(to_dev(b0, cuda_device), mode="unfused")
    torch.cuda.synchronize()
    assert rel_l2(yu.cpu().numpy(), want) <= RTOL_FP32


def test_r2c_window_plan_replays_from_a_cuda_graph(cuda_device):
    """The column-window passes (tensor maps encoded at launch, two launches on
    one pair of buffers) captured in a CUDA graph and replayed: the same bits
    as the eager forward and inverse."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (64, 128, 512), (4, 8)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    x = to_dev(R.scatter(inputs.normal_real(shape, seed=5).numpy(), grid, 0), cuda_device)
    y_ref = p.forward(x)
    z_ref = p.inverse(y_ref.clone())
    y = p.empty_stage(p.g)
    yi = p.empty_stage(p.g)
    z = p.empty_stage(0, real=True)
    work = p.workspace("fused")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.execute(-1, x, y, "fused", work)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.execute(-1, x, y, "fused", work)
        yi.copy_(y)
        p.execute(1, yi, z, "fused", work)
    for t in (y, z):
        t.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert torch.equal(y, y_ref)
    assert torch.equal(z, z_ref)


R2C_CASES = [
    ((8, 12, 480), (2, 2)),          # half-length 240 (2.3.5)
    ((4, 8, 2048), (2, 2)),          # half-length 1024
    ((8, 8, 768), (4,)),             # half-length 384
    ((32, 64, 256), (8,)),           # the r2c slab workload's innermost length, 8 ranks
    ((16, 32, 64), (2, 2)),          # r2c on a pencil grid
    ((12, 10, 128), (3,)),           # uneven slab
    ((24, 64), (4,)),                # 2-D
    ((64,), ()),                     # 1-D real line
]


@pytest.mark.parametrize("shape,grid", R2C_CASES)
def test_r2c_c2r_vs_oracle(cuda_device, shape, grid):
    """Footnote to Eq. multifft: real input, Hermitian half on the last axis;
    fused, unfused and packed paths agree bit for bit."""
    from paper_1804_09536_gb300.plan import Plan
    g = len(grid)
    x = inputs.normal_real(shape, seed=0).numpy()
    cshape = shape[:-1] + (shape[-1] // 2 + 1,)
    b0 = R.scatter(x, grid, 0)
    want = dft.distributed_rfft_forward(b0.astype(np.float64), shape, grid)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    outs, backs = {}, {}
    for mode in ("fused", "unfused", "packed"):
        xin = to_dev(b0, cuda_device)
        y = p.forward(xin, mode=mode)
        torch.cuda.synchronize()
        assert np.array_equal(bits(xin), b0.view(np.uint8)), "r2c keeps its input"
        assert rel_l2(y.cpu().numpy(), want) <= RTOL_FP32, mode
        outs[mode] = bits(y)
        z = p.inverse(y.clone(), mode=mode)
        torch.cuda.synchronize()
        back = z.cpu().numpy()
        want_b = dft.distributed_irfft_backward(want, shape, grid)
        assert rel_l2(back, want_b) <= RTOL_FP32, mode
        assert rel_l2(back, b0) <= RTOL_FP32
        backs[mode] = bits(z)
    for m in ("unfused", "packed"):
        assert np.array_equal(outs["fused"], outs[m])
        assert np.array_equal(backs["fused"], backs[m])
    # the gathered spectrum is the oracle's r2c of the global array
    yg = p.gather(torch.from_numpy(np.frombuffer(outs["fused"].tobytes(), np.complex64).copy()), g)
    assert rel_l2(yg.numpy(), dft.rfftn_forward(x.astype(np.float64))) <= RTOL_FP32


def test_c2r_ignores_dc_and_nyquist_imaginary_parts(cuda_device):
    """c2r reading: Im of k = 0 and k = N/2 on the last axis do not contribute."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (8, 16, 64), (2,)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    x = inputs.normal_real(shape, seed=2).numpy()
    y = p.forward(to_dev(R.scatter(x, grid, 0), cuda_device))
    yg = p.gather(y, 1).cpu().numpy()
    pert = yg.copy()
    pert[..., 0] += 0.5j
    pert[..., -1] -= 0.25j
    z = p.inverse(to_dev(R.scatter(pert, grid, 1), cuda_device))
    want = dft.irfftn_backward(pert.astype(np.complex128), shape[-1])
    assert rel_l2(p.gather(z, 0, real=True).cpu().numpy(), want) <= RTOL_FP32


@pytest.mark.slow
def test_full_size_r2c_256_slab_sampled(cuda_device):
    """The r2c slab workload of bench.py (256^3 real on 8 ranks): sampled outputs of the
    Hermitian half against the oracle's definition (the c2c transform of the real input),
    the real Parseval relation and the c2r round trip."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (256, 256, 256), (8,)
    x = inputs.normal_real(shape, seed=0)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    b0 = p.scatter(x.to(cuda_device), 0, real=True)
    y = p.forward(b0)
    yg = p.gather(y, 1).cpu().numpy()
    assert yg.shape == (256, 256, 129)
    rng = np.random.default_rng(2)
    ks = [(0, 0, 0), (255, 255, 128), (1, 2, 3), (7, 0, 128)] + [
        (int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(rng.integers(0, 129))) for _ in range(4)]
    want = dft.forward_at(x.numpy().astype(np.complex64), ks)
    got = np.array([yg[k] for k in ks])
    rms = float(np.sqrt(np.mean(np.abs(yg.astype(np.complex128)) ** 2)))
    assert np.max(np.abs(got - want)) <= 1e-4 * rms
    # Parseval over the full spectrum: columns 1..127 stand for two conjugate columns
    n = x.numel()
    e_in = float(torch.sum(x.to(torch.float64) ** 2)) / n
    p2 = np.abs(yg.astype(np.complex128)) ** 2
    e_out = float(p2[..., 0].sum() + p2[..., 128].sum() + 2 * p2[..., 1:128].sum())
    assert abs(e_out - e_in) <= 1e-5 * e_in
    back = p.inverse(y.clone())
    assert float(torch.linalg.vector_norm((back - b0).double()) / torch.linalg.vector_norm(b0.double())) <= RTOL_FP32


@pytest.mark.slow
def test_full_size_r2c_512_pencil_sampled(cuda_device):
    """r2c on a pencil grid at the size bench.py measures (512^3 real on 4 x 8): sampled
    outputs of the Hermitian half against the oracle's definition and the c2r round trip."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (512, 512, 512), (4, 8)
    x = inputs.normal_real(shape, seed=0)
    p = Plan(shape, grid, kind="r2c", device=cuda_device)
    b0 = p.scatter(x.to(cuda_device), 0, real=True)
    y = p.forward(b0)
    yg = p.gather(y, 2).cpu().numpy()
    assert yg.shape == (512, 512, 257)
    rng = np.random.default_rng(4)
    ks = [(0, 0, 0), (511, 511, 256), (3, 2, 1)] + [
        (int(rng.integers(0, 512)), int(rng.integers(0, 512)), int(rng.integers(0, 257))) for _ in range(3)]
    want = dft.forward_at(x.numpy().astype(np.complex64), ks, chunk=16)
    got = np.array([yg[k] for k in ks])
    rms = float(np.sqrt(np.mean(np.abs(yg.astype(np.complex128)) ** 2)))
    assert np.max(np.abs(got - want)) <= 1e-4 * rms
    back = p.inverse(y.clone())
    assert float(torch.linalg.vector_norm((back - b0).double()) / torch.linalg.vector_norm(b0.double())) <= RTOL_FP32


@pytest.mark.parametrize("shape,grid,kind", [((32, 32, 32), (2, 2), "c2c"),
                                             ((64, 128, 512), (4, 8), "r2c"),      # column window
                                             ((512, 64, 100), (2, 3), "c2c")])     # rank groups, uneven
def test_repeated_execute_replays_the_same_launches(cuda_device, shape, grid, kind):
    """From the second identical call on, tfft_execute launches a CUDA graph of
    its launches: every call's result equals the plan without graphs bit for
    bit, also after the buffers or the wait limit change (new graphs), and
    more distinct calls than the cache holds keep giving the same bits."""
    from paper_1804_09536_gb300.plan import Plan
    pg = Plan(shape, grid, kind=kind, device=cuda_device)
    pn = Plan(shape, grid, kind=kind, device=cuda_device, graphs=False)
    if kind == "r2c":
        x = to_dev(R.scatter(inputs.normal_real(shape, seed=8).numpy(), grid, 0), cuda_device)
    else:
        x = to_dev(R.scatter(inputs.uniform_complex(shape, seed=8).numpy(), grid, 0), cuda_device)
    ref = pn.forward(x)
    refb = pn.inverse(ref.clone())
    ys = [pg.empty_stage(pg.g) for _ in range(10)]
    zs = [pg.empty_stage(0, real=kind == "r2c") for _ in range(2)]
    w = pg.workspace("fused")
    for rep in range(3):
        for y in ys:                       # ten distinct keys: more than the cache keeps
            y.fill_(float("nan"))
            pg.execute(-1, x, y, "fused", w)
        for z in zs:
            yi = ys[0].clone() if kind == "r2c" else ys[0]
            pg.execute(+1, yi, z, "fused", w)
        torch.cuda.synchronize()
        for y in ys:
            assert torch.equal(y, ref), rep
        for z in zs:
            assert torch.equal(z, refb), rep
    pg.set_wait_limit(1 << 20)             # a new key: captured again
    for _ in range(3):
        pg.execute(-1, x, ys[1], "fused", w)
    pg.set_wait_limit(0)
    torch.cuda.synchronize()
    assert pg.device_status() == 0
    assert torch.equal(ys[1], ref)


def test_execute_from_several_threads(cuda_device):
    """One plan, four host threads, each with its own stream and output buffer,
    calling tfft_execute repeatedly (the graph cache is shared and locked):
    every output equals the single-threaded transform."""
    import threading
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (64, 64, 128), (2, 4)
    p = Plan(shape, grid, device=cuda_device)
    x = to_dev(R.scatter(inputs.uniform_complex(shape, seed=12).numpy(), grid, 0), cuda_device)
    ref = p.forward(x)
    torch.cuda.synchronize()
    outs = [[p.empty_stage(p.g) for _ in range(2)] for _ in range(4)]
    works = [p.workspace("fused").clone() for _ in range(4)]
    streams = [torch.cuda.Stream() for _ in range(4)]
    errors = []

    def run(t):
        try:
            with torch.cuda.device(cuda_device):
                for it in range(6):
                    p.execute(-1, x, outs[t][it % 2], "fused", works[t], stream=streams[t])
                streams[t].synchronize()
        except Exception as e:  # reported below
            errors.append(e)
    threads = [threading.Thread(target=run, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    assert not errors, errors
    assert p.device_status() == 0
    for t in range(4):
        for y in outs[t]:
            assert torch.equal(y, ref), t
