"""GPU: the batched persistent executor (many transforms, one launch) (needs a GPU)."""
import numpy as np
import pytest
import torch

from oracle import dft, redistribute as R
from paper_1804_09536_gb300 import inputs
from gpu_util import RTOL_FP32, bits, rel_l2, to_dev

pytestmark = pytest.mark.gpu

SMALL = [((64, 64, 32), (1, 2)), ((64, 96, 64), (2, 2)), ((96, 64, 128), (2, 4)),
         ((128, 64, 32), (2, 2)), ((64, 160, 96), (1, 2)), ((160, 64, 64), (2, 4)),
         ((64, 128, 256), (2, 4)), ((256, 64, 64), (2, 2))]


def _plans(problems, dev):
    from paper_1804_09536_gb300.plan import Plan
    return [Plan(s, g, device=dev) for s, g in problems]


@pytest.mark.parametrize("sign", [-1, 1])
def test_batch_vs_oracle_and_standalone(cuda_device, sign):
    from paper_1804_09536_gb300.plan import Batch
    plans = _plans(SMALL, cuda_device)
    xs = []
    for k, (shape, grid) in enumerate(SMALL):
        x = inputs.uniform_complex(shape, seed=100 + k).numpy()
        xs.append(x)
    b = Batch(plans, sign=sign)
    for k, (shape, grid) in enumerate(SMALL):
        st = 0 if sign < 0 else len(grid)
        b.ins[k].copy_(to_dev(R.scatter(xs[k], grid, st), cuda_device))
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for k, (shape, grid) in enumerate(SMALL):
        g = len(grid)
        p = plans[k]
        if sign < 0:
            want = dft.distributed_forward(R.scatter(xs[k], grid, 0).astype(np.complex128), shape, grid)
            solo = p.forward(b.ins[k])
        else:
            want = dft.distributed_backward(R.scatter(xs[k], grid, g).astype(np.complex128), shape, grid)
            solo = p.inverse(b.ins[k])
        got = b.outs[k].cpu().numpy()
        assert rel_l2(got, want) <= RTOL_FP32, (k, shape, grid)
        # default executor tiles run the standalone passes' radices: identical bits
        assert np.array_equal(bits(b.outs[k]), bits(solo)), (k, shape, grid)
        torch.cuda.synchronize()


def test_batch_48_graph_and_autotune(cuda_device):
    """The 48-transform workload: one persistent launch per direction, captured in a
    CUDA graph and replayed; autotuned tiles stay within the FP32 tolerance."""
    from paper_1804_09536_gb300.plan import Batch
    problems = inputs.batch_problems(48, seed=0)
    plans = _plans(problems, cuda_device)
    b = Batch(plans, sign=-1)
    for k, (shape, grid) in enumerate(problems):
        b.ins[k].copy_(plans[k].scatter(inputs.uniform_complex(shape, seed=k).to(cuda_device), 0))
    g = b.graph()
    for o in b.outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    refs = [plans[k].forward(b.ins[k]) for k in range(len(problems))]
    torch.cuda.synchronize()
    for k in range(len(problems)):
        assert torch.equal(b.outs[k], refs[k]), k
    items, segs = b.num_items()
    assert segs == 3 * len(problems) and items > 0
    b.autotune(reps=2)
    b.execute()
    torch.cuda.synchronize()
    for k in range(len(problems)):
        assert rel_l2(b.outs[k].cpu().numpy(), refs[k].cpu().numpy()) <= RTOL_FP32, k


def test_batch_wait_expiry_reports_status(cuda_device):
    """A forced, tiny wait limit makes a pass give up on its predecessor: the
    launch stops and the status word says so (no fault, the context stays usable)."""
    from paper_1804_09536_gb300.plan import Batch
    plans = _plans(SMALL[:3], cuda_device)
    b = Batch(plans, sign=-1)
    b.set_wait_limit(1)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status(reset=True) == 1
    b.set_wait_limit(0)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    ref = plans[0].forward(b.ins[0])
    assert torch.equal(b.outs[0], ref)


def test_tma_wait_expiry_reports_status(cuda_device):
    """Same for the TMA passes: one poll per copy wait cannot see the copy land."""
    from paper_1804_09536_gb300.plan import Plan
    shape, grid = (256, 128, 256), (2, 4)
    p = Plan(shape, grid, device=cuda_device)
    assert any("tma" in n for n, _ in p.launch_info(-1))
    x = p.scatter(inputs.uniform_complex(shape, seed=1).to(cuda_device), 0)
    p.set_wait_limit(1)
    p.forward(x)
    torch.cuda.synchronize()
    assert p.device_status(reset=True) == 1
    p.set_wait_limit(0)
    y = p.forward(x)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    pp = Plan(shape, grid, device=cuda_device, tma=False)
    assert torch.equal(y, pp.forward(x))


def test_batch_tma_tiles_match_standalone(cuda_device):
    """The TMA-staged strided tiles of the executor (variants 15-18: lengths 64, 128, 256, 96),
    chosen by hand: the same bits as the standalone passes; and their bounded copy waits
    report an expiry through the status word."""
    from paper_1804_09536_gb300.plan import Batch
    from paper_1804_09536_gb300._lib import TfftError
    plans = _plans(SMALL, cuda_device)
    b = Batch(plans, sign=-1)
    for k, (shape, grid) in enumerate(SMALL):
        b.ins[k].copy_(plans[k].scatter(inputs.uniform_complex(shape, seed=200 + k).to(cuda_device), 0))
    chosen = 0
    for L, v in ((64, 15), (128, 16), (256, 17), (96, 18)):
        try:
            b.set_variant(1, L, v)
            chosen += 1
        except TfftError:
            pass
    assert chosen == 4
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    refs = [p.forward(b.ins[k]) for k, p in enumerate(plans)]
    torch.cuda.synchronize()
    for k in range(len(SMALL)):
        assert torch.equal(b.outs[k], refs[k]), (k, SMALL[k])
    b.set_wait_limit(1)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status(reset=True) == 1
    b.set_wait_limit(0)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for k in range(len(SMALL)):
        assert torch.equal(b.outs[k], refs[k]), k


@pytest.mark.parametrize("nstreams", [1, 3, 8])
def test_stream_executor_matches_standalone(cuda_device, nstreams):
    """The stream executor runs each transform's own pass kernels on forked
    streams: the same bits as the plans' standalone forwards, eagerly and
    replayed from a CUDA graph (which captures the fork and the join)."""
    from paper_1804_09536_gb300.plan import Batch
    plans = _plans(SMALL, cuda_device)
    b = Batch(plans, sign=-1)
    b.set_executor("streams", nstreams)
    assert b.executor == ("streams", min(nstreams, len(SMALL)))
    for k, (shape, grid) in enumerate(SMALL):
        b.ins[k].copy_(to_dev(R.scatter(inputs.uniform_complex(shape, seed=200 + k).numpy(), grid, 0),
                              cuda_device))
    refs = [plans[k].forward(b.ins[k]) for k in range(len(SMALL))]
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for k in range(len(SMALL)):
        assert torch.equal(b.outs[k], refs[k]), k
    g = b.graph()
    for o in b.outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for k in range(len(SMALL)):
        assert torch.equal(b.outs[k], refs[k]), k


def test_stream_executor_reports_plan_status(cuda_device):
    """A copy wait that expires inside a transform run by the stream executor
    lands in its plan's status word, which the batch status ORs in."""
    from paper_1804_09536_gb300.plan import Batch
    problems = [((64, 64, 64), (2, 2)), ((128, 128, 128), (2, 4))]
    plans = _plans(problems, cuda_device)
    b = Batch(plans, sign=-1)
    b.set_executor("streams", 2)
    for k, (shape, grid) in enumerate(problems):
        b.ins[k].copy_(plans[k].scatter(inputs.uniform_complex(shape, seed=k).to(cuda_device), 0))
    names = [n for n, _ in plans[1].launch_info(-1)]
    assert any("tma" in n for n in names), names
    plans[1].set_wait_limit(1)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status(reset=True) == 1
    assert plans[1].device_status() == 0
    plans[1].set_wait_limit(0)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0


def test_autotune_picks_an_executor(cuda_device):
    """Autotuning times the persistent kernel against the stream executor and
    keeps the faster; either way the results stay the oracle's."""
    from paper_1804_09536_gb300.plan import Batch
    plans = _plans(SMALL, cuda_device)
    b = Batch(plans, sign=-1)
    xs = [inputs.uniform_complex(shape, seed=300 + k).numpy() for k, (shape, _) in enumerate(SMALL)]
    for k, (shape, grid) in enumerate(SMALL):
        b.ins[k].copy_(to_dev(R.scatter(xs[k], grid, 0), cuda_device))
    keep = [t.clone() for t in b.ins]
    b.autotune(reps=2)
    kind, n = b.executor
    assert (kind == "persistent" and n == 0) or (kind == "streams" and 1 <= n <= 8)
    for t, k in zip(b.ins, keep):
        t.copy_(k)
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for k, (shape, grid) in enumerate(SMALL):
        want = dft.distributed_forward(R.scatter(xs[k], grid, 0).astype(np.complex128), shape, grid)
        assert rel_l2(b.outs[k].cpu().numpy(), want) <= RTOL_FP32, k


@pytest.mark.parametrize("sign", [-1, 1])
def test_stream_executor_without_workspaces(cuda_device, sign):
    """Inputs as scratch (no workspaces, keep_input=False), both directions, one
    stream per transform and more streams than transforms: the stream executor
    still matches the plans' standalone transforms bit for bit."""
    from paper_1804_09536_gb300.plan import Batch
    probs = SMALL[:3]
    plans = _plans(probs, cuda_device)
    b = Batch(plans, sign=sign, keep_input=False)
    b.set_executor("streams", 16)
    assert b.executor == ("streams", 3)
    xs = []
    for k, (shape, grid) in enumerate(probs):
        st = 0 if sign < 0 else len(grid)
        xs.append(to_dev(R.scatter(inputs.uniform_complex(shape, seed=400 + k).numpy(), grid, st), cuda_device))
        b.ins[k].copy_(xs[k])
    refs = [(p.forward(x) if sign < 0 else p.inverse(x)) for p, x in zip(plans, xs)]
    b.execute()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for k in range(len(probs)):
        assert torch.equal(b.outs[k], refs[k]), k


def test_forward_batch_feeds_inverse_batch(cuda_device):
    """A backward batch built over the forward batch's output buffers (the
    forward + inverse step of the batch workload): both replay from their own
    graphs, each equals the plans' own transforms bit for bit, and the round
    trip returns the input (paper normalisation: 1/N on the forward)."""
    from paper_1804_09536_gb300.plan import Batch
    plans = _plans(SMALL, cuda_device)
    fwd = Batch(plans, sign=-1)
    for k, (shape, grid) in enumerate(SMALL):
        fwd.ins[k].copy_(to_dev(R.scatter(inputs.uniform_complex(shape, seed=600 + k).numpy(), grid, 0), cuda_device))
    inv = Batch(plans, sign=+1, ins=fwd.outs)
    assert all(a.data_ptr() == b.data_ptr() for a, b in zip(inv.ins, fwd.outs))
    gf, gi = fwd.graph(), inv.graph()
    for _ in range(2):
        gf.replay()
        gi.replay()
    torch.cuda.synchronize()
    assert fwd.device_status() == 0 and inv.device_status() == 0
    for k, p in enumerate(plans):
        y = p.forward(fwd.ins[k])
        assert torch.equal(fwd.outs[k], y), k
        assert torch.equal(inv.outs[k], p.inverse(y)), k
        err = rel_l2(inv.outs[k].cpu().numpy(), fwd.ins[k].cpu().numpy())
        assert err <= RTOL_FP32, (k, err)
