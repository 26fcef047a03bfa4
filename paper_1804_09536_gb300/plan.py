"""Python front end of the C ABI: a plan over a global shape and a virtual grid.

PyTorch supplies device memory and streams only; every step of the transform
runs in the library's CUDA kernels.  All buffers are caller-owned torch
tensors passed as raw pointers.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import call


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


_MODES = {"fused": _lib.TFFT_MODE_FUSED, "unfused": _lib.TFFT_MODE_UNFUSED,
          "packed": _lib.TFFT_MODE_PACKED}


class Plan:
    """Transpose-algorithm FFT plan (slab: len(grid) == 1, pencil: 2, ...).

    Stage buffers are 1-D complex64 tensors holding every virtual rank's local
    array, concatenated in rank order.  ``forward`` maps stage 0 to stage g,
    ``inverse`` stage g to stage 0; ``redistribute(v, w)`` is the exchange of
    Alg. 3 between the stages aligned in v and in w.  ``graphs=False`` stops
    ``execute`` from replaying the launches of repeated identical calls from a
    CUDA graph (TFFT_NO_GRAPH).
    """

    def __init__(self, shape, grid, kind: str = "c2c", norm: str = "forward", device=None,
                 bind: bool = True, tma: bool = True, precision: str = "fp32", graphs: bool = True):
        self.shape = tuple(int(n) for n in shape)
        self.grid = tuple(int(m) for m in grid)
        self.kind = kind
        kind_id = {"c2c": _lib.TFFT_C2C, "r2c": _lib.TFFT_R2C}[kind]
        flags = {"forward": _lib.TFFT_NORM_FORWARD, "backward": _lib.TFFT_NORM_BACKWARD}[norm]
        if not tma:
            flags |= _lib.TFFT_NO_TMA
        if not graphs:
            flags |= _lib.TFFT_NO_GRAPH
        h = ctypes.c_void_p()
        shp = (ctypes.c_int64 * len(self.shape))(*self.shape)
        grd = (ctypes.c_int * max(1, len(self.grid)))(*(self.grid or (1,)))
        prec = {"fp32": _lib.TFFT_FP32, "bf16x3": _lib.TFFT_TC_BF16X3, "fp16x3": _lib.TFFT_TC_FP16X3}[precision]
        self.precision = precision
        call("tfft_plan_create", ctypes.byref(h), len(self.shape), shp, len(self.grid), grd,
             kind_id, prec, flags)
        self._h = h
        self.d = len(self.shape)
        self.g = len(self.grid)
        self.device = torch.device(device) if device is not None else None
        self.state = None
        self._work = {}
        if bind:
            self.bind(device)

    # ------------------------------------------------------------ lifetime
    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.load().tfft_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def bind(self, device=None):
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        nbytes = ctypes.c_size_t()
        call("tfft_plan_state_bytes", self._h, ctypes.byref(nbytes))
        self.state = torch.empty(max(256, nbytes.value), dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            call("tfft_plan_bind", self._h, _ptr(self.state), self.state.numel(), _stream_ptr())
        return self

    # ------------------------------------------------------------ queries
    @property
    def num_stages(self) -> int:
        n = ctypes.c_int()
        call("tfft_plan_num_stages", self._h, ctypes.byref(n))
        return n.value

    @property
    def num_ranks(self) -> int:
        n = ctypes.c_int()
        call("tfft_plan_num_ranks", self._h, ctypes.byref(n))
        return n.value

    def stage_axis(self, stage: int) -> int:
        n = ctypes.c_int()
        call("tfft_plan_stage_axis", self._h, stage, ctypes.byref(n))
        return n.value

    def stage_elems(self, stage: int, real: bool = False) -> int:
        n = ctypes.c_int64()
        call("tfft_plan_stage_elems", self._h, stage, int(real), ctypes.byref(n))
        return n.value

    def local_box(self, stage: int, rank: int, real: bool = False):
        st = (ctypes.c_int64 * self.d)()
        sz = (ctypes.c_int64 * self.d)()
        off = ctypes.c_int64()
        call("tfft_plan_local_box", self._h, stage, int(real), rank, st, sz, ctypes.byref(off))
        return tuple(st), tuple(sz), off.value

    def workspace_bytes(self, mode: str = "fused", keep_input: bool = True) -> int:
        n = ctypes.c_size_t()
        call("tfft_plan_workspace_bytes", self._h, _MODES[mode], int(keep_input), ctypes.byref(n))
        return n.value

    def num_launches(self, sign: int, mode: str = "fused") -> int:
        n = ctypes.c_int()
        call("tfft_plan_num_launches", self._h, sign, _MODES[mode], ctypes.byref(n))
        return n.value

    # ------------------------------------------------------------ buffers
    def empty_stage(self, stage: int, real: bool = False) -> torch.Tensor:
        dt = torch.float32 if real else torch.complex64
        return torch.empty(self.stage_elems(stage, real), dtype=dt, device=self.device)

    def workspace(self, mode: str = "fused", keep_input: bool = True) -> torch.Tensor | None:
        nb = self.workspace_bytes(mode, keep_input)
        if nb == 0:
            return None
        key = (mode, keep_input)
        w = self._work.get(key)
        if w is None or w.numel() < nb:
            w = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self._work[key] = w
        return w

    # ------------------------------------------------------------ transforms
    def execute(self, sign: int, x: torch.Tensor, out: torch.Tensor, mode: str = "fused",
                work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        wp = _ptr(work) if work is not None else ctypes.c_void_p(0)
        wb = work.numel() * work.element_size() if work is not None else 0
        call("tfft_execute", self._h, sign, _MODES[mode], _ptr(x), _ptr(out), wp, wb, _stream_ptr(stream))
        return out

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, mode: str = "fused",
                keep_input: bool = True, stream=None) -> torch.Tensor:
        if out is None:
            out = self.empty_stage(self.g)
        work = self.workspace(mode, keep_input)
        return self.execute(_lib.TFFT_FORWARD, x, out, mode, work, stream)

    def inverse(self, y: torch.Tensor, out: torch.Tensor | None = None, mode: str = "fused",
                keep_input: bool = True, stream=None) -> torch.Tensor:
        if out is None:
            out = self.empty_stage(0, real=(self.kind == "r2c"))
        work = self.workspace(mode, keep_input)
        return self.execute(_lib.TFFT_BACKWARD, y, out, mode, work, stream)

    def adjoint(self, y: torch.Tensor, out: torch.Tensor | None = None, mode: str = "fused",
                keep_input: bool = True, stream=None, coef: torch.Tensor | None = None) -> torch.Tensor:
        """F^H y (stage g -> stage 0): the backward passes with 1/N (complex-to-complex);
        times coef[()] (float64 0-d device tensor, read on the device) when given."""
        if out is None:
            out = self.empty_stage(0)
        work = self.workspace(mode, keep_input)
        wp = _ptr(work) if work is not None else ctypes.c_void_p(0)
        wb = work.numel() * work.element_size() if work is not None else 0
        cp = _ptr(coef) if coef is not None else ctypes.c_void_p(0)
        call("tfft_adjoint", self._h, _MODES[mode], _ptr(y), _ptr(out), wp, wb, cp, _stream_ptr(stream))
        return out

    def host_space_bytes(self) -> int:
        """Device bytes tfft_execute_host needs (two buffer sets)."""
        n = ctypes.c_size_t()
        call("tfft_host_space_bytes", self._h, ctypes.byref(n))
        return n.value

    def execute_host(self, signs, h_ins, h_outs, space: torch.Tensor | None = None, stream=None):
        """Transforms signs[0], signs[1], ... of every pinned host tensor in h_ins into the
        matching tensor of h_outs, copies overlapped with the transforms (tfft_execute_host).
        Asynchronous on ``stream``; returns the device space tensor (keep it alive until the
        stream has reached this point)."""
        if space is None:
            space = torch.empty(self.host_space_bytes(), dtype=torch.uint8, device=self.device)
        sg = (ctypes.c_int * len(signs))(*signs)
        n = len(h_ins)
        if len(h_outs) != n:
            raise ValueError("h_ins and h_outs differ in length")
        ins = (ctypes.c_void_p * n)(*[t.data_ptr() for t in h_ins])
        outs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in h_outs])
        call("tfft_execute_host", self._h, len(signs), sg, n, ins, outs, _ptr(space),
             space.numel() * space.element_size(), _stream_ptr(stream))
        return space

    def weighted_energy(self, stage: int, y: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
                        stream=None, u: torch.Tensor | None = None) -> torch.Tensor:
        """sum |y * w|^2 over a stage buffer, as a float64 0-d device tensor; with
        ``u`` given, the same sweep also writes u = w^2 y into it."""
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=y.device)
        up = _ptr(u) if u is not None else ctypes.c_void_p(0)
        call("tfft_weighted_energy", self._h, stage, _ptr(y), _ptr(w), _ptr(out), up, _stream_ptr(stream))
        return out

    def weighted_energy_grad(self, u: torch.Tensor, g: torch.Tensor | None = None, out: torch.Tensor | None = None,
                             mode: str = "fused", keep_input: bool = True, stream=None) -> torch.Tensor:
        """2 g F^H u (stage g -> stage 0): the gradient of g * sum |F(x) w|^2 given
        u = w^2 F(x) from ``weighted_energy(..., u=...)``; ``g`` is a float64 0-d
        device tensor read on the device (None: g = 1)."""
        if out is None:
            out = self.empty_stage(0)
        work = self.workspace(mode, keep_input)
        wp = _ptr(work) if work is not None else ctypes.c_void_p(0)
        wb = work.numel() * work.element_size() if work is not None else 0
        gp = _ptr(g) if g is not None else ctypes.c_void_p(0)
        call("tfft_weighted_energy_grad", self._h, _MODES[mode], _ptr(u), _ptr(out), wp, wb, gp,
             _stream_ptr(stream))
        return out

    def weight_scale(self, stage: int, y: torch.Tensor, w: torch.Tensor, coef: torch.Tensor | None,
                     scale: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """z = scale * coef * w^2 * y elementwise (coef: float64 0-d device tensor or None)."""
        if out is None:
            out = torch.empty_like(y)
        cp = _ptr(coef) if coef is not None else ctypes.c_void_p(0)
        call("tfft_weight_scale", self._h, stage, _ptr(y), _ptr(w), cp, float(scale), _ptr(out),
             _stream_ptr(stream))
        return out

    def redistribute(self, axis_v: int, axis_w: int, x: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        if out is None:
            out = self.empty_stage(self.g - axis_w)
        call("tfft_redistribute", self._h, axis_v, axis_w, _ptr(x), _ptr(out), _stream_ptr(stream))
        return out

    def partial(self, stage: int, axis: int, sign: int, x: torch.Tensor, stream=None) -> torch.Tensor:
        call("tfft_partial", self._h, stage, axis, sign, _ptr(x), _stream_ptr(stream))
        return x

    def device_status(self, reset: bool = False, stream=None) -> int:
        """Status word written by the kernels (1 = a bounded wait expired)."""
        v = ctypes.c_int()
        call("tfft_plan_device_status", self._h, ctypes.byref(v), int(reset), _stream_ptr(stream))
        return v.value

    def launch_info(self, sign: int, mode: str = "fused"):
        """[(kernel name, algorithmic bytes)] for every launch of one execute."""
        out = []
        for k in range(self.num_launches(sign, mode)):
            buf = ctypes.create_string_buffer(64)
            nb = ctypes.c_int64()
            call("tfft_plan_launch_info", self._h, sign, _MODES[mode], k, buf, 64, ctypes.byref(nb))
            out.append((buf.value.decode(), nb.value))
        return out

    def set_wait_limit(self, polls: int):
        """Polls of a TMA copy wait before it gives up (0: default); for error-path tests."""
        call("tfft_plan_set_wait_limit", self._h, int(polls))

    def set_launch_events(self, events):
        """Record torch.cuda.Event objects around every launch of later executes."""
        if not events:
            call("tfft_plan_set_launch_events", self._h, None, 0)
            return
        handles = []
        for ev in events:
            if not ev.cuda_event:
                ev.record()  # creates the underlying cudaEvent_t
            handles.append(ev.cuda_event)
        arr = (ctypes.c_void_p * len(handles))(*handles)
        call("tfft_plan_set_launch_events", self._h, arr, len(handles))

    # ------------------------------------------------------------ host helpers (tests / IO)
    def scatter(self, x: torch.Tensor, stage: int = 0, real: bool = False) -> torch.Tensor:
        """Global array -> stage buffer (each rank's block in rank order).  Not the hot path."""
        parts = []
        for r in range(self.num_ranks):
            st, sz, _ = self.local_box(stage, r, real)
            sl = tuple(slice(a, a + n) for a, n in zip(st, sz))
            parts.append(x[sl].reshape(-1))
        return torch.cat(parts)

    def gather(self, buf: torch.Tensor, stage: int, real: bool = False) -> torch.Tensor:
        """Stage buffer -> global array.  Not the hot path."""
        shape = self.shape if (real or self.kind == "c2c") else self.shape[:-1] + (self.shape[-1] // 2 + 1,)
        out = torch.empty(shape, dtype=buf.dtype, device=buf.device)
        for r in range(self.num_ranks):
            st, sz, off = self.local_box(stage, r, real)
            n = math.prod(sz)
            sl = tuple(slice(a, a + k) for a, k in zip(st, sz))
            out[sl] = buf[off:off + n].reshape(sz)
        return out


class Batch:
    """Many independent transforms (one direction) run by one persistent launch.

    ``plans``: bound complex-to-complex Plans.  Inputs / outputs / workspaces are
    allocated here unless given (one stage buffer each; ``keep_input=False``
    lets each input serve as its transform's scratch).  ``execute()`` is one
    memset plus one kernel launch, so ``graph()`` can capture it.
    """

    def __init__(self, plans, sign: int = -1, ins=None, outs=None, works=None, keep_input: bool = True):
        self.plans = list(plans)
        self.sign = sign
        dev = self.plans[0].device
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        call("tfft_batch_create", ctypes.byref(h), n, arr, sign)
        self._h = h
        self.ins = ins if ins is not None else [
            p.empty_stage(0 if sign < 0 else p.g) for p in self.plans]
        self.outs = outs if outs is not None else [
            p.empty_stage(p.g if sign < 0 else 0) for p in self.plans]
        if works is None:
            works = [p.workspace("fused", True) if keep_input else None for p in self.plans]
            # each transform needs its own workspace (they run concurrently)
            works = [None if w is None else torch.empty_like(w) for w in works]
        self.works = works
        nb = ctypes.c_size_t()
        call("tfft_batch_state_bytes", self._h, ctypes.byref(nb))
        self.state = torch.empty(max(256, nb.value), dtype=torch.uint8, device=dev)
        self._bind()

    def _bind(self, stream=None):
        n = len(self.plans)
        ins = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self.ins])
        outs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self.outs])
        works = (ctypes.c_void_p * n)(*[0 if w is None else w.data_ptr() for w in self.works])
        call("tfft_batch_bind", self._h, _ptr(self.state), self.state.numel(), ins, outs, works,
             _stream_ptr(stream))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.load().tfft_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def execute(self, stream=None):
        call("tfft_batch_execute", self._h, _stream_ptr(stream))

    def autotune(self, reps: int = 3, stream=None):
        call("tfft_batch_autotune", self._h, int(reps), _stream_ptr(stream))

    def num_items(self):
        items = ctypes.c_int64()
        segs = ctypes.c_int()
        call("tfft_batch_num_items", self._h, ctypes.byref(items), ctypes.byref(segs))
        return items.value, segs.value

    def set_variant(self, kind: int, L: int, variant: int, stream=None):
        """Choose the executor tile variant of (kind, L) by hand (tfft_batch_set_variant)."""
        call("tfft_batch_set_variant", self._h, kind, L, variant, _stream_ptr(stream))

    def variant(self, kind: int, L: int) -> int:
        v = ctypes.c_int()
        call("tfft_batch_variant", self._h, kind, L, ctypes.byref(v))
        return v.value

    def set_executor(self, executor: str = "persistent", nstreams: int = 4):
        """'persistent': one persistent kernel over every pass; 'streams': each
        transform's own pass kernels, transforms dealt over `nstreams` forked
        streams (tfft_batch_set_executor)."""
        kind = {"persistent": _lib.TFFT_BATCH_PERSISTENT, "streams": _lib.TFFT_BATCH_STREAMS}[executor]
        call("tfft_batch_set_executor", self._h, kind, int(nstreams))

    @property
    def executor(self):
        """('persistent', 0) or ('streams', number of streams)."""
        e = ctypes.c_int()
        k = ctypes.c_int()
        call("tfft_batch_executor", self._h, ctypes.byref(e), ctypes.byref(k))
        return ("streams" if e.value == _lib.TFFT_BATCH_STREAMS else "persistent", k.value)

    def set_wait_limit(self, cycles: int):
        call("tfft_batch_set_wait_limit", self._h, int(cycles))

    def device_status(self, reset: bool = False, stream=None) -> int:
        v = ctypes.c_int()
        call("tfft_batch_device_status", self._h, ctypes.byref(v), int(reset), _stream_ptr(stream))
        return v.value

    def graph(self):
        """A torch.cuda.CUDAGraph holding one execute (replay() runs the batch)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.execute(s)          # warm-up outside the capture (lazy CUDA set-up)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.execute()
        return g
