"""Benchmark: 512^3 complex-to-complex FFT, forward + inverse, on a virtual 4 x 8 pencil grid.

One step = one forward and one inverse transform of a seeded 512^3 complex64
array (Eqs. pencil0-pencil2 and their reverse), redistributions fused into
the FFT passes.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64 DFT matrices) on a bounded
sample of the same workload instead.  With N > 1 (torchrun) every rank runs
its own replica on its own GPU (the path has no cross-GPU exchange); the
timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (512, 512, 512)
GRID = (4, 8)
METRIC = "512^3 c2c fwd+inv ms, 5NlogN GFLOP/s, % HBM roofline; fused vs pack/unpack"
UNIT = "GFLOP/s"


def _set_workload(shape, grid):
    """Workload constants (the default is the 512^3 4 x 8 headline case; other
    shapes serve profiling of small cases)."""
    global SHAPE, GRID, WORKLOAD, N_ELEMS, FLOP_PER_TRANSFORM, FLOP_PER_STEP
    SHAPE, GRID = tuple(shape), tuple(grid)
    WORKLOAD = (f"{'x'.join(map(str, SHAPE))} c2c complex64, virtual "
                f"{'pencil' if len(GRID) == 2 else 'slab' if len(GRID) == 1 else 'grid'} grid "
                f"{'x'.join(map(str, GRID))}, forward+inverse, fused redistribution")
    N_ELEMS = math.prod(SHAPE)
    FLOP_PER_TRANSFORM = 5.0 * N_ELEMS * math.log2(N_ELEMS)   # 5 N log2 N
    FLOP_PER_STEP = 2.0 * FLOP_PER_TRANSFORM                    # forward + inverse


_set_workload(SHAPE, GRID)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"tfft_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def _traffic_per_launch(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    sources that define that kernel are unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        k = rec["kernels"][kernel]
        if k["sources_sha256_16"] != kernel_source_hash(k["sources"]):
            return None
        return k["per_launch_bytes"]
    except Exception:
        return None


# The device sources each measured kernel is compiled from (its translation
# unit, the headers it includes, and the argument structs it is passed).
KERNEL_SOURCES = {
    "fft_strided_tma_L512": ["tfft_tma.cu", "tfft_tma.cuh", "tfft_tiles.cuh", "tfft_common.cuh",
                             "tfft_internal.h", "tfft_device_cache.h"],
    "fft_contig_L512": ["tfft_spec.cu", "tfft_spec_table.h", "tfft_tiles.cuh", "tfft_common.cuh",
                        "tfft_internal.h", "tfft_device_cache.h"],
}


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and blank lines (so that editing a
    comment does not void a record taken on the same code)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_source_hash(names) -> str:
    """sha256 (16 hex digits) over the code (comments stripped) of the named
    files of the library's csrc/."""
    csrc = os.path.join(ROOT, "paper_1804_09536_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(names):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _l2_note() -> str:
    """How the timed inputs relate to the 129 MB L2 (no flush between steps)."""
    mib = 8 * N_ELEMS / 2**20
    size = f"{mib / 1024:.0f} GiB" if mib >= 1024 else f"{mib:.0f} MiB"
    if 8 * N_ELEMS > 129e6:
        return f"inputs larger than L2 ({size} per stage buffer vs 129 MB L2), no flush"
    return f"inputs not larger than L2 ({size} per stage buffer vs 129 MB L2): L2-warm, no flush"


def max_over_ranks(value: float, world: int) -> float:
    """The slowest rank's time (MAX all-reduce over the process group; gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, flop_per_step: float, ms_per_step: float) -> float:
    """Whole-job GFLOP/s: every replica's flops over the slowest replica's time."""
    return world * flop_per_step / (ms_per_step * 1e-3) / 1e9


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_1804_09536_gb300.plan import Plan
    from paper_1804_09536_gb300 import build as _build, inputs

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world > 1:
        _build.build()
    if args.profile_only and args.profile_workload != "fft":
        profile_workload(args, dev)
        return
    plan = Plan(SHAPE, GRID, device=dev, tma=not args.no_tma, precision=args.precision)
    stream = torch.cuda.current_stream()

    # seeded input: complex N(0, 1), the same array on every replica
    x_host = inputs.normal_complex(SHAPE, seed=0)
    x = plan.scatter(x_host.to(dev), 0)
    y = plan.empty_stage(2)
    z = plan.empty_stage(0)
    # the headline loop runs the fused path; profiling runs may pick another mode
    hmode = args.profile_mode if args.profile_only else "fused"
    work = plan.workspace(hmode, keep_input=True)

    def step(mode=hmode, w=work, events=None):
        if events is not None:
            plan.set_launch_events(events[0])
        plan.execute(-1, x, y, mode, w)
        if events is not None:
            plan.set_launch_events(events[1])
        plan.execute(+1, y, z, mode, w)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    nf, nb = plan.num_launches(-1, hmode), plan.num_launches(+1, hmode)
    info_f, info_b = plan.launch_info(-1, hmode), plan.launch_info(+1, hmode)
    for _ in range(args.warmup):
        step()
    # per-launch events for every timed step (recorded on the launching stream)
    ev = [([torch.cuda.Event(enable_timing=True) for _ in range(nf + 1)],
           [torch.cuda.Event(enable_timing=True) for _ in range(nb + 1)]) for _ in range(args.steps)]
    for pair in ev:
        for e in pair[0] + pair[1]:
            e.record(stream)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(events=ev[k])
    t1.record(stream)
    barrier()
    clocks = sampler.stop()
    plan.set_launch_events([])
    total_ms = t0.elapsed_time(t1)
    per_step = [ev[k][0][0].elapsed_time(ev[k][1][-1]) for k in range(args.steps)]
    # per-kernel durations over the timed region
    kern = {}
    for k in range(args.steps):
        for evs, info in ((ev[k][0], info_f), (ev[k][1], info_b)):
            for i, (name, nbytes) in enumerate(info):
                kern.setdefault(name, {"ms": [], "bytes": nbytes})["ms"].append(evs[i].elapsed_time(evs[i + 1]))
    gpu_launches = args.steps * (nf + nb)

    total_ms = max_over_ranks(total_ms, world)
    ms_step = total_ms / args.steps
    value = whole_job_value(world, FLOP_PER_STEP, ms_step)

    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "workload": WORKLOAD, "ms_per_step": ms_step,
                              "kernels": {n: statistics.fmean(r["ms"]) for n, r in kern.items()}}))
        return
    # the same step replayed from a CUDA graph, without the per-launch events
    # (outside the headline timing; reported beside it)
    ksteps = max(3, min(args.steps, 20))
    ms_graph = graph_replay_ms(lambda: step(), ksteps, barrier)
    # comparison paths, same protocol, fewer steps (outside the headline timing):
    # the whole step, then every launch on its own (events around each launch)
    extra, extra_kernels = {}, {}
    for mode in ("unfused", "packed"):
        w2 = plan.workspace(mode)
        for _ in range(2):
            step(mode, w2)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(ksteps):
            step(mode, w2)
        b.record(stream)
        barrier()
        extra[mode] = a.elapsed_time(b) / ksteps
        extra_kernels[mode] = per_launch_times(plan, step, mode, w2, ksteps, barrier, stream)

    # the r2c slab workload (256^3 real, 8-rank slab): fused vs packed, forward + inverse
    r2c = r2c_slab(plan_cls=Plan, dev=dev, steps=max(5, min(args.steps, 50)), barrier=barrier,
                   tma=not args.no_tma)

    # r2c on pencils (the paper's own benchmark kind): 512^3 real on 4 x 8
    r2c_p = r2c_slab(plan_cls=Plan, dev=dev, steps=max(3, min(args.steps, 20)), barrier=barrier,
                     tma=not args.no_tma, shape=(512, 512, 512), grid=(4, 8))

    # the 4-D case: 128^4 on a 3-D virtual grid
    # the appendix's shape with non-2/3/5 lengths (127 by Bluestein) on a 3 x 4 grid
    appa = appendix_a(plan_cls=Plan, dev=dev, steps=max(3, min(args.steps, 20)), barrier=barrier)
    # the same kind of axis (127, Bluestein) in an array larger than L2
    blue = appendix_a(plan_cls=Plan, dev=dev, steps=max(3, min(args.steps, 20)), barrier=barrier,
                      shape=(512, 127, 512), grid=(4, 4))
    fd = fourd_128(plan_cls=Plan, dev=dev, steps=max(3, min(args.steps, 20)), barrier=barrier,
                   tma=not args.no_tma)

    # the tensor-core radix-16 stage on the same workload, FP32 beside it
    fwd_outputs = {"fp32": y.cpu()}
    tc = tc_modes(x, y, dev, steps=max(3, min(args.steps, 20)), barrier=barrier, ms_fp32=ms_step,
                  keep=fwd_outputs if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None)
    # the differentiable 512^3 workload: loss = sum |F(x) w|^2 and its gradient
    ag = autograd_step(plan, x, dev, steps=max(3, min(args.steps, 20)), barrier=barrier)
    # the batch of 48 uneven transforms: one persistent launch in a CUDA graph
    bt = batch48(dev, steps=max(3, min(args.steps, 20)), barrier=barrier, autotune=not args.no_autotune)

    # end to end through the public API with host buffers (tfft_execute_host):
    # every step copies its input from pinned host memory, runs forward +
    # inverse and copies the result back; the copies of neighbouring steps
    # overlap the transforms.  Measured with the pinned buffers where the
    # allocator put them and, when the GPU reports a NUMA affinity, on the
    # host node nearest the GPU (first touch from that node's CPUs).
    esteps = max(3, min(args.steps, 20))
    space = torch.empty(plan.host_space_bytes(), dtype=torch.uint8, device=dev)
    placements = {}
    near = gpu_numa_affinity(local)
    for where in ("default", "gpu_near"):
        if where == "gpu_near" and near is None:
            continue
        h_in, h_out = pinned_pair(x, near if where == "gpu_near" else None)
        plan.execute_host([-1, +1], [h_in] * 2, [h_out] * 2, space, stream)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.execute_host([-1, +1], [h_in] * esteps, [h_out] * esteps, space, stream)
        b.record(stream)
        barrier()
        ms = max_over_ranks(a.elapsed_time(b) / esteps, world)
        # round-trip check of the last step (the timed work really happened)
        err = float(torch.linalg.vector_norm(h_out - h_in) / torch.linalg.vector_norm(h_in))
        rec = {"ms_per_step": round(ms, 4), "round_trip_rel_l2": err,
               "numa_node_in": numa_node_of(h_in), "numa_node_out": numa_node_of(h_out)}
        rec.update(copy_rates(h_in, h_out, dev, stream))
        placements[where] = (ms, rec, h_in, h_out, err)
    del space
    best = min(placements, key=lambda k: placements[k][0])
    e2e_ms, _, h_in, h_out, err = placements[best]
    peak, peak_kind = _peaks()
    dom = max(kern.items(), key=lambda kv: sum(kv[1]["ms"]))
    dom_name, dom_rec = dom
    avg_ms = statistics.fmean(dom_rec["ms"])
    achieved = dom_rec["bytes"] / (avg_ms * 1e-3) / 1e9
    step_bytes = sum(nb_ for _, nb_ in info_f + info_b)
    kernels = {n: {"launches": len(r["ms"]), "avg_ms": round(statistics.fmean(r["ms"]), 4),
                   "share": round(sum(r["ms"]) / sum(sum(q["ms"]) for q in kern.values()), 4),
                   "GBps": round(r["bytes"] / (statistics.fmean(r["ms"]) * 1e-3) / 1e9, 1)}
               for n, r in kern.items()}
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "ms_step_min": round(min(per_step), 4),
        "ms_step_median": round(statistics.median(per_step), 4),
        "graph_ms_per_step": round(ms_graph, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: complex N(0,1) per component, torch CPU generator seed 0",
        "config": {"workload": WORKLOAD, "shape": list(SHAPE), "grid": list(GRID),
                   "l2": _l2_note(),
                   "replicas": world},
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": peak_kind,
                     "traffic": _traffic_per_launch(dom_name),
                     "algorithmic_bytes_per_launch": dom_rec["bytes"]},
        "step_hbm_frac": round(step_bytes / (ms_step * 1e-3) / 1e9 / peak, 4),
        "kernels": kernels,
        "comparison_ms_per_step": {"fused": round(ms_step, 4),
                                   "unfused": round(extra["unfused"], 4),
                                   "packed": round(extra["packed"], 4)},
        "fused_vs_packed_speedup": round(extra["packed"] / ms_step, 3),
        "comparison_kernels": extra_kernels,
        "r2c_slab_256": r2c,
        "r2c_pencil_512": r2c_p,
        "fourd_128": fd,
        "appendix_a_42x127x256": appa,
        "bluestein_512x127x512": blue,
        "tensor_core_512": tc,
        "autograd_512": ag,
        "batch48": bt,
        "e2e": {"value": round(world * FLOP_PER_STEP / (e2e_ms * 1e-3) / 1e9, 2), "unit": UNIT,
                "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": h_in.numel() * h_in.element_size(),
                "d2h_bytes_per_step": h_out.numel() * h_out.element_size(),
                "placement": best, "gpu_numa_affinity": near,
                "placements": {k: v[1] for k, v in placements.items()}},
        "round_trip_rel_l2": err,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fwd_outputs)
        par = line["cpu_baseline"]["parity_vs_oracle"]
        for prec in ("bf16x3", "fp16x3"):
            if f"{prec}_forward_rel_l2" in par:
                line["tensor_core_512"][prec]["rel_l2_vs_oracle"] = par[f"{prec}_forward_rel_l2"]
        if "fp32_forward_rel_l2" in par:
            line["tensor_core_512"]["fp32_rel_l2_vs_oracle"] = par["fp32_forward_rel_l2"]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def per_launch_times(plan, step, mode, work, steps, barrier, stream):
    """Per-kernel average ms and GB/s of algorithmic bytes for one mode, from CUDA
    events recorded around every launch (on the launching stream)."""
    import torch
    info_f, info_b = plan.launch_info(-1, mode), plan.launch_info(+1, mode)
    evs = [([torch.cuda.Event(enable_timing=True) for _ in range(len(info_f) + 1)],
            [torch.cuda.Event(enable_timing=True) for _ in range(len(info_b) + 1)]) for _ in range(steps)]
    for pair in evs:
        for e in pair[0] + pair[1]:
            e.record(stream)
    barrier()
    for k in range(steps):
        step(mode, work, events=evs[k])
    barrier()
    plan.set_launch_events([])
    rec = {}
    for k in range(steps):
        for ev, info in ((evs[k][0], info_f), (evs[k][1], info_b)):
            for i, (name, nbytes) in enumerate(info):
                r = rec.setdefault(name, {"ms": [], "bytes": []})
                r["ms"].append(ev[i].elapsed_time(ev[i + 1]))
                r["bytes"].append(nbytes)
    peak, _ = _peaks()
    out = {}
    for name, r in rec.items():
        ms = statistics.fmean(r["ms"])
        gbps = sum(r["bytes"]) / (sum(r["ms"]) * 1e-3) / 1e9
        out[name] = {"launches_per_step": len(r["ms"]) // steps, "avg_ms": round(ms, 4),
                     "GBps": round(gbps, 1), "hbm_frac": round(gbps / peak, 4)}
    return out


def gpu_numa_affinity(gpu: int):
    """The host NUMA node nvidia-smi reports as nearest this GPU, or None."""
    try:
        txt = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=20).stdout
    except Exception:
        return None
    lines = [ln for ln in txt.splitlines() if ln.strip()]
    head = next((ln for ln in lines if "NUMA Affinity" in ln), None)
    row = next((ln for ln in lines if ln.split() and ln.split()[0] == f"GPU{gpu}"), None)
    if head is None or row is None:
        return None
    cols = [c.strip() for c in head.split("\t") if c.strip()]
    vals = [c.strip() for c in row.split("\t") if c.strip()][1:]
    if "NUMA Affinity" not in cols or len(vals) != len(cols):
        return None
    v = vals[cols.index("NUMA Affinity")]
    try:
        return int(v.split(",")[0].split("-")[0])
    except ValueError:
        return None


def _node_cpus(node: int):
    try:
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            spec = f.read().strip()
    except OSError:
        return None
    cpus = set()
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def pinned_pair(x, node=None):
    """Pinned host copies of x (input) and an output buffer; with `node`, allocated
    and touched while the thread runs on that node's CPUs (first-touch placement)."""
    import torch
    old = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    cpus = _node_cpus(node) if node is not None else None
    if cpus and old is not None:
        allowed = cpus & old if cpus & old else cpus
        try:
            os.sched_setaffinity(0, allowed)
        except OSError:
            pass
    try:
        h_in = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        h_in.copy_(x)
        h_out = torch.empty_like(h_in, pin_memory=True)
        h_out.zero_()
    finally:
        if cpus and old is not None:
            os.sched_setaffinity(0, old)
    return h_in, h_out


def numa_node_of(t):
    """NUMA node(s) holding a host tensor's pages, from /proc/self/numa_maps."""
    addr = t.data_ptr()
    try:
        with open("/proc/self/numa_maps") as f:
            maps = f.read().splitlines()
        with open("/proc/self/maps") as f:
            ranges = f.read().splitlines()
    except OSError:
        return None
    starts = {}
    for ln in ranges:
        lo, hi = ln.split()[0].split("-")
        starts[int(lo, 16)] = int(hi, 16)
    for ln in maps:
        parts = ln.split()
        lo = int(parts[0], 16)
        hi = starts.get(lo)
        if hi is None or not (lo <= addr < hi):
            continue
        nodes = {}
        for p in parts[1:]:
            if p.startswith("N") and "=" in p:
                k, v = p[1:].split("=")
                if k.isdigit():
                    nodes[int(k)] = int(v)
        return nodes or None
    return None


def copy_rates(h_in, h_out, dev, stream):
    """GB/s of one host-to-device and one device-to-host copy of these buffers alone."""
    import torch
    d = torch.empty(h_in.numel(), dtype=h_in.dtype, device=dev)
    out = {}
    for name, fn in (("h2d_GBps", lambda: d.copy_(h_in.reshape(-1), non_blocking=True)),
                     ("d2h_GBps", lambda: h_out.reshape(-1).copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = round(3 * h_in.numel() * h_in.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    del d
    return out


def profile_workload(args, dev):
    """A short loop of one secondary workload for profiler captures (--profile-only)."""
    import torch
    from paper_1804_09536_gb300 import inputs
    from paper_1804_09536_gb300.plan import Batch, Plan
    if args.profile_workload == "r2c":
        plan = Plan(SHAPE, GRID, kind="r2c", device=dev)
        xr = plan.scatter(inputs.normal_real(SHAPE, seed=0).to(dev), 0, real=True)
        yc = plan.empty_stage(plan.g)
        zr = plan.empty_stage(0, real=True)
        work = plan.workspace("fused")

        def one():
            plan.execute(-1, xr, yc, "fused", work)
            plan.execute(1, yc, zr, "fused", work)
    elif args.profile_workload == "batch":
        problems = inputs.batch_problems(48, seed=0)[:args.batch_count]
        plans = [Plan(sh, gr, device=dev) for sh, gr in problems]
        b = Batch(plans, sign=-1)
        for k, (sh, gr) in enumerate(problems):
            b.ins[k].copy_(plans[k].scatter(inputs.uniform_complex(sh, seed=k).to(dev), 0))
        one = b.execute
    else:
        from paper_1804_09536_gb300.autograd import spectral_weight_loss
        plan = Plan(SHAPE, GRID, device=dev)
        x = plan.scatter(inputs.normal_complex(SHAPE, seed=0).to(dev), 0).requires_grad_(True)
        w = plan.scatter(inputs.uniform01_real(SHAPE, seed=1).to(dev), plan.g)

        def one():
            x.grad = None
            spectral_weight_loss(x, w, plan).backward()
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        one()
    e.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_only": True, "workload": args.profile_workload,
                      "ms_per_step": a.elapsed_time(e) / args.steps}))


def graph_replay_ms(one, steps, barrier):
    """ms per replay of `one` captured in a CUDA graph (the same launches without
    the host's per-launch cost), timed with CUDA events after warm-up replays."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        one()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        one()
    for _ in range(3):
        g.replay()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        g.replay()
    b.record()
    barrier()
    return a.elapsed_time(b) / steps


def r2c_slab(plan_cls, dev, steps, barrier, tma=True, shape=(256, 256, 256), grid=(8,)):
    """Real-to-complex forward + inverse on a virtual grid (default: 256^3 on an
    8-rank slab, output 256 x 256 x 129), fused and packed; ms per step and the
    HBM fraction of the fused path's algorithmic bytes."""
    import torch
    from paper_1804_09536_gb300 import inputs
    p = plan_cls(shape, grid, kind="r2c", device=dev, tma=tma)
    x = p.scatter(inputs.normal_real(shape, seed=0).to(dev), 0, real=True)
    y = p.empty_stage(p.g)
    z = p.empty_stage(0, real=True)
    out = {}
    nbytes = 0
    for mode in ("fused", "packed"):
        w = p.workspace(mode)

        def one():
            p.execute(-1, x, y, mode, w)
            p.execute(+1, y, z, mode, w)
        for _ in range(3):
            one()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            one()
        b.record()
        barrier()
        out[mode] = a.elapsed_time(b) / steps
        if mode == "fused":
            nbytes = sum(n for _, n in p.launch_info(-1, mode) + p.launch_info(+1, mode))
            out["graph"] = graph_replay_ms(one, steps, barrier)
    # every launch of the fused path on its own (CUDA events around each launch)
    wf = p.workspace("fused")

    def step(mode="fused", work=wf, events=None):
        if events is not None:
            p.set_launch_events(events[0])
        p.execute(-1, x, y, mode, work)
        if events is not None:
            p.set_launch_events(events[1])
        p.execute(+1, y, z, mode, work)
    kernels = per_launch_times(p, step, "fused", wf, max(3, steps // 2), barrier, torch.cuda.current_stream())
    peak, _ = _peaks()
    n = math.prod(shape)
    oshape = "x".join(str(v) for v in shape[:-1] + (shape[-1] // 2 + 1,))
    return {"workload": f"{'x'.join(map(str, shape))} r2c float32 -> {oshape} complex64, virtual grid "
                        f"{'x'.join(map(str, grid))}, forward+inverse",
            "fused_ms": round(out["fused"], 4), "packed_ms": round(out["packed"], 4),
            "fused_vs_packed_speedup": round(out["packed"] / out["fused"], 3),
            "GFLOPs": round(2 * 2.5 * n * math.log2(n) / (out["fused"] * 1e-3) / 1e9, 1),
            "hbm_frac": round(nbytes / (out["fused"] * 1e-3) / 1e9 / peak, 4),
            "fused_graph_ms": round(out["graph"], 4),
            "hbm_frac_graph": round(nbytes / (out["graph"] * 1e-3) / 1e9 / peak, 4),
            "kernels": kernels,
            "note": "c2r overwrites its input; the forward output is reused as the inverse's input; "
                    "fused_ms: launches from the host each step; fused_graph_ms: the same step "
                    "replayed from a CUDA graph"}


def appendix_a(plan_cls, dev, steps, barrier, shape=(42, 127, 256), grid=(3, 4)):
    """App. A's 42 x 127 x 256 c2c on a 3 x 4 grid (42 = 2.3.7 and the prime 127 by
    Bluestein's convolution form), or another shape: fused forward + inverse,
    per-launch times and GB/s of algorithmic bytes (16 B per element per pass)."""
    import torch
    from paper_1804_09536_gb300 import inputs
    p = plan_cls(shape, grid, device=dev)
    x = p.scatter(inputs.uniform_complex(shape, seed=0).to(dev), 0)
    y = p.empty_stage(p.g)
    z = p.empty_stage(0)
    w = p.workspace("fused", True)
    stream = torch.cuda.current_stream()

    def step(mode="fused", work=w, events=None):
        if events is not None:
            p.set_launch_events(events[0])
        p.execute(-1, x, y, mode, work)
        if events is not None:
            p.set_launch_events(events[1])
        p.execute(+1, y, z, mode, work)
    for _ in range(3):
        step()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    barrier()
    ms = a.elapsed_time(b) / steps
    ms_graph = graph_replay_ms(step, steps, barrier)
    kernels = per_launch_times(p, step, "fused", w, steps, barrier, stream)
    err = float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x))
    n = math.prod(shape)
    peak, _ = _peaks()
    nbytes = sum(nb for _, nb in p.launch_info(-1) + p.launch_info(+1))
    mib = 8 * n / 2**20
    return {"workload": f"{'x'.join(map(str, shape))} c2c complex64 (lengths without a 2/3/5 factorisation by "
                        f"Bluestein), virtual grid {'x'.join(map(str, grid))}, forward+inverse, fused; "
                        f"{mib:.1f} MiB per stage buffer ({'L2-resident' if 8 * n < 129e6 else 'larger than L2'})",
            "ms_per_step": round(ms, 4), "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
            "graph_ms_per_step": round(ms_graph, 4),
            "hbm_frac_graph": round(nbytes / (ms_graph * 1e-3) / 1e9 / peak, 4),
            "kernels": kernels, "round_trip_rel_l2": err}


def fourd_128(plan_cls, dev, steps, barrier, tma=True):
    """128^4 c2c on a virtual 4 x 4 x 2 grid (a 4-D array on a 3-D grid, the
    paper's 4-D case): forward + inverse, fused and packed; ms per step and
    the HBM fraction of the fused path's algorithmic bytes."""
    import torch
    from paper_1804_09536_gb300 import inputs
    shape, grid = (128, 128, 128, 128), (4, 4, 2)
    p = plan_cls(shape, grid, device=dev, tma=tma)
    x = p.scatter(inputs.normal_complex(shape, seed=0).to(dev), 0)
    y = p.empty_stage(p.g)
    z = p.empty_stage(0)
    out = {}
    nbytes = 0
    for mode in ("fused", "packed"):
        w = p.workspace(mode)

        def one():
            p.execute(-1, x, y, mode, w)
            p.execute(+1, y, z, mode, w)
        for _ in range(2):
            one()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            one()
        b.record()
        barrier()
        out[mode] = a.elapsed_time(b) / steps
        if mode == "fused":
            nbytes = sum(n for _, n in p.launch_info(-1, mode) + p.launch_info(+1, mode))
            err = float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x))
        del w
    peak, _ = _peaks()
    n = math.prod(shape)
    return {"workload": "128x128x128x128 c2c complex64, virtual grid 4x4x2, forward+inverse",
            "fused_ms": round(out["fused"], 4), "packed_ms": round(out["packed"], 4),
            "fused_vs_packed_speedup": round(out["packed"] / out["fused"], 3),
            "GFLOPs": round(2 * 5 * n * math.log2(n) / (out["fused"] * 1e-3) / 1e9, 1),
            "hbm_frac": round(nbytes / (out["fused"] * 1e-3) / 1e9 / peak, 4),
            "kernels": sorted({k for k, _ in p.launch_info(-1, "fused")}),
            "round_trip_rel_l2": err}


def tc_modes(x, y_fp32, dev, steps, barrier, ms_fp32, keep=None):
    """512^3 fwd+inv with the length-512 contiguous passes' radix-16 stage on the
    tensor cores (split hi/lo BF16 or FP16, FP32 accumulate); error of the forward
    output relative to the FP32 path (whose own error vs the FP64 oracle is pinned
    by the tests at <= 1e-5; the tests report the TC modes against the oracle)."""
    import torch
    from paper_1804_09536_gb300.plan import Plan

    def rel_l2(a, b, chunks=16):
        num = den = 0.0
        for ca, cb in zip(a.chunk(chunks), b.chunk(chunks)):
            d = (ca.to(torch.complex128) - cb.to(torch.complex128))
            num += float(torch.sum(d.real ** 2 + d.imag ** 2))
            cb2 = cb.to(torch.complex128)
            den += float(torch.sum(cb2.real ** 2 + cb2.imag ** 2))
        return math.sqrt(num / den)

    out = {"fp32_ms_per_step": round(ms_fp32, 4)}
    for prec in ("bf16x3", "fp16x3"):
        p = Plan(SHAPE, GRID, device=dev, precision=prec)
        yp = p.empty_stage(2)
        zp = p.empty_stage(0)
        w = p.workspace("fused", True)
        for _ in range(2):
            p.execute(-1, x, yp, "fused", w)
            p.execute(+1, yp, zp, "fused", w)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            p.execute(-1, x, yp, "fused", w)
            p.execute(+1, yp, zp, "fused", w)
        b.record()
        barrier()
        ms = a.elapsed_time(b) / steps
        p.execute(-1, x, yp, "fused", w)
        torch.cuda.synchronize()
        out[prec] = {"ms_per_step": round(ms, 4), "kernels": [n for n, _ in p.launch_info(-1)],
                     "forward_rel_l2_vs_fp32_path": rel_l2(yp, y_fp32),
                     "round_trip_rel_l2": rel_l2(zp, x)}
        if keep is not None:
            keep[prec] = yp.cpu()
        del p, yp, zp, w
    return out


def autograd_step(plan, x, dev, steps, barrier):
    """loss = sum |F(x) w|^2 (w seeded U[0,1) on the spectrum) and its gradient via the
    adjoint, through torch.autograd; ms per loss + backward step."""
    import torch
    from paper_1804_09536_gb300 import inputs
    from paper_1804_09536_gb300.autograd import spectral_weight_loss
    w = plan.scatter(inputs.uniform01_real(SHAPE, seed=1).to(dev), plan.g)
    xr = x.clone().requires_grad_(True)

    def one():
        xr.grad = None
        loss = spectral_weight_loss(xr, w, plan)
        loss.backward()
        return loss
    for _ in range(2):
        one()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        one()
    b.record()
    barrier()
    ms = a.elapsed_time(b) / steps
    n = math.prod(SHAPE)
    # algorithmic bytes: forward 3 sweeps (2 x 8 B), the loss sweep (read y 8 B + w 4 B, write
    # u = w^2 y 8 B), adjoint 3 sweeps (the factor 2 g applied by its last pass)
    nbytes = n * (6 * 16 + 20)
    peak, _ = _peaks()
    return {"workload": "512^3 c2c pencil 4x8: loss = sum |F(x) w|^2, w U[0,1) seed 1; forward + loss "
                        "+ gradient (adjoint transform) via torch.autograd",
            "ms_per_step": round(ms, 4), "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
            "algorithmic_bytes": nbytes}


def batch48(dev, steps, barrier, autotune=True):
    """48 transforms drawn from the uneven-shape set: the autotuned batch executor
    (one persistent launch, or the plans' own kernels on forked streams) replayed
    from a CUDA graph, vs the same transforms launched plan by plan, eagerly and
    from one CUDA graph."""
    import torch
    from paper_1804_09536_gb300 import inputs
    from paper_1804_09536_gb300.plan import Batch, Plan
    problems = inputs.batch_problems(48, seed=0)
    # graphs=False: the per-plan baselines below launch every kernel directly
    # (the fastest way to run 48 different plans one after the other; a graph
    # per plan adds a graph launch per transform)
    plans = [Plan(sh, gr, device=dev, graphs=False) for sh, gr in problems]
    b = Batch(plans, sign=-1)
    for k, (sh, gr) in enumerate(problems):
        b.ins[k].copy_(plans[k].scatter(inputs.uniform_complex(sh, seed=k).to(dev), 0))
    if autotune:
        x_keep = [t.clone() for t in b.ins]
        b.autotune(reps=3)
        for t, k in zip(b.ins, x_keep):
            t.copy_(k)
    chosen = b.executor
    g = b.graph()

    def timed(fn):
        for _ in range(2):
            fn()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        e.record()
        barrier()
        return a.elapsed_time(e) / steps
    ms_graph = timed(g.replay)
    # both executors, each replayed from its own graph
    execs = {}
    for kind, n in (("persistent", 0), ("streams", chosen[1] if chosen[0] == "streams" else 4)):
        b.set_executor(kind, max(1, n))
        execs[kind if kind == "persistent" else f"streams{n}"] = round(timed(b.graph().replay), 4)
    b.set_executor(chosen[0], max(1, chosen[1]))
    works = [p.workspace("fused", True) for p in plans]

    def per_plan():
        for k, p in enumerate(plans):
            p.execute(-1, b.ins[k], b.outs[k], "fused", works[k])
    ms_plans = timed(per_plan)
    # the per-plan loop captured in one CUDA graph (one stream): the baseline
    # without host launch cost
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        per_plan()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp):
        per_plan()
    ms_plans_graph = timed(gp.replay)
    # forward + inverse: a second batch (sign +1) reads the forward's outputs;
    # each direction replayed from its own graph, and the same two directions
    # plan by plan in one graph
    bi = Batch(plans, sign=+1, ins=b.outs)
    if autotune:
        y_keep = [t.clone() for t in bi.ins]
        bi.autotune(reps=3)
        for t, k in zip(bi.ins, y_keep):
            t.copy_(k)
    gi = bi.graph()

    def fwd_inv():
        g.replay()
        gi.replay()
    ms_fi = timed(fwd_inv)
    rt_num = sum(float((bi.outs[k] - x).abs().pow(2).sum()) for k, x in enumerate(b.ins))
    rt_den = sum(float(x.abs().pow(2).sum()) for x in b.ins)

    def per_plan_fi():
        for k, p in enumerate(plans):
            p.execute(-1, b.ins[k], b.outs[k], "fused", works[k])
            p.execute(+1, b.outs[k], bi.outs[k], "fused", works[k])
    with torch.cuda.stream(s):
        per_plan_fi()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gpi = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gpi):
        per_plan_fi()
    ms_plans_fi_graph = timed(gpi.replay)
    nsum = sum(math.prod(sh) for sh, _ in problems)
    flops = sum(5.0 * math.prod(sh) * math.log2(math.prod(sh)) for sh, _ in problems)
    nbytes = 3 * 16 * nsum
    peak, _ = _peaks()
    items, segs = b.num_items()
    return {"workload": "48 c2c complex64 transforms, shapes drawn (seed 0) from {64^3, 96^3, 128^3, "
                        "64x128x256, 160^3, 256^3}, grids from {1x2, 2x2, 2x4}; forward",
            "elements": nsum, "items": items, "segments": segs,
            "executor": {"kind": chosen[0], "streams": chosen[1]},
            "graph_ms": round(ms_graph, 4), "executor_graph_ms": execs,
            "per_plan_ms": round(ms_plans, 4), "per_plan_graph_ms": round(ms_plans_graph, 4),
            "speedup_vs_per_plan": round(ms_plans / ms_graph, 3),
            "speedup_vs_per_plan_graph": round(ms_plans_graph / ms_graph, 3),
            "GFLOPs": round(flops / (ms_graph * 1e-3) / 1e9, 1),
            "hbm_frac": round(nbytes / (ms_graph * 1e-3) / 1e9 / peak, 4),
            "autotuned": bool(autotune),
            "fwd_inv": {"graph_ms": round(ms_fi, 4), "executor": {"kind": bi.executor[0], "streams": bi.executor[1]},
                        "per_plan_graph_ms": round(ms_plans_fi_graph, 4),
                        "speedup_vs_per_plan_graph": round(ms_plans_fi_graph / ms_fi, 3),
                        "GFLOPs": round(2 * flops / (ms_fi * 1e-3) / 1e9, 1),
                        "hbm_frac": round(2 * nbytes / (ms_fi * 1e-3) / 1e9 / peak, 4),
                        "round_trip_rel_l2": math.sqrt(rt_num / rt_den),
                        "note": "forward batch then inverse batch (each its own graph, executor "
                                "autotuned per direction); baseline: both directions plan by plan "
                                "in one graph"},
            "variants": {f"{'contig' if k == 0 else 'strided'}_{L}": b.variant(k, L)
                         for k in (0, 1) for L in (64, 96, 128, 160, 256) if _has_variant(b, k, L)}}


def _has_variant(b, kind, L):
    try:
        b.variant(kind, L)
        return True
    except Exception:
        return False


# ---------------------------------------------------------------- oracle arm

def _oracle_sample(x, k):
    """The oracle's per-axis DFTs (forward then inverse, axes in the paper's order)
    over k slices of each axis' lines: fraction k / 512 of one step's arithmetic."""
    from oracle import dft
    import numpy as np
    t = time.perf_counter()
    blk = x[:k]                                   # lines along axes 2 and 1
    y = dft.partial_dft(blk, 2, -1)
    y = dft.partial_dft(y, 1, -1)
    col = x[:, :k]                                # lines along axis 0
    c = dft.partial_dft(col, 0, -1)
    c = dft.partial_dft(c, 0, +1)
    y = dft.partial_dft(y, 1, +1)
    y = dft.partial_dft(y, 2, +1)
    _ = float(np.abs(y[0, 0, 0])) + float(np.abs(c[0, 0, 0]))
    return time.perf_counter() - t


def _rel_l2_np(got, ref, chunks=64):
    import numpy as np
    num = den = 0.0
    for a, b in zip(np.array_split(np.asarray(got).reshape(-1), chunks),
                    np.array_split(np.asarray(ref).reshape(-1), chunks)):
        d = a.astype(np.complex128) - b
        num += float(np.vdot(d, d).real)
        den += float(np.vdot(b, b).real)
    return math.sqrt(num / den)


def cpu_baseline(fwd_outputs=None):
    """The oracle on the host cores: one whole step (forward + backward of the whole
    array on the same virtual grid, FP64 DFT matrices and Alg. 3 exchanges).  Its
    forward output also gives the whole-array error of the GPU forward outputs
    (FP32 and the tensor-core modes) against the oracle."""
    import numpy as np
    from oracle import dft, redistribute
    from paper_1804_09536_gb300 import inputs
    x = inputs.normal_complex(SHAPE, seed=0).numpy()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    b0 = redistribute.scatter(x, GRID, 0)
    t = time.perf_counter()
    yf = dft.distributed_forward(b0, SHAPE, GRID)
    tf = time.perf_counter() - t
    t = time.perf_counter()
    zb = dft.distributed_backward(yf, SHAPE, GRID)
    tb = time.perf_counter() - t
    secs = tf + tb
    g = "x".join(map(str, GRID))
    out = {"value": round(FLOP_PER_STEP / secs / 1e9, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
           "ms_per_step": round(secs * 1e3, 1),
           "sample": f"one whole step: the oracle's distributed_forward + distributed_backward of the "
                     f"{'x'.join(map(str, SHAPE))} array on the {g} virtual grid (FP64 exact-angle DFT "
                     f"matrices, Alg. 3 exchanges), {tf:.1f} s + {tb:.1f} s, 5NlogN flops"}
    parity = {"oracle_round_trip_rel_l2": _rel_l2_np(zb, b0)}
    del zb
    for name, yh in (fwd_outputs or {}).items():
        parity[f"{name}_forward_rel_l2"] = _rel_l2_np(yh.numpy(), yf)
    parity["note"] = "whole-array rel-L2 of the GPU forward outputs (stage buffers) against the oracle's"
    out["parity_vs_oracle"] = parity
    del yf
    # the oracle's index-level redistribution (Alg. 3 subarray copies), one exchange
    # of the whole stage buffer
    t = time.perf_counter()
    _ = redistribute.exchange_subarray(b0, SHAPE, GRID, 0, 1)
    tr = time.perf_counter() - t
    out["redistribution"] = {"ms": round(tr * 1e3, 1), "GBps": round(2 * b0.nbytes / tr / 1e9, 2),
                             "sample": "oracle exchange_subarray, stage 0 -> 1 of the whole "
                                       f"{'x'.join(map(str, SHAPE))} complex64 buffer (read + write)"}
    del b0, _
    # context, not the oracle: a library CPU FFT on the same input and cores
    try:
        import scipy.fft
        scipy.fft.ifftn(scipy.fft.fftn(x[:8], workers=cores, norm="forward"), workers=cores, norm="forward")
        t = time.perf_counter()
        y = scipy.fft.fftn(x, workers=cores, norm="forward")
        z = scipy.fft.ifftn(y, workers=cores, norm="forward")
        tl = time.perf_counter() - t
        del y, z
        out["library_context"] = {"value": round(FLOP_PER_STEP / tl / 1e9, 2), "unit": UNIT,
                                  "ms_per_step": round(tl * 1e3, 1),
                                  "sample": f"scipy.fft.fftn + ifftn (pocketfft, complex64, workers={cores}) "
                                            "of the whole array, one step; a library, not the oracle"}
    except ImportError:
        pass
    return out


def run_reference(args):
    """The oracle arm: the FP64 oracle on a bounded sample of the workload per step.

    Each step runs the oracle's per-axis DFTs (forward then inverse along all
    axes) over k of the 512 slices, k chosen so that the whole warm-up + timed
    run stays near --ref-seconds; ms_per_step is the measured time of that
    sampled step (nothing is extrapolated) and value the sampled flops over it.
    """
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1804_09536_gb300 import inputs
    x = inputs.normal_complex(SHAPE, seed=0).numpy()
    t1 = _oracle_sample(x, 2)
    per_step = args.ref_seconds / max(1, args.steps + args.warmup)
    k = int(max(1, min(SHAPE[0], round(2 * per_step / max(t1, 1e-3)))))
    for _ in range(args.warmup):
        _oracle_sample(x, k)
    ts = [_oracle_sample(x, k) for _ in range(args.steps)]
    frac = k / SHAPE[0]
    secs = sum(ts) / len(ts)
    value = frac * FLOP_PER_STEP / secs / 1e9
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"oracle FP64 exact-angle DFT matrices, forward+inverse along all 3 axes over {k} of "
              f"{SHAPE[0]} slices per step ({frac:.4f} of the step's lines); ms_per_step is the "
              f"measured time of that sampled step")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs * 1e3, 3), "sample_fraction": round(frac, 6),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic: complex N(0,1), seed 0",
            "config": {"workload": WORKLOAD, "shape": list(SHAPE), "grid": list(GRID)},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: CPU seconds the whole warm-up + timed run aims at")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", type=int, nargs="+", default=list(SHAPE))
    ap.add_argument("--grid", type=int, nargs="*", default=list(GRID))
    ap.add_argument("--no-tma", action="store_true",
                    help="plain load/store passes only (comparison and profiling)")
    ap.add_argument("--no-autotune", action="store_true", help="batch executor with default tiles")
    ap.add_argument("--profile-only", action="store_true",
                    help="headline loop only (no comparison paths, e2e or CPU baseline)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "fp16x3"],
                    help="arithmetic of the length-512 contiguous passes in the headline loop")
    ap.add_argument("--profile-workload", default="fft", choices=["fft", "batch", "loss", "r2c"],
                    help="with --profile-only: the loop to run (fft: the headline step; batch: the "
                         "batch executor over the first --batch-count transforms; loss: the "
                         "loss + gradient step; r2c: real-to-complex forward + complex-to-real "
                         "inverse of --shape on --grid)")
    ap.add_argument("--batch-count", type=int, default=48)
    ap.add_argument("--profile-mode", default="fused", choices=["fused", "unfused", "packed"],
                    help="with --profile-only: the execution mode of the headline loop")
    args = ap.parse_args()
    if args.precision != "fp32" and not args.profile_only:
        ap.error("--precision is for profiling runs (--profile-only); the headline is FP32")
    _set_workload(args.shape, args.grid)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
