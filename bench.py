"""Benchmark: 3D R2C + C2R FFT pair on one GB300 (replicas across GPUs).

One step = one forward R2C + one normalised inverse C2R of a 1024^3 real
grid, in place in the padded layout, FP32 storage and arithmetic (twiddles
generated in FP64).  The same pair in FP64 is timed too and reported under
"fp64".  Input: the synthetic turbulence-like field (random-phase Fourier
modes, amplitude |k|^(-11/6) for 1 <= |k| <= 512, seed 2) taken to real space
by the library's own FP64 inverse, normalised to unit RMS and rounded once to
FP32.  The arrays (4.3 GB FP32, 8.6 GB FP64) are far larger than the 129 MB
L2, so no L2 flush is needed between steps.  The headline is timed with the
library's per-pass profiling off; per-pass times come from a second, profiled
run of the same pairs right after it.  On one GPU the other grids of the
paper's runs (512^3 FP64, 1536^3 and 2048^3 FP32, 2048^3 FP64; Sec. 4, Tables
3-4) are timed as well, under "configs".  "e2e" times the same pair from a
field in pinned host memory back to pinned host memory, host transfers
included (the fastest of four ways of keeping the CPU-GPU link busy).

metric: GFLOP/s with 2.5 N^3 log2(N^3) flops per real transform (5 per pair
element-log), i.e. 5 N^3 log2(N^3) per pair; also HBM GB/s of the three
read+write passes per transform.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N]
Under torchrun each rank times its own replica; rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "R2C+C2R 3D FFT GFLOP/s & HBM GB/s, FP32 vs FP64 at 1024³, 1×GB300"
UNIT = "GFLOP/s"


def pair_flops(n0, n1, n2):
    """2.5 N log2 N per real transform of N points, two transforms per pair."""
    n = n0 * n1 * n2
    return 2 * 2.5 * n * math.log2(n)


def pass_bytes(n0, n1, n2, rsize):
    """HBM bytes of the 3 read+write passes of one transform."""
    c = n0 * n1 * (n2 // 2 + 1) * 2 * rsize
    r = n0 * n1 * n2 * rsize
    return (c + r) + 2 * c + 2 * c


def kernel_sources_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2202_12756_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


def fp64_op_counts(workload):
    """FP64 instructions per complex half-spectrum element of each pass
    (dadd, dmul, dfma; counted by ncu on a small case of the same line
    lengths), or None when the kernels changed since they were counted."""
    p = os.path.join(ROOT, "profiles", "fp64_ops.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_sources_hash():
        return None
    return d.get("workloads", {}).get(workload)


def fp64_roofline(stats, ops, peak, units):
    """FP64-ALU roofline of the slowest FP64 pass: its FP64 instructions per
    launch (ops per element x units) over its mean launch time, against the
    measured FP64 instruction rate (the best of FMA, add and multiply; each
    takes one FP64 issue slot)."""
    if not stats or not peak:
        return None
    top = max(stats, key=lambda s: s["total_ms"])
    avg_ms = top["total_ms"] / top["launches"]
    peak_inst = max(peak["fma_gflops"] / 2.0, peak["add_gflops"], peak["mul_gflops"])
    r = {"bound": "fp64_alu", "kernel": top["name"], "avg_launch_ms": round(avg_ms, 4),
         "peak": round(peak_inst, 1), "unit": "G FP64 instructions/s",
         "peak_measured_gflops": {k: round(v, 1) for k, v in peak.items()}}
    c = (ops or {}).get(top["name"])
    if c is None:
        r.update({"achieved": None, "frac": None, "ops_per_element": None})
        return r
    per_el = c["dadd"] + c["dmul"] + c["dfma"]
    achieved = per_el * units / (avg_ms * 1e-3) / 1e9
    flops = (c["dadd"] + c["dmul"] + 2 * c["dfma"]) * units / (avg_ms * 1e-3) / 1e9
    r.update({"achieved": round(achieved, 1), "frac": round(achieved / peak_inst, 4),
              "ops_per_element": c, "achieved_gflops": round(flops, 1),
              "flops_frac_of_fma_peak": round(flops / peak["fma_gflops"], 4)})
    return r


def ncu_traffic(workload):
    """Per-launch DRAM bytes of each pass from the committed ncu summary, or
    None when the kernels changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_sources_hash():
        return None
    return d.get("workloads", {}).get(workload)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (at most 5 s) for its first
        # sample, then keep only the samples taken from here on
        deadline = time.time() + 5.0
        while not self.lines and self.proc.poll() is None and time.time() < deadline:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def io_bytes_of(grid):
    """Bytes of one dense FP32 real field of the grid."""
    n0, n1, n = grid
    return n0 * n1 * n * 4


def copy_streams_that_fit(field_bytes, ranks, meminfo="/proc/meminfo"):
    """Fields in flight (3, 2, or 0 for none) for the copy-engine end-to-end
    runs: with s streams every rank locks s + 1 host arrays of field_bytes
    (the input and s results); keep that within half of MemAvailable."""
    avail = None
    try:
        with open(meminfo) as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    avail = int(ln.split()[1]) * 1024
    except OSError:
        pass
    if avail is None:
        return 2
    for s in (3, 2):
        if ranks * (s + 1) * field_bytes <= avail // 2:
            return s
    return 0


class HostBuffers:
    """Page-locked host arrays for the end-to-end runs: anonymous memory
    (transparent huge pages requested) registered with cudaHostRegister.
    Measured on these boxes after other GPU work in the same machine, copies
    in both directions at once between HBM and cudaHostAlloc-pinned arrays of
    4 GB fell to 164 GB/s in total, against 343 GB/s for registered ones."""

    def __init__(self):
        self.held = []

    def empty(self, shape):
        import mmap
        import numpy as np
        import torch
        nbytes = int(np.prod(shape)) * 4
        m = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        if hasattr(mmap, "MADV_HUGEPAGE"):
            m.madvise(mmap.MADV_HUGEPAGE)
        a = np.frombuffer(m, dtype=np.float32).reshape(shape)
        a[...] = 0.0  # touch every page before it is locked
        rc = torch.cuda.cudart().cudaHostRegister(a.ctypes.data, nbytes, 0)
        if int(rc) != 0:
            raise RuntimeError(f"cudaHostRegister failed ({rc})")
        self.held.append((m, a))
        return torch.from_numpy(a)

    def release(self):
        import torch
        torch.cuda.synchronize()
        for m, a in self.held:
            torch.cuda.cudart().cudaHostUnregister(a.ctypes.data)
        for m, a in self.held:
            del a
        self.held = []


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)  # one GPU per rank, bound before NCCL starts
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x, pg, device=None):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def make_field(grid, dev):
    """Turbulence-like field of the headline workload, FP64 on the device,
    padded in-place layout, unit RMS."""
    import torch

    import synth
    import paper_2202_12756_gb300 as fft3d
    n0, n1, n2 = grid
    plan64 = fft3d.get_plan(grid, torch.float64, dev)
    buf = plan64.empty_padded()
    spec = buf.view(torch.complex128)
    spec.copy_(synth.turbulence_spectrum_device(n0, n1, n2, seed=2, device=dev))
    plan64.c2r_(buf)
    view = buf[..., :n2]
    rms = torch.sqrt(torch.mean(view * view))
    view.div_(rms)
    torch.cuda.synchronize(dev)
    return plan64, buf


def time_pairs(plan, buf, steps, warmup, dev, pg, profile=False):
    """ms over `steps` in-place pairs on the current stream (after `warmup`
    untimed ones), the plan's launches in them, per-pass stats when
    `profile`, and the sorted per-step times."""
    import torch
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        plan.r2c_(buf)
        plan.c2r_(buf)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    plan.profile_read()  # clear
    plan.set_profiling(profile)
    l0 = plan.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        plan.r2c_(buf)
        plan.c2r_(buf)
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    ms = ev[0].elapsed_time(ev[-1])
    per_step = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(steps))
    launches = plan.launch_count() - l0
    stats = plan.profile_read() if profile else []
    plan.set_profiling(False)
    return ms, launches, stats, per_step


def per_pass(stats, nd=4):
    return {s["name"]: round(s["total_ms"] / s["launches"], nd) for s in stats}


def roofline_from(stats, peak_gbs, traffic):
    if not stats:
        return None
    top = max(stats, key=lambda s: s["total_ms"])
    avg_ms = top["total_ms"] / top["launches"]
    achieved = top["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": top["name"], "achieved": round(achieved, 1), "peak": peak_gbs,
            "unit": "GB/s", "frac": round(achieved / peak_gbs, 4),
            "traffic": (traffic or {}).get(top["name"]),
            "avg_launch_ms": round(avg_ms, 4),
            "per_pass_ms": per_pass(stats)}


def cpu_baseline(budget_s=12.0, n=256):
    """FP64 oracle pairs at n^3 on the host cores for about budget_s seconds."""
    import oracle
    import synth
    f = synth.uniform_field((n, n, n), 0)
    oracle.irfft3(oracle.rfft3(f), f.shape)  # warm the library
    t0 = time.perf_counter()
    pairs = 0
    while True:
        oracle.irfft3(oracle.rfft3(f), f.shape)
        pairs += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(pair_flops(n, n, n) * pairs / dt / 1e9, 3), "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{pairs} FP64 R2C+C2R pairs of a {n}^3 uniform field ({dt:.1f} s)"}


def torch_fft_reference(x_padded, grid, dev, steps=10, warmup=3):
    """torch.fft.rfftn + irfftn (cuFFT) on the same field and GPU, out of
    place: a timed reference point only; the library never calls it."""
    import torch
    n0, n1, n = grid
    x = x_padded[..., :n].contiguous()
    stream = torch.cuda.current_stream(dev)

    def pair():
        return torch.fft.irfftn(torch.fft.rfftn(x), s=(n0, n1, n))

    for _ in range(warmup):
        pair()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pair()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    del x
    torch.cuda.empty_cache()
    return {"ms_per_step": round(ms, 3), "gflops": round(pair_flops(n0, n1, n) / (ms * 1e-3) / 1e9, 1),
            "steps": steps, "what": "torch.fft.rfftn + torch.fft.irfftn (cuFFT), out of place, same FP32 field "
                                    "and GPU; timed reference point, not called by the library"}


def round_trip_error(plan, host_in, host_out):
    """Relative L2 error of the last e2e step's round trip (host tensors)."""
    d = (host_out.double() - host_in.double()).norm() / host_in.double().norm()
    return float(d)


def workload_config(grid, world):
    """The `config` of the bench line (both arms)."""
    n0, n1, n = grid
    return {"workload": f"{n0}x{n1}x{n} real grid, R2C+C2R pair in place (padded rows), FP32, "
                        f"turbulence-like field (|k|^-11/6, seed 2)",
            "grid": list(grid), "layout": "in-place padded", "parallelism": f"replicas x{world}",
            "l2": f"inputs ({n0 * n1 * (n // 2 + 1) * 8 / 1e9:.2f} GB) larger than L2, no flush"}


def reference_config(n, world):
    """The `config` of the reference arm: what it actually times."""
    return {"workload": f"{n}x{n}x{n} real grid, FP64 R2C+C2R pair out of place, the CPU oracle "
                        f"(plain mixed-radix FFT, OpenMP over lines) on the host cores, uniform field (seed 0)",
            "grid": [n, n, n], "dtype": "f64", "layout": "out-of-place dense", "device": "host cores",
            "parallelism": f"rank 0 of {world}"}


def bench_grid(args):
    return tuple(int(x) for x in args.grid.split(",")) if args.grid else (args.n,) * 3


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    if world > 1:
        # torchrun gives every rank one OpenMP thread; rank 0 runs the oracle alone, on the host's cores.
        # torch has already started the OpenMP runtime the oracle's library binds to, so set it there.
        cores = len(os.sched_getaffinity(0))
        os.environ["OMP_NUM_THREADS"] = str(cores)
        try:
            import ctypes
            ctypes.CDLL("libgomp.so.1").omp_set_num_threads(cores)
        except (OSError, AttributeError):
            pass
    import oracle
    import synth
    n = args.ref_n
    f = synth.uniform_field((n, n, n), 0)
    for _ in range(args.warmup):
        oracle.irfft3(oracle.rfft3(f), f.shape)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.irfft3(oracle.rfft3(f), f.shape)
    dt = time.perf_counter() - t0
    val = pair_flops(n, n, n) * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": reference_config(n, world),
            "cpu_baseline": {"value": round(val, 3), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"each step one FP64 R2C+C2R pair of a {n}^3 uniform field (the oracle "
                                       f"as it stands; the GFLOP/s rate uses that pair's flops)"},
            "e2e": {"value": round(val, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# The paper's other grids (Sec. 4, Tables 3-4), timed on one GPU beside the
# headline: (grid, dtype, warm-up pairs, timed pairs).  Each runs in place on a
# device-drawn uniform field; its round-trip error is sampled on four planes.
OTHER_CONFIGS = [((512, 512, 512), "f64", 3, 10), ((1536, 1536, 1536), "f32", 3, 10),
                 ((2048, 2048, 2048), "f32", 3, 5), ((2048, 2048, 2048), "f64", 1, 2)]


def other_configs(dev, peak_gbs):
    import torch
    import paper_2202_12756_gb300 as fft3d
    out = []
    for grid, name, warm, steps in OTHER_CONFIGS:
        n0, n1, n2 = grid
        dt = torch.float32 if name == "f32" else torch.float64
        plan = fft3d.Plan(grid, dt, dev)
        buf = plan.empty_padded()
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        buf.uniform_(-1.0, 1.0, generator=gen)
        planes = [0, n0 // 3, 2 * n0 // 3, n0 - 1]
        x0 = buf[planes, :, :n2].clone()
        plan.r2c_(buf)
        plan.c2r_(buf)
        rt = float((buf[planes, :, :n2] - x0).double().norm() / x0.double().norm())
        del x0
        ms, _, _, _ = time_pairs(plan, buf, steps, warm, dev, None)
        _, _, stats, _ = time_pairs(plan, buf, 1, 0, dev, None, profile=True)
        t = ms / steps
        rsize = 4 if name == "f32" else 8
        gbs = 2 * pass_bytes(n0, n1, n2, rsize) / (t * 1e-3) / 1e9
        out.append({"grid": list(grid), "dtype": name, "layout": "in-place padded", "pairs_timed": steps,
                    "ms_per_pair": round(t, 3), "gflops": round(pair_flops(n0, n1, n2) / (t * 1e-3) / 1e9, 1),
                    "pass_gbs": round(gbs, 1), "hbm_frac_of_peak": round(gbs / peak_gbs, 4),
                    "per_pass_ms": per_pass(stats, 3), "round_trip_rel_l2_sampled": rt,
                    "field": "uniform[-1,1) drawn on the device (torch generator, seed 7); round trip on planes "
                             + ",".join(map(str, planes))})
        del buf, plan
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2202_12756_gb300 as fft3d
    fft3d.load_library()
    grid = bench_grid(args)
    n0, n1, n = grid
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"]

    plan64, buf64 = make_field(grid, dev)
    plan32 = fft3d.get_plan(grid, torch.float32, dev)
    if args.fused:
        plan32.set_fused(True)
    buf32 = plan32.empty_padded()
    buf32.copy_(buf64)

    # ---- FP32 headline: device-resident inputs, profiling off
    clocks = ClockSampler(local)
    clocks.start()
    ms32, launches32, _, steps32 = time_pairs(plan32, buf32, args.steps, args.warmup, dev, pg)
    clk = clocks.stop()
    ms32 = max_over_ranks(ms32, pg, dev)
    t_step = ms32 / args.steps
    flops = pair_flops(n0, n1, n)
    bytes_pair = 2 * pass_bytes(n0, n1, n, 4)
    value = flops * world / (t_step * 1e-3) / 1e9
    # per-pass CUDA events (on the plan's stream) from a second run of the same pairs
    prof_steps = max(5, args.steps // 4)
    ms32p, _, stats32, _ = time_pairs(plan32, buf32, prof_steps, 1, dev, pg, profile=True)

    # ---- reference point: cuFFT through torch.fft on the same field (rank 0)
    torch_ref = torch_fft_reference(buf32, grid, dev) if rank == 0 else None

    # ---- FP64 pair (same field), then its per-pass times and the FP64 roof
    steps64 = max(2, args.steps // 10)
    ms64, launches64, _, _ = time_pairs(plan64, buf64, steps64, args.warmup, dev, pg)
    ms64 = max_over_ranks(ms64, pg, dev)
    t64 = ms64 / steps64
    _, _, stats64, _ = time_pairs(plan64, buf64, 2, 0, dev, pg, profile=True)
    del buf64
    fp64_peak = fft3d.fft3d_measure_fp64_peak()
    units = n0 * n1 * (n // 2 + 1)  # complex half-spectrum elements per pass launch

    # ---- end to end through the public API with the field in pinned host
    # memory, two ways: (a) the forward's first pass reads it straight from
    # host memory and the inverse's last pass writes the result straight back
    # (the only two passes that touch the real array; the strided passes stay
    # in HBM); (b) copy engines move the field into a dense device array and
    # the result back out (cudaMemcpyAsync on the pair's stream) around the
    # device-resident transforms, so the SMs stay free for another field.
    hostbufs = HostBuffers()
    host_in = hostbufs.empty(grid)
    host_in.copy_(buf32[..., :n])
    host_out = hostbufs.empty(grid)
    extra_outs = []  # the other streams' result arrays, reused across the runs
    del buf32
    # enough pairs that filling and draining three streams' pipelines is a small part of the timed region
    e2e_steps = max(24, 2 * max(1, args.steps // 20))

    def e2e_time(nstreams, copies=False):
        """ms per pair with `nstreams` fields in flight (one plan, spectrum
        buffer and output per stream; pair k runs on stream k mod nstreams);
        copies: through a dense device array per stream and the copy engines."""
        plans = [plan32] + [fft3d.Plan(grid, torch.float32, dev) for _ in range(nstreams - 1)]
        cplx = [p.empty_complex() for p in plans]
        while len(extra_outs) < nstreams - 1:
            extra_outs.append(hostbufs.empty(grid))
        outs = [host_out] + extra_outs[:nstreams - 1]
        dreal = [torch.empty(grid, dtype=torch.float32, device=dev) for _ in range(nstreams)] if copies else None
        # every field on a stream of its own; the timing events go on the current stream
        main = torch.cuda.current_stream(dev)
        streams = [torch.cuda.Stream(dev) for _ in range(nstreams)]

        def step(k):
            i = k % nstreams
            with torch.cuda.stream(streams[i]):
                if copies:
                    dreal[i].copy_(host_in, non_blocking=True)
                    plans[i].r2c(dreal[i], cplx[i])
                    plans[i].c2r_overwrite(cplx[i], dreal[i])
                    outs[i].copy_(dreal[i], non_blocking=True)
                else:
                    plans[i].r2c(host_in, cplx[i])
                    plans[i].c2r_overwrite(cplx[i], outs[i])

        for k in range(2 * nstreams):
            step(k)
        torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(main)
        for st in streams:
            st.wait_stream(main)
        for k in range(e2e_steps):
            step(k)
        for st in streams:
            main.wait_stream(st)
        b.record(main)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(a.elapsed_time(b), pg, dev) / e2e_steps
        del plans, cplx, outs, dreal
        torch.cuda.empty_cache()
        return ms

    ms_e2e_1 = e2e_time(1)
    ms_e2e_2 = e2e_time(2)
    # the copy-engine runs lock one more host array per extra stream on every rank of this host
    fields = copy_streams_that_fit(io_bytes_of(grid), world)
    ms_e2e_c2 = e2e_time(2, copies=True) if fields >= 2 else None
    ms_e2e_c3 = e2e_time(3, copies=True) if fields >= 3 else None
    ms_e2e = min(x for x in (ms_e2e_1, ms_e2e_2, ms_e2e_c2, ms_e2e_c3) if x is not None)
    e2e_val = flops * world / (ms_e2e * 1e-3) / 1e9
    io_bytes = io_bytes_of(grid)

    gname = f"{n0}x{n1}x{n}"
    traffic = ncu_traffic(f"{gname} f32")
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step, 4),
        "ms_per_step_min": round(steps32[0], 4), "ms_per_step_median": round(steps32[len(steps32) // 2], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(grid, world),
        "hbm_gbs": round(bytes_pair / (t_step * 1e-3) / 1e9, 1),
        "hbm_frac_of_peak": round(bytes_pair / (t_step * 1e-3) / 1e9 / peak, 4),
        "gflops_paper_convention": round(2 * value, 1),
        "roofline": roofline_from(stats32, peak, traffic),
        "per_pass_timing": f"CUDA events around each pass on the plan's stream, {prof_steps} profiled pairs "
                           f"right after the timed region ({ms32p / prof_steps:.4f} ms per pair with the events)",
        "fp64": {"ms_per_step": round(t64, 3),
                 "gflops": round(flops * world / (t64 * 1e-3) / 1e9, 1),
                 "hbm_gbs": round(2 * pass_bytes(n0, n1, n, 8) / (t64 * 1e-3) / 1e9, 1),
                 "per_pass_ms": per_pass(stats64, 3),
                 "roofline": fp64_roofline(stats64, fp64_op_counts(f"{n0}x{n1}x{n} f64"), fp64_peak, units),
                 "fp32_speedup": round(t64 / t_step, 2)},
        "e2e": {"value": round(e2e_val, 1), "unit": UNIT, "ms_per_step": round(ms_e2e, 3),
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                "ms_per_step_one_stream": round(ms_e2e_1, 3), "ms_per_step_two_streams": round(ms_e2e_2, 3),
                "ms_per_step_copies_two_streams": None if ms_e2e_c2 is None else round(ms_e2e_c2, 3),
                "ms_per_step_copies_three_streams": None if ms_e2e_c3 is None else round(ms_e2e_c3, 3),
                "how": "each pair starts from the field in page-locked host memory (anonymous memory registered with "
                       "cudaHostRegister) and ends with the result there; "
                       "either the forward's first pass reads the host field over the CPU-GPU link and the "
                       "inverse's last pass writes the result back (fft3d_exec_r2c / fft3d_exec_c2r_overwrite "
                       "with host pointers; one or two streams), or cudaMemcpyAsync moves the field into a dense "
                       "device array and the result out around fft3d_exec_r2c / fft3d_exec_c2r_overwrite on "
                       "device arrays (two or three streams); one plan, spectrum and output buffer per stream, "
                       "pair k on stream k mod n; value = the fastest of the four"},
        "gpu_launches": int(launches32),
        "clocks": clk,
        "peak_source": peaks["src"],
    }
    if torch_ref is not None:
        torch_ref["ours_speedup"] = round(torch_ref["ms_per_step"] / t_step, 2)
        line["torch_fft_reference"] = torch_ref
    rt = round_trip_error(plan32, host_in, host_out)
    line["fp32_round_trip_rel_l2"] = rt
    del host_in, host_out, extra_outs
    hostbufs.release()
    if world == 1 and not args.no_configs:
        del plan64, plan32
        torch.cuda.empty_cache()
        line["configs"] = other_configs(dev, peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--grid", type=str, default=None,
                    help="N0,N1,N2 instead of N^3 (profiling and smaller cases)")
    ap.add_argument("--ref-n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other grids (512^3 FP64, 1536^3 / 2048^3 FP32, 2048^3 FP64)")
    ap.add_argument("--fused", action="store_true",
                    help="run the FP32 plans with the opt-in fused plane pass (profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
