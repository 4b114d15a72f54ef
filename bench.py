#!/usr/bin/env python
"""Benchmark of the AM-QFT batched complex DFT on GB300.

Workload (one step): forward then unnormalised inverse AM-QFT of a batch of
4096 complex64 transforms of length N = 2^16 (2^28 points, Re/Im iid N(0,1),
synthetic), i.e. 2^29 transformed points per step.  Every buffer is 2 GiB,
far larger than the 126 MB L2, so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  `value` is device time only (inputs resident
in HBM); `e2e` is the batch's forward transform from pinned host memory to
pinned host memory through the library's host-memory entry point (every step
copies the whole input in and the whole result out, chunk by chunk, the
copies overlapping the transforms); `roofline` is the forward kernel (16 bytes
per point) against the measured HBM copy bandwidth; `cpu_baseline` is the CPU
oracle (float64 recursion) on the host cores.  --workload c1|c3|c4|c5 prints
the line of another configuration instead.

  python bench.py [--steps K] [--warmup W] [--variant V]
  python -m torch.distributed.run --nproc-per-node N bench.py --gpus N   (weak scaling)
  python bench.py --impl reference     (the CPU oracle as the reference arm)
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AM-QFT batched FFT Gpoints/s and % HBM roofline at stated rel-L2 vs FP64 oracle"
UNIT = "Gpoints/s"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_POINT = 16  # complex64 read + write


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="amqft", choices=["amqft", "reference"])
    ap.add_argument("--variant", type=int, default=4)
    ap.add_argument("--log2n", type=int, default=16)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "c4", "c5"],
                    help="c2 (default): the batched complex64 forward+inverse line; c1: N=1024 latency of "
                         "all variants; c3: 16-bit storage; c4: ragged batch in one CUDA graph; c5: autograd "
                         "forward+backward")
    ap.add_argument("--dtype16", default="bf16", choices=["bf16", "fp16", "i16"])
    ap.add_argument("--constants", default="table", choices=["table", "fly", "auto"],
                    help="band-level trig constants: the plan's table, evaluated on the fly in the kernels, or "
                         "whichever the autotuner times faster on this workload")
    return ap.parse_args()


def workload(args):
    n = 1 << args.log2n
    return {
        "workload": f"batched complex64 forward+inverse AM-QFT, N=2^{args.log2n}, batch {args.batch} "
                    f"({args.batch * n} points), Re/Im iid N(0,1)",
        "log2n": args.log2n,
        "batch_per_gpu": args.batch,
        "variant": args.variant,
        "step": "forward + inverse (2 transforms of every point)",
        "points_per_step_per_gpu": 2 * args.batch * n,
        "l2": "inputs larger than L2 (each buffer 2 GiB vs 126 MB L2), no flush",
    }


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources that define the forward kernel of a configuration: its code and
# the launch-shape constants it is compiled and launched with.  Variant 4 at
# 2^14 .. 2^16 (complex64) runs the paired-region kernel, every other
# single-pass configuration the fused kernel.
FUSED_KERNEL_SOURCES = ("amqft_device.cuh", "amqft_bands.cuh", "amqft_fused_impl.cuh")
PAIRED_KERNEL_SOURCES = ("amqft_paired.cuh", "amqft_paired_impl.cuh")


def uses_paired_kernel(variant, log2n) -> bool:
    return variant == 4 and 14 <= log2n <= 16


def kernel_name(variant, log2n) -> str:
    if uses_paired_kernel(variant, log2n):
        return f"paired-region forward kernel, variant {variant}"
    if log2n <= 16:
        return f"fused forward kernel, variant {variant}"
    return f"multi-pass forward sequence (all its kernels), variant {variant}"


def kernel_source_sha(variant=4, log2n=16) -> str:
    h = hashlib.sha256()
    names = PAIRED_KERNEL_SOURCES if uses_paired_kernel(variant, log2n) else FUSED_KERNEL_SOURCES
    for name in names:
        with open(os.path.join(ROOT, "paper_1404_1810_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(variant, log2n, batch):
    """bytes per launch of the forward kernel from a committed ncu summary, if
    it was taken on the current kernel sources (else None)."""
    sha = kernel_source_sha(variant, log2n)
    pat = re.compile(r"bench-traffic:\s*variant=(\d+)\s+log2n=(\d+)\s+batch=(\d+)\s+source_sha=(\w+)"
                     r"\s+bytes_per_launch=(\d+)")
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(p):
            m = pat.search(line)
            if m and int(m.group(1)) == variant and int(m.group(2)) == log2n and m.group(4) == sha:
                per_launch = int(m.group(5))
                return int(per_launch * batch / int(m.group(3)))
    return None


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        else:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(dev):
    """Host CPUs and NUMA node local to the GPU, from sysfs (read only)."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(dev)],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = bus.split(":", 1)
        sysid = f"{int(dom, 16):04x}:{rest}".lower()
        base = f"/sys/bus/pci/devices/{sysid}"
        with open(base + "/numa_node") as f:
            node = int(f.read())
        with open(base + "/local_cpulist") as f:
            cpus = _cpulist(f.read())
        return (cpus or None), node
    except Exception:
        return None, None


def copy_bandwidth(xh, yh, xd, yd, stream, reps=3):
    """Plain pinned-host <-> device copies of the e2e buffers, in the same run:
    each direction alone and both at once on two streams."""
    import torch

    nbytes = xh.numel() * xh.element_size()
    s2 = torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def h2d():
        with torch.cuda.stream(stream):
            xd.copy_(xh, non_blocking=True)

    def d2h():
        with torch.cuda.stream(stream):
            yh.copy_(yd, non_blocking=True)

    def both():
        ev = torch.cuda.Event()
        ev.record(stream)
        s2.wait_event(ev)
        with torch.cuda.stream(stream):
            xd.copy_(xh, non_blocking=True)
        with torch.cuda.stream(s2):
            yh.copy_(yd, non_blocking=True)
        ev2 = torch.cuda.Event()
        ev2.record(s2)
        stream.wait_event(ev2)

    t_in, t_out, t_both = timed(h2d), timed(d2h), timed(both)
    g_in, g_out, g_both = nbytes / t_in / 1e6, nbytes / t_out / 1e6, nbytes / t_both / 1e6
    # a pinned -> pinned transform moves 8 bytes a point each way; a direction
    # cannot beat its own copy rate, so min(h2d, d2h) / 8 bounds the points a
    # second; with the two directions overlapped (as the chunked call runs
    # them) the tighter bound is their rate when both run at once
    return {"h2d_gbs": g_in, "d2h_gbs": g_out, "both_directions_gbs_each": g_both,
            "bound_gpts": min(g_in, g_out) / 8.0, "bidirectional_bound_gpts": g_both / 8.0, "bytes_each": nbytes}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(x_host_rows, variant, sign_pair=True):
    """float64 oracle recursion (forward + inverse) over a bounded sample."""
    import numpy as np

    import oracle

    oracle.build()
    n = x_host_rows.shape[1]
    t0 = time.perf_counter()
    _, threads = oracle.amqft_batch(x_host_rows[:1], variant, threads=1)
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    # about 12 s of wall time on all cores: S transforms forward + S inverse,
    # one transform pair taking about 2 * t1 on each core
    s = max(cores, int(12.0 * cores / max(2 * t1, 1e-3)) // cores * cores)
    s = min(s, x_host_rows.shape[0])
    rows = np.ascontiguousarray(x_host_rows[:s])
    t0 = time.perf_counter()
    y, threads = oracle.amqft_batch(rows, variant, threads=cores)
    oracle.amqft_batch(y, variant, threads=cores, sign=+1)
    dt = time.perf_counter() - t0
    return {"value": 2 * s * n / dt / 1e9, "unit": UNIT, "cores": int(threads), "kind": "oracle",
            "sample": f"{s} transforms of N={n} forward + inverse, float64 AM-QFT variant {variant}, "
                      f"OpenMP over the batch ({threads} threads), {dt:.2f} s wall"}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (bounded sample
    per step); rank 0 only."""
    import numpy as np

    import oracle
    import synth

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    oracle.build()
    n = 1 << args.log2n
    cores = os.cpu_count() or 1
    s = cores  # one forward + one inverse transform per core per step
    x = synth.normal_complex(n, s, config=2, stream=0)
    for _ in range(args.warmup):
        y, thr = oracle.amqft_batch(x, args.variant, threads=cores)
        oracle.amqft_batch(y, args.variant, threads=cores, sign=+1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y, thr = oracle.amqft_batch(x, args.variant, threads=cores)
        oracle.amqft_batch(y, args.variant, threads=cores, sign=+1)
    dt = time.perf_counter() - t0
    value = 2 * s * n * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(thr), "kind": "oracle",
                         "sample": f"each step: {s} transforms of N={n} forward + inverse (float64 "
                                   f"AM-QFT variant {args.variant}, OpenMP over the sample)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _event_steps(torch, stream, K, fns):
    """Time K steps of the callables fns (each one launch group) with CUDA
    events on `stream`; returns (total ms, mean ms of each callable)."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(K)]
    torch.cuda.synchronize()
    for i in range(K):
        ev[i][0].record(stream)
        for j, f in enumerate(fns):
            f()
            ev[i][j + 1].record(stream)
    torch.cuda.synchronize()
    total = ev[0][0].elapsed_time(ev[K - 1][len(fns)])
    per = [statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(K)) for j in range(len(fns))]
    return total, per


def oracle_amqft(x, variant):
    import oracle

    oracle.build()
    return oracle.amqft(x, variant)


def run_extra(args):
    """The other configurations of the workload list, each as its own JSON
    line, measured beside the plain float32 batched form on the same GPU."""
    import numpy as np
    import torch

    import synth
    from paper_1404_1810_gb300 import Plan, amqft_autograd, build, dequantize, load

    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    build.build()
    load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    peak, kind = measured_peak()
    K, W = args.steps, max(args.warmup, 3)
    sampler = ClockSampler(0)

    def fp32_reference(log2n, batch):
        n = 1 << log2n
        x = synth.device_normal_complex64(n, batch, dev)
        y, z = torch.empty_like(x), torch.empty_like(x)
        p = Plan(log2n, args.variant, batch)
        for _ in range(W):
            p.fwd(x, y, stream)
            p.inv(y, z, stream)
        tot, per = _event_steps(torch, stream, K, [lambda: p.fwd(x, y, stream), lambda: p.inv(y, z, stream)])
        p.close()
        del x, y, z
        return {"value": 2 * batch * n / (tot / K * 1e-3) / 1e9, "unit": UNIT, "fwd_kernel_ms": per[0],
                "config": f"complex64 N=2^{log2n} x {batch}, variant {args.variant}"}

    if args.workload == "c1":
        import oracle

        oracle.build()
        n = 1024
        x = synth.uniform_complex(n, 1, config=1)
        truth = oracle.naive_dft(x[0].astype(np.complex64).astype(np.complex128))
        xd = torch.from_numpy(x.astype(np.complex64)).to(dev)
        res = {}
        sampler.start()
        for v in range(1, 9):
            p = Plan(10, v, 1)
            y = torch.empty_like(xd)
            for _ in range(W):
                p.fwd(xd, y, stream)
            tot, per = _event_steps(torch, stream, K, [lambda: p.fwd(xd, y, stream)])
            err = float(np.linalg.norm(y.cpu().numpy()[0] - truth) / np.linalg.norm(truth))
            res[str(v)] = {"us_per_transform": 1e3 * per[0], "rel_l2_vs_long_double_dft": err}
            p.close()
        clocks = sampler.stop()
        best = min(r["us_per_transform"] for r in res.values())
        line = {"metric": "AM-QFT single complex DFT latency, N=1024, all 8 variants", "value": best, "unit": "us",
                "higher_is_better": False, "n_gpus": 1, "steps": K, "warmup": W, "dtype": "f32",
                "data": "synthetic", "config": {"workload": "single complex DFT N=1024, Re/Im iid U[-1,1)",
                                                "batch": 1}, "per_variant": res, "clocks": clocks,
                "gpu_launches": 8 * K, "vs_baseline": None, "impl": "amqft"}
        print(json.dumps(line), flush=True)
        return 0

    if args.workload == "c3":
        import oracle

        oracle.build()
        dt = {"bf16": 1, "fp16": 2, "i16": 3}[args.dtype16]
        tdt = {1: torch.bfloat16, 2: torch.float16, 3: torch.int16}[dt]
        log2n = args.log2n
        n = 1 << log2n
        batch = 1 << (27 - log2n)
        x = torch.view_as_real(synth.device_normal_complex64(n, batch, dev))
        # int16 block floating point: the signal times 2^12 as integers, exponent 0
        x = (x * 4096.0).round().to(tdt).contiguous() if dt == 3 else x.to(tdt).contiguous()
        y, z = torch.empty_like(x), torch.empty_like(x)
        ey = torch.empty(batch, dtype=torch.int32, device=dev)
        ez = torch.empty(batch, dtype=torch.int32, device=dev)
        p = Plan(log2n, args.variant, batch, dt)
        for _ in range(W):
            p.fwd(x, y, stream, ey)
            p.inv(y, z, stream, exp_in=ey, exp_out=ez)
        sampler.start()
        launches0 = p.launches()
        tot, per = _event_steps(torch, stream, K, [lambda: p.fwd(x, y, stream, ey),
                                                   lambda: p.inv(y, z, stream, exp_in=ey, exp_out=ez)])
        launches = p.launches() - launches0
        clocks = sampler.stop()
        value = 2 * batch * n / (tot / K * 1e-3) / 1e9
        achieved = 8 * batch * n / (per[0] * 1e-3) / 1e9
        errs, maxe = [], []
        for i in (0, batch - 1):
            xin = torch.view_as_complex(x[i].double()).cpu().numpy()
            r64 = oracle.amqft(xin, args.variant)
            yi = dequantize(y[i:i + 1], ey[i:i + 1]).cpu().numpy()[0]
            errs.append(float(np.linalg.norm(yi - r64) / np.linalg.norm(r64)))
            maxe.append(float(np.max(np.abs(yi - r64)) / np.max(np.abs(r64))))
        p.close()
        del x, y, z
        ref = fp32_reference(log2n, batch)
        line = {"metric": f"AM-QFT {args.dtype16} storage / f32 compute, Gpoints/s", "value": value, "unit": UNIT,
                "higher_is_better": True, "n_gpus": 1, "steps": K, "warmup": W, "dtype": f"{args.dtype16}-storage",
                "data": "synthetic",
                "config": {"workload": f"16-bit storage forward+inverse, N=2^{log2n}, batch {batch} (2^27 points), "
                                       f"Re/Im iid N(0,1){' x 2^12' if dt == 3 else ''} rounded to {args.dtype16}",
                           "variant": args.variant,
                           "l2": "inputs larger than L2"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "peak_kind": kind,
                             "kernel_ms": per[0], "algorithmic_bytes_per_launch": 8 * batch * n},
                "accuracy": {"rel_l2_vs_f64_oracle": max(errs), "max_abs_over_max": max(maxe), "tol": 4e-3,
                             "sample": "transforms 0 and batch-1, oracle on the 16-bit input"},
                "vs_fp32_same_gpu": ref, "clocks": clocks, "gpu_launches": launches, "vs_baseline": None,
                "impl": "amqft"}
        print(json.dumps(line), flush=True)
        return 0

    if args.workload == "c4":
        from paper_1404_1810_gb300 import RaggedPlan
        from paper_1404_1810_gb300.autotune import tune_ragged

        count = 20000
        lg = synth.ragged_log2n(count, 4, 18)
        off = synth.ragged_offsets(lg)
        total = int((np.int64(1) << lg.astype(np.int64)).sum())
        g = torch.Generator(device=dev)
        g.manual_seed(synth.SEED_BASE + 4)
        x = torch.view_as_complex(torch.rand((total, 2), generator=g, device=dev) * 2 - 1)
        y = torch.empty_like(x)
        lgd, offd = torch.from_numpy(lg).to(dev), torch.from_numpy(off).to(dev)
        p = RaggedPlan(18, args.variant, count, total)
        knobs = tune_ragged(p, x, lgd, offd, y, reps=3)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            p.exec(x, lgd, offd, y, stream=side)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        launches0 = p.launches()
        with torch.cuda.graph(graph):
            p.exec(x, lgd, offd, y)
        per_replay = p.launches() - launches0  # kernels captured in the graph
        for _ in range(W):
            graph.replay()
        sampler.start()
        tot, per = _event_steps(torch, stream, K, [graph.replay])
        clocks = sampler.stop()
        value = total / (tot / K * 1e-3) / 1e9
        achieved = 16 * total / (per[0] * 1e-3) / 1e9
        # sampled accuracy: the longest transform and a short one vs the float64 oracle
        errs = []
        for i in (int(np.argmax(lg)), int(np.argmin(lg))):
            n = 1 << int(lg[i])
            xs = x[int(off[i]):int(off[i]) + n].cpu().numpy().astype(np.complex128)
            ys = y[int(off[i]):int(off[i]) + n].cpu().numpy()
            r64 = oracle_amqft(xs, args.variant)
            errs.append(float(np.linalg.norm(ys - r64) / np.linalg.norm(r64)))
        skipped = p.skipped()
        p.close()
        # the same lengths as per-length batched calls on contiguous buffers
        hist = np.bincount(lg, minlength=19)
        bufs = []
        for c in range(4, 19):
            if hist[c]:
                n = 1 << c
                xb = torch.view_as_complex(torch.rand((int(hist[c]), n, 2), generator=g, device=dev) * 2 - 1)
                bufs.append((Plan(c, args.variant, int(hist[c])), xb, torch.empty_like(xb)))
        fns = [lambda b=b: b[0].fwd(b[1], b[2], stream) for b in bufs]
        for f in fns:
            f()
        btot, _ = _event_steps(torch, stream, K, fns)
        for b in bufs:
            b[0].close()
        del bufs
        line = {"metric": "AM-QFT ragged batch Gpoints/s (one CUDA graph)", "value": value, "unit": UNIT,
                "higher_is_better": True, "n_gpus": 1, "steps": K, "warmup": W, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "ragged batch: 20000 complex64 transforms, log2 N ~ U{4..18}, Re/Im iid "
                                       "U[-1,1), packed offsets", "points": total, "variant": args.variant,
                           "length_histogram": {str(c): int(hist[c]) for c in range(4, 19)},
                           "launch": "bucket pass + persistent launch (N <= 2^13) + persistent cluster launches "
                                     "(2^14..2^16) + multi-pass (2^17, 2^18), replayed as one CUDA graph",
                           "autotuned_knobs": knobs, "l2": "inputs larger than L2"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "peak_kind": kind,
                             "kernel_ms": per[0], "algorithmic_bytes_per_launch": 16 * total,
                             "kernel": "whole graph (16 B per point)"},
                "accuracy": {"rel_l2_vs_f64_oracle": max(errs), "skipped": skipped,
                             "sample": "longest and shortest transform"},
                "vs_fp32_same_gpu": {"value": total / (btot / K * 1e-3) / 1e9, "unit": UNIT,
                                     "config": "the same lengths as 15 per-length batched forward calls"},
                "clocks": clocks, "vs_baseline": None, "impl": "amqft",
                "gpu_launches": per_replay * K, "gpu_launches_per_replay": per_replay}
        print(json.dumps(line), flush=True)
        return 0

    # c5: autograd, 512 real signals of N = 2^14 lifted to complex
    import oracle

    oracle.build()
    log2n, batch = 14, 512
    n = 1 << log2n
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_BASE + 5)
    xr = (torch.rand((batch, n), generator=g, device=dev) * 2 - 1).requires_grad_(True)
    w = torch.rand((n,), generator=g, device=dev)
    state = {}

    def fwd():
        z = torch.complex(xr, torch.zeros_like(xr))
        X = amqft_autograd(z, args.variant)
        state["loss"] = (w * (X.real ** 2 + X.imag ** 2)).sum()

    def bwd():
        xr.grad = None
        state["loss"].backward()

    for _ in range(W):
        fwd()
        bwd()
    sampler.start()
    tot, per = _event_steps(torch, stream, K, [fwd, bwd])
    clocks = sampler.stop()
    value = batch * n / (tot / K * 1e-3) / 1e9
    # kernel-only: the two transforms of a step
    p = Plan(log2n, args.variant, batch)
    zc = torch.complex(xr.detach(), torch.zeros_like(xr.detach())).contiguous()
    yk, gk = torch.empty_like(zc), torch.empty_like(zc)
    for _ in range(W):
        p.fwd(zc, yk, stream)
        p.inv(yk, gk, stream)
    ktot, kper = _event_steps(torch, stream, K, [lambda: p.fwd(zc, yk, stream), lambda: p.inv(yk, gk, stream)])
    p.close()
    achieved = 32 * batch * n / ((kper[0] + kper[1]) * 1e-3) / 1e9
    x0 = xr.detach()[0].double().cpu().numpy().astype(np.complex128)
    wn = w.double().cpu().numpy()
    X0 = oracle.amqft(x0, args.variant)
    gref = 2.0 * oracle.amqft(wn * X0, args.variant, sign=+1).real
    gerr = float(np.linalg.norm(xr.grad[0].double().cpu().numpy() - gref) / np.linalg.norm(gref))
    ref = fp32_reference(log2n, batch)
    line = {"metric": "AM-QFT autograd forward+backward Gpoints/s", "value": value, "unit": UNIT,
            "higher_is_better": True, "n_gpus": 1, "steps": K, "warmup": W, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "autograd: 512 real signals N=2^14 lifted to complex, loss = sum_k w_k |X_k|^2, "
                                   "w ~ U[0,1); step = forward + backward", "variant": args.variant},
            "step_ms": {"forward_incl_loss": per[0], "backward": per[1]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": kind,
                         "kernel_ms": {"forward": kper[0], "adjoint": kper[1]},
                         "algorithmic_bytes": "32 B per point for the two transforms; mask and loss elementwise "
                                              "ops excluded"},
            "accuracy": {"grad_rel_l2_vs_oracle_adjoint": gerr, "sample": "signal 0, 2 Re F^H(w X), float64"},
            "vs_fp32_same_gpu": ref, "clocks": clocks, "gpu_launches": 2 * K, "vs_baseline": None,
            "impl": "amqft"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        return run_extra(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_1404_1810_gb300 import Plan, build, load
    from paper_1404_1810_gb300.multi import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    build.build()
    load()

    n = 1 << args.log2n
    dev = torch.device("cuda", local)
    x = synth.device_normal_complex64(n, args.batch, dev, seed_offset=rank)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    plan = Plan(args.log2n, args.variant, args.batch)
    from paper_1404_1810_gb300.autotune import tune_constants
    if args.constants == "auto":
        const_tune = tune_constants(plan, x, reps=3, use_cache=False)
    else:
        plan.constants = args.constants
        const_tune = None
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        plan.fwd(x, y, stream)
        plan.inv(y, z, stream)
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches0 = plan.launches()
    for i in range(K):
        ev[i][0].record(stream)
        plan.fwd(x, y, stream)
        ev[i][1].record(stream)
        plan.inv(y, z, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = plan.launches() - launches0  # this library's kernels in the timed region
    clocks = sampler.stop()
    total_ms = ev[0][0].elapsed_time(ev[K - 1][2])
    fwd_ms = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(K))
    inv_ms = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(K))
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / K
    points_step = 2 * args.batch * n * world
    value = points_step / (ms_step * 1e-3) / 1e9

    # accuracy on sampled transforms (float64 oracle), after the timed region
    accuracy = None
    e2e = None
    cpu = None
    if rank == 0 and args.log2n <= 20:  # the oracle's sample stays within seconds up to 2^20
        import oracle

        oracle.build()
        rows = [0, args.batch - 1]
        xr = x[rows].cpu().numpy().astype(np.complex128)
        yr = y[rows].cpu().numpy().astype(np.complex128)
        errs, e32s, exact = [], [], True
        for i in range(len(rows)):
            r64 = oracle.amqft(xr[i], args.variant)
            r32 = oracle.amqft(xr[i], args.variant, prec="f32")
            errs.append(float(np.linalg.norm(yr[i] - r64) / np.linalg.norm(r64)))
            e32s.append(float(np.linalg.norm(r32 - r64) / np.linalg.norm(r64)))
            exact = exact and bool(np.array_equal(yr[i].astype(np.complex64), r32.astype(np.complex64)))
        stated = 2e-7 * args.log2n
        enforced = max(stated, 2.0 * max(e32s))
        accuracy = {"rel_l2_vs_f64_oracle": max(errs), "stated_tol": stated,
                    "f32_recursion_rel_l2": max(e32s), "enforced_tol": enforced,
                    "within_enforced_tol": max(errs) <= enforced,
                    "note": ("the paper's recursion evaluated in float32 exceeds 2e-7*log2N from N = 2^14 on; "
                             "the enforced bound is max(2e-7*log2N, 2 x that error)"),
                    "bitexact_vs_f32_recursion": exact, "sample": "transforms 0 and batch-1"}

    if not args.no_e2e:
        # through the host-memory entry point: the batch's forward transform
        # from pinned host memory to pinned host memory, the copies of each
        # chunk overlapping the transform of the next inside the call
        cpus, node = gpu_local_cpus(local)
        old_aff = None
        if cpus:
            try:  # allocate (and first-touch) the pinned buffers on the GPU's own host node
                old_aff = os.sched_getaffinity(0)
                os.sched_setaffinity(0, cpus)
            except Exception:
                old_aff = None
        xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        yh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        xh.copy_(x)
        yh.copy_(x)
        if old_aff is not None:
            os.sched_setaffinity(0, old_aff)
        copies = copy_bandwidth(xh, yh, x, y, stream)
        copies["numa_node"] = node
        ke = max(1, args.e2e_steps)
        for _ in range(2):
            plan.fwd_host(xh, yh, stream=stream)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            plan.fwd_host(xh, yh, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(e0.elapsed_time(e1) / ke)
        nbytes = x.numel() * x.element_size()
        e2e = {"value": args.batch * n * world / (te * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": te, "steps": ke,
               "step": "one forward transform of the batch, pinned host -> pinned host, through amqft_exec_host",
               "copies": copies,
               "frac_of_copy_bound": (args.batch * n * world / (te * 1e-3) / 1e9) / copies["bound_gpts"]
               if copies.get("bound_gpts") else None,
               "frac_of_bidirectional_copy_bound":
                   (args.batch * n * world / (te * 1e-3) / 1e9) / copies["bidirectional_bound_gpts"]
                   if copies.get("bidirectional_bound_gpts") else None}
        del xh, yh

    # both constants modes' forward kernel time on this workload, after the timed region
    mode_used = plan.constants
    if const_tune is None:
        const_tune = tune_constants(plan, x, reps=3, use_cache=False)
        plan.constants = mode_used
    constants = {"mode": mode_used, "chosen_by": "autotuner" if args.constants == "auto" else "flag",
                 "table_kernel_ms": const_tune["table_ms"], "fly_kernel_ms": const_tune["fly_ms"]}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x[:256].cpu().numpy().astype(np.complex128), args.variant)

    if rank == 0:
        peak, kind = measured_peak()
        achieved = BYTES_PER_POINT * args.batch * n / (fwd_ms * 1e-3) / 1e9
        traffic = recorded_traffic(args.variant, args.log2n, args.batch)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kernel_name(args.variant, args.log2n),
                         "peak_kind": kind, "kernel_ms": fwd_ms, "inverse_kernel_ms": inv_ms,
                         "algorithmic_bytes_per_launch": BYTES_PER_POINT * args.batch * n},
            "clocks": clocks,
            "e2e": e2e,
            "constants": constants,
            "gpu_launches": launches,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "impl": "amqft",
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
