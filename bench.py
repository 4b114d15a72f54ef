#!/usr/bin/env python
"""Benchmark of the AM-QFT batched complex DFT on GB300.

Workload (one step): forward then unnormalised inverse AM-QFT of a batch of
4096 complex64 transforms of length N = 2^16 (2^28 points, Re/Im iid N(0,1),
synthetic), i.e. 2^29 transformed points per step.  Every buffer is 2 GiB,
far larger than the 126 MB L2, so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  `value` is device time only (inputs resident
in HBM); `e2e` adds the pinned host->device copy of the input and the
device->host copy of the result every step; `roofline` is the forward kernel
(16 bytes per point) against the measured HBM copy bandwidth; `cpu_baseline`
is the CPU oracle (float64 recursion) on the host cores.

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


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1404_1810_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(variant, log2n, batch):
    """bytes per launch of the forward kernel from a committed ncu summary, if
    it was taken on the current kernel sources (else None)."""
    sha = kernel_source_sha()
    pat = re.compile(r"bench-traffic:\s*variant=(\d+)\s+log2n=(\d+)\s+batch=(\d+)\s+source_sha=(\w+)"
                     r"\s+bytes_per_launch=(\d+)")
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(p):
            m = pat.search(line)
            if m and int(m.group(1)) == variant and int(m.group(2)) == log2n and m.group(4) == sha:
                per_launch = int(m.group(5))
                return int(per_launch * batch / int(m.group(3)))
    return None


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


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_1404_1810_gb300 import Plan, build, load

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
    for i in range(K):
        ev[i][0].record(stream)
        plan.fwd(x, y, stream)
        ev[i][1].record(stream)
        plan.inv(y, z, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    total_ms = ev[0][0].elapsed_time(ev[K - 1][2])
    fwd_ms = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(K))
    inv_ms = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(K))
    t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_step = total_ms / K
    points_step = 2 * args.batch * n * world
    value = points_step / (ms_step * 1e-3) / 1e9

    # accuracy on sampled transforms (float64 oracle), after the timed region
    accuracy = None
    e2e = None
    cpu = None
    if rank == 0:
        import oracle

        oracle.build()
        rows = [0, args.batch - 1]
        xr = x[rows].cpu().numpy().astype(np.complex128)
        yr = y[rows].cpu().numpy().astype(np.complex128)
        errs, exact = [], True
        for i in range(len(rows)):
            r64 = oracle.amqft(xr[i], args.variant)
            r32 = oracle.amqft(xr[i], args.variant, prec="f32")
            errs.append(float(np.linalg.norm(yr[i] - r64) / np.linalg.norm(r64)))
            exact = exact and bool(np.array_equal(yr[i].astype(np.complex64), r32.astype(np.complex64)))
        accuracy = {"rel_l2_vs_f64_oracle": max(errs), "north_star_tol": 2e-7 * args.log2n,
                    "bitexact_vs_f32_recursion": exact, "sample": "transforms 0 and batch-1"}

    if not args.no_e2e:
        xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        zh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        xh.copy_(x)
        xd = torch.empty_like(x)
        ke = max(1, args.e2e_steps)
        for _ in range(2):
            xd.copy_(xh, non_blocking=True)
            plan.fwd(xd, y, stream)
            plan.inv(y, z, stream)
            zh.copy_(z, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            xd.copy_(xh, non_blocking=True)
            plan.fwd(xd, y, stream)
            plan.inv(y, z, stream)
            zh.copy_(z, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = torch.tensor([e0.elapsed_time(e1) / ke], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        nbytes = x.numel() * x.element_size()
        e2e = {"value": points_step / (float(te.item()) * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": float(te.item()), "steps": ke}
        del xh, zh, xd

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
                         "kernel": f"fused forward kernel, variant {args.variant}",
                         "peak_kind": kind, "kernel_ms": fwd_ms, "inverse_kernel_ms": inv_ms,
                         "algorithmic_bytes_per_launch": BYTES_PER_POINT * args.batch * n},
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": 2 * K,
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
