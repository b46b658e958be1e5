#!/usr/bin/env python3
"""Benchmark of the flyte hot path on GB300 (prints one JSON line on rank 0).

Workload (one step): y <- 1.5 op(A) x - 0.5 y on a 16384 x 16384 row-major
matrix A with N(0,1) entries stored double-based at k = 3, 4, 5, 6 bytes per
element, op = N and T for every k: eight flyte_gemv calls per step.  A, x and
y are synthetic and seeded; A (0.75 to 1.5 GiB per k) is larger than the L2
cache, so no flush is needed between steps.

Reported:
  value      effective GB/s of the whole step: algorithmic bytes (A k bytes per
             element, x read, y read and written) / device time, summed over
             ranks (replicas: every rank runs the same workload on its GPU)
  per_k      per (k, op): time, GB/s, GFLOP/s and the speedup over native
             binary64 gemv (cuBLAS DGEMV through torch.mv on the same GPU)
  roofline   the kernel with the largest share of the step against the
             measured HBM copy bandwidth
  e2e        the same metric through the public API with the coded matrices,
             x and y in pinned host memory, copied in and y copied back every step
  rows       the other hot-path rows measured on their own (pack/unpack,
             dot/axpy, gemm), each against its roofline
  cpu_baseline  the CPU oracle on a bounded sample of the workload

`--impl reference` times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M = N = 16384
KS = (3, 4, 5, 6)
ALPHA, BETA = 1.5, -0.5
WORKLOAD = "gemv y=1.5*op(A)x-0.5*y, A 16384x16384 N(0,1) double-based k in {3,4,5,6}, op in {N,T}"
METRIC = "effective GB/s and GFLOP/s per byte width k; k-byte vs native FP64 gemv speedup"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["flyte", "reference"], default="flyte")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row measurements")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=6144, help="rows of the CPU-baseline sample")
    ap.add_argument("--case", choices=["gemv", "convert", "blas1", "gemm", "batch"],
                    help="run one small invocation of these kernels (for profilers) and exit; no JSON line")
    ap.add_argument("--k", type=int, default=6, help="byte width for --case")
    ap.add_argument("--size", type=int, default=8192, help="matrix side (gemv, gemm) for --case")
    return ap.parse_args()


def run_case(args):
    """One call of the kernels of a hot-path row on a small, seeded case (inputs larger than L2 but a few
    GB at most), with one untimed call before it; used to capture hardware counters."""
    import torch

    from paper_1601_07789_gb300 import flyte
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    k, size = args.k, args.size
    if args.case == "gemv":
        codes = flyte.pack(torch.randn(size * size, dtype=torch.float64, device=dev, generator=gen), k)
        x = torch.randn(size, dtype=torch.float64, device=dev, generator=gen)
        y = torch.randn(size, dtype=torch.float64, device=dev, generator=gen)
        for _ in range(2):
            for t in "NT":
                flyte.gemv(t, size, size, ALPHA, codes, (k, 1), size, x, BETA, y)
    elif args.case == "convert":
        n = 1 << 26
        v = torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
        c = torch.empty(n * k, dtype=torch.uint8, device=dev)
        for _ in range(2):
            flyte.pack(v, k, out=c)
            flyte.unpack(c, k, flyte.F64, out=v)
    elif args.case == "blas1":
        n = 1 << 26
        xs = flyte.pack(torch.randn(n, dtype=torch.float64, device=dev, generator=gen), k)
        ys = flyte.pack(torch.randn(n, dtype=torch.float64, device=dev, generator=gen), k)
        for _ in range(2):
            flyte.dot(xs, (k, 1), ys, (k, 1))
            flyte.axpy(1.5, xs, (k, 1), ys, (k, 1))      # binary32 alpha: the exact binary32 path
            flyte.axpy(0.1, xs, (k, 1), ys, (k, 1))      # any other alpha: two binary32 parts (k <= 4)
            flyte.scal(1.5, xs, (k, 1))                  # in place, the paper's "scale"
    elif args.case == "batch":
        from paper_1601_07789_gb300 import inputs
        specs = inputs.batch_specs(512, seed=5)
        pools = {f: flyte.pack(torch.randn(1 << 24, dtype=torch.float32 if f[1] == 0 else torch.float64, device=dev,
                                           generator=gen), f[0]) for f in inputs.BATCH_FORMATS}
        xv = torch.randn(4096, dtype=torch.float64, device=dev, generator=gen)
        jobs, keep = [], []
        for sp in specs:
            f = (sp["k"], sp["base"])
            n_, m_ = sp["n"], sp["m"]
            if sp["op"] == 0:
                out = torch.empty(n_, dtype=torch.float32 if f[1] == 0 else torch.float64, device=dev)
                keep.append(out)
                jobs.append(flyte.job(flyte.JOB_UNPACK, f, n_, pools[f], out))
            elif sp["op"] == 1:
                r = torch.empty((), dtype=torch.float64, device=dev)
                keep.append(r)
                jobs.append(flyte.job(flyte.JOB_DOT, f, n_, pools[f], pools[f], fy=f, result=r))
            elif sp["op"] == 2:
                yy = pools[f][: n_ * f[0]].clone()
                keep.append(yy)
                jobs.append(flyte.job(flyte.JOB_AXPY, f, n_, pools[f], yy, fy=f, alpha=1.5))
            else:
                yy = torch.zeros(max(m_, n_), dtype=torch.float64, device=dev)
                keep.append(yy)
                jobs.append(flyte.job(flyte.JOB_GEMV_N if sp["op"] == 3 else flyte.JOB_GEMV_T, f, n_, pools[f], yy,
                                      m=m_, xv=xv, alpha=1.0, beta=0.0))
        ws = flyte.batch_prepare(jobs, device=dev)
        for _ in range(2):
            flyte.batch_launch(ws)
    elif args.case == "gemm":
        base = 0 if k <= 4 else 1
        dt = torch.float32 if base == 0 else torch.float64
        A = flyte.pack(torch.rand(size * size, dtype=dt, device=dev, generator=gen) * 2 - 1, k)
        B = flyte.pack(torch.rand(size * size, dtype=dt, device=dev, generator=gen) * 2 - 1, k)
        C = torch.empty(size * size, dtype=dt, device=dev)
        for _ in range(2):
            flyte.gemm(size, size, size, A, (k, base), B, (k, base), C=C)
    torch.cuda.synchronize()


def gemv_bytes(k: int, trans: str) -> int:
    lenx, leny = (N, M) if trans == "N" else (M, N)
    return M * N * k + 8 * lenx + 16 * leny


def step_bytes() -> int:
    return sum(gemv_bytes(k, t) for k in KS for t in "NT")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    for rel in ("paper_1601_07789_gb300/csrc/gemv.cu", "paper_1601_07789_gb300/csrc/dwacc.cuh",
                "paper_1601_07789_gb300/csrc/flyte_internal.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get(kernel_key)
        if e and e.get("source_hash") == source_hash():
            return e["traffic_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.samples = []
        self.proc = None
        self.thread = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.monotonic(), parts))

    def mark(self):
        self.marks.append(time.monotonic())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        t0, t1 = (self.marks + [0, 0])[:2] if len(self.marks) >= 2 else (0, 1e30)
        inside = [p for t, p in self.samples if t0 <= t <= t1]
        use = inside if len(inside) >= 3 else [p for _, p in self.samples]

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[1]) for p in use if num(p[1]) is not None]
        smax = [num(p[2]) for p in use if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in use for i in range(4) if p[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


# ---- distributed plumbing -------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, local):
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist
    return None


def max_over_ranks(dist, v: float, device: str = "cuda") -> float:
    """The largest value over the ranks (every rank gets it); v itself without a process group."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, bytes_per_step: int, elapsed_ms: float) -> float:
    """Whole-job GB/s of `world` replicas that each ran `steps` steps, over the slowest rank's time."""
    return world * steps * bytes_per_step / (elapsed_ms * 1e-3) / 1e9


# ---- CPU oracle sample ------------------------------------------------------------------

def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def median_ms(fn, stream, reps: int = 20, warmup: int = 3) -> float:
    """Median over `reps` calls of fn's device time (CUDA events on `stream` around each call), after
    `warmup` untimed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def oracle_sample(rows: int, reps: int = 1, threads: int = 1):
    """Time the oracle on `rows` x 16384 slices of the workload; returns (GB/s, seconds, desc).

    With threads > 1 the rows are cut into that many contiguous blocks and each block's oracle
    call runs on its own host thread (the oracle's C calls release the GIL); 'T' then yields one
    partial y per block, which the timing includes adding up."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    from paper_1601_07789_gb300 import inputs
    g = np.random.default_rng(2)
    A = g.standard_normal((rows, N))
    x = inputs.normal_f64(max(M, N), 3)
    y = inputs.normal_f64(max(M, N), 4)
    codes = {k: oracle.pack(A.reshape(-1), 1, k) for k in KS}
    threads = max(1, min(threads, rows))
    cut = [rows * t // threads for t in range(threads + 1)]
    blocks = [(cut[t], cut[t + 1]) for t in range(threads)]

    def part(k, trans, r0, r1):
        sub = codes[k][r0 * N * k:r1 * N * k]
        if trans == "N":
            return oracle.gemv("N", r1 - r0, N, ALPHA, sub, (1, k), N, x, 1, BETA, y[r0:r1], 1)[0]
        return oracle.gemv("T", r1 - r0, N, ALPHA, sub, (1, k), N, x[r0:r1], 1, 0.0, y[:N], 1)[0]

    nbytes = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        for _ in range(reps):
            for k in KS:
                for trans in "NT":
                    outs = list(ex.map(lambda b: part(k, trans, *b), blocks))
                    if trans == "N":
                        nbytes += rows * N * k + 8 * N + 16 * rows
                    else:
                        _ = np.add.reduce(outs) + BETA * y[:N]
                        nbytes += rows * N * k + 8 * rows + 16 * N
        dt = time.perf_counter() - t0
    how = "single-threaded C oracle" if threads == 1 else f"C oracle on {threads} host threads (row blocks)"
    desc = f"{rows} of {M} rows of A (x full length) per (k, op), all eight gemv calls of a step, {how}"
    return nbytes / dt / 1e9, dt, desc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    rows, threads = 1024, host_threads()
    for _ in range(args.warmup):
        oracle_sample(rows, threads=threads)
    total_t, total_gbs = 0.0, []
    for _ in range(args.steps):
        gbs, dt, desc = oracle_sample(rows, threads=threads)
        total_t += dt
        total_gbs.append(gbs)
    value = statistics.mean(total_gbs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1))",
        "config": {"workload": WORKLOAD, "sample_rows": rows, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- GPU arm ------------------------------------------------------------------------------

def run_flyte(args):
    import torch

    from paper_1601_07789_gb300 import flyte

    rank, world, local = dist_env()
    dist = init_dist(world, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flyte.lib()
    stream = torch.cuda.current_stream()

    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    A64 = torch.randn(M * N, dtype=torch.float64, device=dev, generator=gen)
    gen.manual_seed(3)
    x = torch.randn(max(M, N), dtype=torch.float64, device=dev, generator=gen)
    gen.manual_seed(4)
    y = torch.randn(max(M, N), dtype=torch.float64, device=dev, generator=gen)
    codes = {k: flyte.pack(A64, k) for k in KS}
    ws = {t: torch.empty(flyte.workspace_bytes("gemv_n" if t == "N" else "gemv_t", M, N, 0, (6, 1)),
                         dtype=torch.uint8, device=dev) for t in "NT"}

    def call(k, trans, A=None, yv=None):
        flyte.gemv(trans, M, N, ALPHA, codes[k] if A is None else A, (k, 1), N, x, BETA,
                   y if yv is None else yv, ws=ws[trans])

    calls = [(k, t) for k in KS for t in "NT"]
    # each call: the x split, the main kernel and the partial-sum epilogue (16384 columns are 4 'N' tiles)
    launches_per_step = 3 * len(calls)

    for _ in range(args.warmup):
        for k, t in calls:
            call(k, t)
    torch.cuda.synchronize()

    ev = {c: [] for c in calls}
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for c in calls:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call(*c)
            b.record(stream)
            ev[c].append((a, b))
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    if dist:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    elapsed_ms = max_over_ranks(dist, elapsed_ms)
    sampler.stop()
    clocks = sampler.summary()

    per_call_ms = {c: statistics.mean(a.elapsed_time(b) for a, b in ev[c]) for c in calls}
    value = replica_value(world, args.steps, step_bytes(), elapsed_ms)

    # native binary64 gemv on the same GPU (cuBLAS through torch) and our own k = 8
    Am = A64.view(M, N)

    def timeit(fn):
        return median_ms(fn, stream)

    yn = torch.empty(M, dtype=torch.float64, device=dev)
    native_ms = {"N": timeit(lambda: torch.mv(Am, x[:N], out=yn)),
                 "T": timeit(lambda: torch.mv(Am.t(), x[:M], out=yn))}
    a8 = A64.view(torch.uint8)
    k8_ms = {t: timeit(lambda t=t: flyte.gemv(t, M, N, ALPHA, a8, (8, 1), N, x, BETA, y, ws=ws[t]))
             for t in "NT"}

    per_k = {}
    for k in KS:
        per_k[f"k{k}"] = {}
        for t in "NT":
            ms = per_call_ms[(k, t)]
            per_k[f"k{k}"][t] = {
                "ms": round(ms, 4),
                "GBps": round(gemv_bytes(k, t) / (ms * 1e-3) / 1e9, 1),
                "GFLOPs": round(2 * M * N / (ms * 1e-3) / 1e9, 1),
                "speedup_vs_native_fp64": round(native_ms[t] / ms, 3),
                # against this library's own gemv on binary64 storage (k = 8, same kernels): the
                # 8/k storage ratio, free of cuBLAS's binary64-FMA bound
                "speedup_vs_flyte_k8": round(k8_ms[t] / ms, 3),
            }
    hbm_peak, peak_kind = load_peaks()
    dom = max(calls, key=lambda c: per_call_ms[c])
    dom_key = f"gemv_n_pc<F64,{dom[0]}>" if dom[1] == "N" else f"gemv_t_kernel<F64,{dom[0]}>"
    achieved = gemv_bytes(*dom) / (per_call_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom_key, "achieved": round(achieved, 1), "peak": hbm_peak,
                "peak_kind": f"of {peak_kind}", "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "traffic": traffic_for(dom_key),
                "note": "time of the whole flyte_gemv call (x preparation and, for T, the tile sum included)"}

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1), generated on the device)",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "ks": list(KS), "ops": ["N", "T"],
                   "step_bytes": step_bytes(), "l2": "inputs larger than L2 (A is 0.75-1.5 GiB per k)",
                   "parallelism": f"replicas x{world}"},
        "per_k": per_k,
        "native_fp64": {"cublas_dgemv_ms": {t: round(v, 4) for t, v in native_ms.items()},
                        "cublas_dgemv_GBps": {t: round(8 * M * N / (v * 1e-3) / 1e9, 1)
                                              for t, v in native_ms.items()},
                        "flyte_k8_ms": {t: round(v, 4) for t, v in k8_ms.items()}},
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }

    if not args.no_e2e:
        out["e2e"] = run_e2e(args, codes, x, y, ws, dev, dist, world)
    if not args.no_rows and rank == 0:
        out["rows"] = run_rows(dev, hbm_peak)   # per-row figures: rank 0 only
    del A64, codes
    if rank == 0 and world == 1:
        threads = host_threads()
        gbs, dt, desc = oracle_sample(args.cpu_rows, reps=3 if threads > 1 else 1, threads=threads)
        gbs1, dt1, _ = oracle_sample(max(1, args.cpu_rows // 4))
        out["cpu_baseline"] = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                               "sample": desc + (", three passes" if threads > 1 else ""),
                               "seconds": round(dt, 2), "single_thread_value": round(gbs1, 4),
                               "single_thread_sample": f"{max(1, args.cpu_rows // 4)} rows, one host thread"}
    else:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(args, codes, x, y, ws, dev, dist, world):
    """Same metric through the public API from pinned host buffers, y read back every step."""
    import torch

    from paper_1601_07789_gb300 import flyte
    host = {k: codes[k].cpu().pin_memory() for k in KS}
    hx = x.cpu().pin_memory()
    hy = y.cpu().pin_memory()
    out_y = torch.empty_like(hy).pin_memory()
    dA = {k: torch.empty_like(codes[k]) for k in KS}
    dx = torch.empty_like(x)
    dy = torch.empty_like(y)
    steps = max(1, min(args.steps, 20))
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream(device=dev)
    landed = {k: torch.cuda.Event() for k in KS}
    done = torch.cuda.Event()

    def step():
        # the copies run on their own stream and each width's gemvs start as soon as its matrix
        # has landed, so copies of the next widths overlap the compute of the current one
        copy_stream.wait_event(done)
        with torch.cuda.stream(copy_stream):
            dx.copy_(hx, non_blocking=True)
            dy.copy_(hy, non_blocking=True)
            for k in KS:
                dA[k].copy_(host[k], non_blocking=True)
                landed[k].record(copy_stream)
        for k in KS:
            stream.wait_event(landed[k])
            for t in "NT":
                flyte.gemv(t, M, N, ALPHA, dA[k], (k, 1), N, dx, BETA, dy, ws=ws[t])
        out_y.copy_(dy, non_blocking=True)
        done.record(stream)

    done.record(stream)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(dist, e0.elapsed_time(e1))
    h2d = sum(host[k].numel() for k in KS) + hx.numel() * 8 + hy.numel() * 8
    return {"value": round(replica_value(world, steps, step_bytes(), ms), 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": out_y.numel() * 8, "steps": steps,
            "ms_per_step": round(ms / steps, 3)}


def run_rows(dev, hbm_peak):
    """Each other hot-path row timed on its own (CUDA events around each call, median of 20 calls after 3
    untimed ones)."""
    import torch

    from paper_1601_07789_gb300 import flyte
    stream = torch.cuda.current_stream()
    rows = {}

    def timeit(fn):
        return median_ms(fn, stream)

    def entry(nbytes, ms, flops=None):
        d = {"ms": round(ms, 4), "GBps": round(nbytes / (ms * 1e-3) / 1e9, 1),
             "frac_hbm": round(nbytes / (ms * 1e-3) / 1e9 / hbm_peak, 4)}
        if flops:
            d["GFLOPs"] = round(flops / (ms * 1e-3) / 1e9, 1)
        return d

    n = 1 << 28
    gen = torch.Generator(device=dev)
    gen.manual_seed(1601)
    v = torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
    out = torch.empty_like(v)
    for k in KS:
        s = torch.empty(n * k, dtype=torch.uint8, device=dev)
        rows[f"pack_f64_k{k}"] = entry(n * (8 + k), timeit(lambda: flyte.pack_raw(s, v, n, (k, 1))))
        rows[f"unpack_f64_k{k}"] = entry(n * (8 + k), timeit(lambda: flyte.unpack_raw(out, s, n, (k, 1))))
        del s
    xs = flyte.pack(v, 4)
    gen.manual_seed(1602)
    ys = flyte.pack(torch.randn(n, dtype=torch.float64, device=dev, generator=gen), 4)
    res = torch.empty((), dtype=torch.float64, device=dev)
    wsd = torch.empty(flyte.workspace_bytes("dot", 0, n, 0, (4, 1)), dtype=torch.uint8, device=dev)
    rows["dot_f64_k4"] = entry(2 * 4 * n, timeit(lambda: flyte.dot(xs, (4, 1), ys, (4, 1), n=n, out=res, ws=wsd)),
                               2 * n)
    rows["axpy_f64_k4"] = entry(3 * 4 * n, timeit(lambda: flyte.axpy(1.5, xs, (4, 1), ys, (4, 1), n=n)), 2 * n)
    # alpha = 0.1 is not a binary32 number: the two-part binary32 path
    rows["axpy_f64_k4_alpha_not_binary32"] = entry(3 * 4 * n, timeit(lambda: flyte.axpy(0.1, xs, (4, 1), ys, (4, 1), n=n)), 2 * n)
    rows["n"] = n
    del xs, ys
    # double-based k = 5 axpy (x, y as exact binary32 pairs; the binary64 fma was 46 % of HBM)
    xs5 = flyte.pack(v, 5)
    gen.manual_seed(1602)
    ys5 = flyte.pack(torch.randn(n, dtype=torch.float64, device=dev, generator=gen), 5)
    rows["axpy_f64_k5"] = entry(3 * 5 * n, timeit(lambda: flyte.axpy(1.5, xs5, (5, 1), ys5, (5, 1), n=n)), 2 * n)
    # in-place scale by 1.5 (the 23 calls grow x by at most 1.5^23, inside the binary32 window)
    rows["scal_f64_k5"] = entry(2 * 5 * n, timeit(lambda: flyte.scal(1.5, xs5, (5, 1), n=n)), n)
    del v, out, xs5, ys5
    rows.update(run_gemm_rows(dev))
    rows.update(run_refine_rows(dev))
    rows.update(run_batch_rows(dev))
    return rows


def run_gemm_rows(dev):
    """gemm rows: float-based k = 2, 3, 4 at 8192^3 and double-based k = 5 at 4096^3, U(-1,1)."""
    import torch

    from paper_1601_07789_gb300 import flyte
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    out = {}

    def timeit(fn, reps):
        return median_ms(fn, stream, reps=reps)

    # binary64 tensor rate measured here and now: cuBLAS DGEMM (torch.matmul, float64) at 4096^3,
    # the denominator of the double-based rows (as cuBLAS bf16 is the driver's bf16 peak)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    a64 = torch.rand(4096, 4096, dtype=torch.float64, device=dev, generator=gen)
    b64 = torch.rand(4096, 4096, dtype=torch.float64, device=dev, generator=gen)
    c64 = torch.empty(4096, 4096, dtype=torch.float64, device=dev)
    ms64 = timeit(lambda: torch.matmul(a64, b64, out=c64), 10)
    fp64_peak = 2.0 * 4096 ** 3 / (ms64 * 1e-3) / 1e12
    out["fp64_peak_cublas_dgemm_4096"] = {"ms": round(ms64, 3), "TFLOPs": round(fp64_peak, 3)}
    del a64, b64, c64

    for k, size, reps in ((2, 8192, 20), (3, 8192, 20), (4, 8192, 20), (5, 4096, 20)):
        base = 0 if k <= 4 else 1
        f = (k, base)
        dt = torch.float32 if base == 0 else torch.float64
        gen = torch.Generator(device=dev)
        gen.manual_seed(5)
        A = flyte.pack(torch.rand(size * size, dtype=dt, device=dev, generator=gen) * 2 - 1, k)
        gen.manual_seed(6)
        B = flyte.pack(torch.rand(size * size, dtype=dt, device=dev, generator=gen) * 2 - 1, k)
        C = torch.empty(size * size, dtype=dt, device=dev)
        ws = torch.empty(max(flyte.workspace_bytes("gemm", size, size, size, f), 256), dtype=torch.uint8, device=dev)
        ms = timeit(lambda: flyte.gemm(size, size, size, A, f, B, f, C=C, ws=ws), reps)
        useful = 2.0 * size ** 3 / (ms * 1e-3) / 1e12
        nprod = {2: 1, 3: 4, 4: 6}.get(k, 1)
        if base == 0:
            executed = useful * nprod
            out[f"gemm_f32_k{k}_{size}"] = {"ms": round(ms, 3), "useful_TFLOPs": round(useful, 1),
                                            "tensor_TFLOPs": round(executed, 1), "bf16_products": nprod,
                                            "frac_bf16_peak": round(executed / bf16_peak, 4)}
        else:
            out[f"gemm_f64_k{k}_{size}"] = {"ms": round(ms, 3), "useful_TFLOPs": round(useful, 3),
                                            "frac_fp64_measured_dgemm": round(useful / fp64_peak, 4)}
        del A, B, C, ws
    return out


def run_refine_rows(dev):
    """Refinement rows: n = 8192, A = G/sqrt(n) + n I, b N(0,1), to 1e-12 relative residual with two
    Jacobi sweeps per correction on A stored at k = 3, 4, 5, against the same solver with the binary64
    matrix (k = 8) in the sweeps (the native-FP64 baseline)."""
    import torch

    from paper_1601_07789_gb300 import flyte
    n = 8192
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    gen.manual_seed(8)
    A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=gen) / n ** 0.5
    A.diagonal().add_(float(n))
    gen.manual_seed(9)
    b = torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
    A = A.reshape(-1)
    ws = torch.empty(flyte.workspace_bytes("refine", n, n, 0, (4, 1)), dtype=torch.uint8, device=dev)
    out = {}
    for k in (3, 4, 5, 8):
        Ak = flyte.pack(A, k) if k < 8 else A.view(torch.uint8)
        best = None
        for _ in range(4):
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rel = flyte.refine_jacobi(A, Ak, (k, 1), b, x, 1e-12, 50, 2, ws=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        key = f"refine_n{n}_k{k}" if k < 8 else f"refine_n{n}_native_fp64"
        out[key] = {"ms_to_solution": round(best, 3), "corrections": it, "relres": rel}
    # a harder system, A = G/sqrt(n) + 10 I (Jacobi contraction about 1/10 per sweep), with 8 sweeps per
    # correction: the stored precision, not the sweeps, then limits each correction, so fewer bytes
    # per element cost corrections (k = 3) or not (k >= 4) while every sweep reads less
    A.view(n, n).diagonal().sub_(float(n) - 10.0)
    for k in (3, 4, 5, 8):
        Ak = flyte.pack(A, k) if k < 8 else A.view(torch.uint8)
        best = None
        for _ in range(3):
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rel = flyte.refine_jacobi(A, Ak, (k, 1), b, x, 1e-12, 50, 8, ws=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        key = f"refine_n{n}_diag10_inner8_k{k}" if k < 8 else f"refine_n{n}_diag10_inner8_native_fp64"
        out[key] = {"ms_to_solution": round(best, 3), "corrections": it, "relres": rel}
    return out


def run_batch_rows(dev):
    """Batched uneven jobs: 4096 jobs (unpack / dot / axpy with lengths log-uniform in 10^3..10^6,
    gemv N / T with sides log-uniform in 64..4096; double-based k = 2..7 or float-based k = 2, 3) as one
    persistent launch replayed from a CUDA graph, against one launch per job (eager, and the same
    per-job launches captured in a CUDA graph).  Inputs are shared read-only pools per format."""
    import torch

    from paper_1601_07789_gb300 import flyte, inputs
    stream = torch.cuda.current_stream()
    specs = inputs.batch_specs(4096, seed=5)
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    pool_len = max(max(s["n"] * max(s["m"], 1) for s in specs), 1 << 20)
    pools = {}
    for k, base in inputs.BATCH_FORMATS:
        dt = torch.float32 if base == 0 else torch.float64
        pools[(k, base)] = flyte.pack(torch.randn(pool_len, dtype=dt, device=dev, generator=gen), k)
    xpool = torch.randn(4096, dtype=torch.float64, device=dev, generator=gen)
    jobs, calls, keep = [], [], []
    total_bytes = 0
    for s in specs:
        op, k, base, n, m = s["op"], s["k"], s["base"], s["n"], s["m"]
        f = (k, base)
        W = 4 if base == 0 else 8
        pool = pools[f]
        if op == 0:
            out = torch.empty(n, dtype=torch.float32 if base == 0 else torch.float64, device=dev)
            keep.append(out)
            jobs.append(flyte.job(flyte.JOB_UNPACK, f, n, pool, out))
            calls.append(lambda n=n, f=f, out=out, pool=pool: flyte.unpack_raw(out, pool, n, f))
            total_bytes += n * (k + W)
        elif op == 1:
            res = torch.empty((), dtype=torch.float64, device=dev)
            wsd = torch.empty(flyte.workspace_bytes("dot", 0, n, 0, f), dtype=torch.uint8, device=dev)
            keep += [res, wsd]
            ysl = pool[k * (pool_len - n):]
            jobs.append(flyte.job(flyte.JOB_DOT, f, n, pool, ysl, fy=f, result=res))
            calls.append(lambda n=n, f=f, res=res, wsd=wsd, pool=pool, ysl=ysl:
                         flyte.dot_raw(res, n, pool, f, 1, ysl, f, 1, wsd, wsd.numel()))
            total_bytes += 2 * n * k
        elif op == 2:
            y = pool[: n * k].clone()
            keep.append(y)
            jobs.append(flyte.job(flyte.JOB_AXPY, f, n, pool, y, fy=f, alpha=1.5))
            calls.append(lambda n=n, f=f, y=y, pool=pool: flyte.axpy(1.5, pool, f, y, f, n=n))
            total_bytes += 3 * n * k
        else:
            trans = "N" if op == 3 else "T"
            ly = m if op == 3 else n
            lx = n if op == 3 else m
            y = torch.zeros(ly, dtype=torch.float64, device=dev)
            wsg = torch.empty(flyte.workspace_bytes("gemv_n" if op == 3 else "gemv_t", m, n, 0, f),
                              dtype=torch.uint8, device=dev)
            keep += [y, wsg]
            jobs.append(flyte.job(flyte.JOB_GEMV_N if op == 3 else flyte.JOB_GEMV_T, f, n, pool, y, m=m, xv=xpool,
                                  alpha=1.0, beta=0.0))
            calls.append(lambda trans=trans, m=m, n=n, f=f, y=y, wsg=wsg, pool=pool:
                         flyte.gemv_raw(trans, m, n, 1.0, pool, f, n, xpool, 1, 0.0, y, 1, wsg, wsg.numel()))
            total_bytes += m * n * k + 8 * lx + 8 * ly
    ws = flyte.batch_prepare(jobs, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    g1 = torch.cuda.CUDAGraph()
    s1 = torch.cuda.Stream()
    with torch.cuda.graph(g1, stream=s1):
        flyte.batch_launch(ws, stream=s1)
    t_batch = timed(g1.replay, 5)

    def per_job():
        for c in calls:
            c()
    t_eager = timed(per_job, 2)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s1):
        with torch.cuda.stream(s1):
            per_job()
    t_graph = timed(g2.replay, 3)
    flyte.batch_autotune(device=dev)
    ws = flyte.batch_prepare(jobs, ws=ws, device=dev)
    g3 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g3, stream=s1):
        flyte.batch_launch(ws, stream=s1)
    t_tuned = timed(g3.replay, 5)
    # tuned on this very job mix: resident blocks per SM and the tile size of each (op, k, base)
    flyte.batch_autotune_jobs(jobs, device=dev)
    ws = flyte.batch_prepare(jobs, ws=ws, device=dev)
    g4 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g4, stream=s1):
        flyte.batch_launch(ws, stream=s1)
    t_mix = timed(g4.replay, 5)
    names = {0: "unpack", 1: "dot", 2: "axpy", 3: "gemv_n", 4: "gemv_t"}
    table = {f"{names[op]}_{'f64' if base else 'f32'}_k{k}": flyte.batch_tile_size(op, (k, base))
             for op in range(5) for (k, base) in inputs.BATCH_FORMATS}
    gb = total_bytes / 1e9
    return {"batch_4096_jobs": {
        "jobs": len(specs), "GB": round(gb, 3),
        "persistent_graph_ms": round(t_batch, 3), "persistent_graph_GBps": round(gb / (t_batch * 1e-3), 1),
        "persistent_graph_autotuned_ms": round(t_tuned, 3),
        "persistent_graph_autotuned_GBps": round(gb / (t_tuned * 1e-3), 1),
        "persistent_graph_tuned_on_mix_ms": round(t_mix, 3),
        "persistent_graph_tuned_on_mix_GBps": round(gb / (t_mix * 1e-3), 1),
        "tuned_resident_blocks_per_sm": flyte.batch_resident_blocks(),
        "tuned_tiles": table,
        "per_job_launches_ms": round(t_eager, 3), "per_job_launches_GBps": round(gb / (t_eager * 1e-3), 1),
        "per_job_launches_graph_ms": round(t_graph, 3),
        "per_job_launches_graph_GBps": round(gb / (t_graph * 1e-3), 1)}}


def main():
    args = parse_args()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_flyte(args)


if __name__ == "__main__":
    main()
