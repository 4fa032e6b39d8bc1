"""Benchmark of the batched C2C FFT on one B300 (or N, one rank per GPU).

Workload (default, "sweep"): the power-of-two sweep N = 2^10 .. 2^24, each
size holding 2^26 complex64 elements (512 MiB per buffer; batch 2^26/N),
inputs i.i.d. normal(0,1) re-seeded per size with seed 1; one step = forward
then inverse of every size.  Metric: GFLOP/s with the nominal 5*N*log2(N)
flops per transform and direction.  Inputs are larger than L2 (126 MB), so
no flush is needed between iterations.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the slow reference arm), on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1203_4938_b300 import inputs  # noqa: E402

TOTAL_LOG2 = 26
LO, HI = 10, 24
METRIC = "C2C FFT GFLOP/s (5N*log2N/t), fwd+inv sweep N=2^10..2^24, 2^26 complex64 per size"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum per launch) of
# each sweep size's kernel at the full sweep size (2^26 elements), from the
# one-kernel ncu captures summarised in profiles/sweep_dram_traffic.md.  The
# numbers belong to the kernel sources hashed there and to the plan printed
# beside each size; when either differs the benchmark reports the traffic as
# null until a new capture replaces them.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_dram_traffic.md")
TRAFFIC_SOURCES = ["butterfly.cuh", "stockham_pow2.cuh", "persist.cuh", "threestep.cuh", "tma.cuh",
                   "rows_staged.cuh", "kernels_launch.cuh", "k_rows.cu", "k_rows_staged.cu", "k_persist.cu",
                   "k_three.cu", "twiddle.cu"]


def _code_only(src: str) -> str:
    """C/CUDA source without comments and with whitespace runs collapsed, so
    that editing a comment does not invalidate a capture of the same code."""
    out, i, n, quote = [], 0, len(src), None
    while i < n:
        c = src[i]
        if quote:
            out.append(c)
            if c == "\\" and i + 1 < n:
                out.append(src[i + 1])
                i += 2
                continue
            if c == quote:
                quote = None
            i += 1
        elif c in "\"'":
            quote = c
            out.append(c)
            i += 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(" ".join(ln.split()) for ln in "".join(out).splitlines() if ln.strip())


def traffic_sources_sha(read=None) -> str:
    """Hash of the code (comments ignored) of the kernels the traffic table
    was captured from; `read(name)` returns a source's text (default: the
    working tree)."""
    import hashlib
    if read is None:
        def read(f):
            with open(os.path.join(ROOT, "paper_1203_4938_b300", "csrc", f), encoding="utf-8") as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(f.encode())
        h.update(_code_only(read(f)).encode())
    return h.hexdigest()[:16]


def traffic_table(path: str = TRAFFIC_FILE):
    """(sources hash, {log2 N: (plan, DRAM bytes per launch)}) parsed from the
    profile summary; ({}, None) when it is missing."""
    sha, rows = None, {}
    try:
        with open(path) as fh:
            for line in fh:
                if line.startswith("Kernel sources hash:"):
                    sha = line.split(":", 1)[1].strip().strip("`")
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                if len(cells) >= 3 and cells[0].isdigit():
                    rows[int(cells[0])] = (cells[1].strip("`"), float(cells[2]) * 1e6)
    except OSError:
        return None, {}
    return sha, rows


def measured_traffic(logn: int, plan_desc: str):
    """DRAM bytes per launch of the sweep kernel for 2^logn, or None when the
    kernel sources or the plan differ from the captured ones (or the size was
    not captured)."""
    sha, rows = traffic_table()
    try:
        if sha is None or traffic_sources_sha() != sha:
            return None
    except OSError:
        return None
    if logn not in rows or rows[logn][0] != plan_desc:
        return None
    return rows[logn][1]


def flops_per_step(lo=LO, hi=HI, total_log2=TOTAL_LOG2):
    # per size and direction: batch * 5 N log2 N = 5 * 2^total * log2 N
    return sum(2 * 5.0 * (1 << total_log2) * k for k in range(lo, hi + 1))


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, device) -> float:
    """Slowest rank's time (the job finishes when the last replica does)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job GFLOP/s: every rank runs the full workload (replicas, weak
    scaling) and the job takes as long as the slowest rank."""
    return world * flops_per_rank / (ms_max * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle arm (bounded sample)
# --------------------------------------------------------------------------
def oracle_sample(budget_elems: int = 1 << 21, sizes=None, threads: int = 0):
    """Time the FP64 oracle (forward + inverse) on min(batch, budget/N) transforms
    of each sweep size on `threads` host threads (0: all cores); returns
    (GFLOP/s, seconds, threads, description)."""
    import oracle
    threads = threads or oracle.num_cpus()
    sizes = sizes or inputs.sweep_sizes(TOTAL_LOG2, LO, HI)
    fl, secs = 0.0, 0.0
    for k, n, b in sizes:
        m = max(1, min(b, budget_elems // n))
        x = inputs.normal_batch(m, n, seed=1)
        t0 = time.perf_counter()
        y = oracle.fft(x, -1, threads)
        oracle.fft(y, +1, threads)
        secs += time.perf_counter() - t0
        fl += 2 * 5.0 * n * k * m
    desc = (f"FP64 C oracle (radix-2), fwd+inv of min(batch, 2^{int(math.log2(budget_elems))}/N) transforms per size "
            f"N=2^{LO}..2^{HI}, {threads} threads")
    return fl / secs / 1e9, secs, threads, desc


def sweep_config(args, world: int) -> dict:
    """The sweep's `config` object (shared by both arms)."""
    return {"workload": f"sweep N=2^{args.lo}..2^{args.hi}, 2^{TOTAL_LOG2} complex64/size"
                        f"{' (quick: 1/16 batch)' if args.quick else ''}, fwd+inv, normal(0,1) seed 1",
            "l2": "inputs (512 MiB per size) larger than L2; no flush", "parallelism": f"replicas{world}"}


def reference_budget(steps: int) -> int:
    """Elements per size and step of the reference arm, so that warm-up plus
    timed steps take a few minutes on the host cores in total."""
    if steps <= 8:
        return 1 << 21
    if steps <= 24:
        return 1 << 19
    return 1 << 17


def oracle_step(step: int, budget: int, threads: int, sizes):
    """One reference-arm step: forward + inverse of min(batch, budget/N)
    transforms of every sweep size N <= budget, plus one transform of one
    larger size, taken in turn (step mod their count).  Returns (flops, s)."""
    import oracle
    small = [t for t in sizes if t[1] <= budget]
    large = [t for t in sizes if t[1] > budget]
    pick = small + ([large[step % len(large)]] if large else [])
    fl, secs = 0.0, 0.0
    for k, n, b in pick:
        m = max(1, min(b, budget // n))
        x = inputs.normal_batch(m, n, seed=1)
        t0 = time.perf_counter()
        y = oracle.fft(x, -1, threads)
        oracle.fft(y, +1, threads)
        secs += time.perf_counter() - t0
        fl += 2 * 5.0 * n * k * m
    return fl, secs


def run_reference(args):
    """The FP64 oracle on the host cores, on this benchmark's metric and
    config: W untimed steps, then K timed ones; value = flops / seconds over
    the timed steps.  Rank 0 only."""
    import oracle
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    threads = oracle.num_cpus()
    sizes = inputs.sweep_sizes(TOTAL_LOG2, args.lo, args.hi)
    steps = max(1, args.steps)
    budget = reference_budget(steps + max(0, args.warmup))
    if args.quick:
        budget = min(budget, 1 << 17)
    for w in range(max(0, args.warmup)):
        oracle_step(w, budget, threads, sizes)
    fl, secs = 0.0, 0.0
    for i in range(steps):
        f, s = oracle_step(args.warmup + i, budget, threads, sizes)
        fl += f
        secs += s
    value = fl / secs / 1e9
    nlarge = sum(1 for t in sizes if t[1] > budget)
    desc = (f"FP64 C oracle (radix-2) on {threads} threads; per step fwd+inv of min(batch, 2^{budget.bit_length() - 1}"
            f"/N) transforms of each size N<=2^{budget.bit_length() - 1}"
            + (f", plus one transform of one of the {nlarge} larger sizes in turn" if nlarge else ""))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": sweep_config(args, world),
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def fma_ceiling():
    """Measured FP32 FMA rate of the GPU (the library's probe kernel: 16
    independent chains per thread, 8 CTAs of 256 threads per SM), timed alone
    outside the sweep's timed region.  Context for the butterflies' arithmetic,
    which the HBM roofline does not cover."""
    import torch
    from paper_1203_4938_b300 import fft as F
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = sms * 8, 1 << 14
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    for _ in range(3):
        F.fma_probe(blocks, iters, out)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, flops = F.fma_probe(blocks, iters, out)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    if not bool((out == 120.0 + 16.0 * iters).all()):
        raise RuntimeError("FMA probe returned wrong values")
    return flops / best / 1e12



def run_gpu(args):
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    F.load()
    stream = torch.cuda.current_stream(dev)
    sizes = inputs.sweep_sizes(TOTAL_LOG2, args.lo, args.hi)
    if args.quick:
        sizes = [(k, n, max(1, b // 16)) for k, n, b in sizes]

    # inputs resident in HBM; one output and one scratch buffer shared by all sizes
    plans, xs = [], []
    for k, n, b in sizes:
        x = inputs.sweep_input(k, TOTAL_LOG2, seed=1)[:b]
        xs.append(torch.from_numpy(x).to(dev))
        plans.append(F.Plan((n,), b))
    maxel = max(n * b for _, n, b in sizes)
    y = torch.empty(maxel, dtype=torch.complex64, device=dev)
    z = torch.empty(maxel, dtype=torch.complex64, device=dev)

    launches = []  # (size index, direction, kernel index)
    for i, p in enumerate(plans):
        for d in (-1, +1):
            for kk in range(p.kernel_count):
                launches.append((i, d, kk))

    def step(events=None):
        j = 0
        for i, p in enumerate(plans):
            n, b = sizes[i][1], sizes[i][2]
            yy, zz = y[:n * b].view(b, n), z[:n * b].view(b, n)
            for d, src, dst in ((-1, xs[i], yy), (+1, yy, zz)):
                for kk in range(p.kernel_count):
                    if events is not None:
                        events[j][0].record(stream)
                    p.exec_kernel(kk, src, dst, d)
                    if events is not None:
                        events[j][1].record(stream)
                    j += 1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in launches] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dev)

    # per-kernel durations inside the timed region
    per = {}
    for s in range(args.steps):
        for j, (i, d, kk) in enumerate(launches):
            dt = ev[s][j][0].elapsed_time(ev[s][j][1])
            per.setdefault((i, kk), []).append(dt)
    tot = {key: sum(v) for key, v in per.items()}
    dom = max(tot, key=tot.get)
    di, dk = dom
    dn, db = sizes[di][1], sizes[di][2]
    avg_ms = statistics.mean(per[dom])
    alg_bytes = 16.0 * dn * db  # each kernel reads and writes every element once
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6400.0))
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    share = tot[dom] / sum(tot.values())

    fl = sum(2 * 5.0 * n * b * k for k, n, b in sizes)
    value = job_throughput(fl, world, ms)
    fma_tflops = fma_ceiling()

    # end to end through the public API: pinned host input -> device, fwd+inv,
    # result -> host.  The copies run on their own streams, double-buffered,
    # so size i+1's input crosses the host link while size i transforms and
    # size i-1's result comes back (the link carries both directions at once).
    e2e = None
    if not args.no_e2e:
        hin = [torch.empty(xs[i].shape, dtype=torch.complex64, pin_memory=True) for i in range(len(sizes))]
        for i in range(len(sizes)):
            hin[i].copy_(xs[i].cpu())
        hout = [torch.empty(maxel, dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        xin = [torch.empty(maxel, dtype=torch.complex64, device=dev) for _ in range(2)]
        zout = [torch.empty(maxel, dtype=torch.complex64, device=dev) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        in_free, out_free = [None, None], [None, None]
        turn = [0]

        def e2e_step():
            for i, p in enumerate(plans):
                n, b = sizes[i][1], sizes[i][2]
                k = turn[0] % 2
                turn[0] += 1
                xi, yy, zk = xin[k][:n * b].view(b, n), y[:n * b].view(b, n), zout[k][:n * b].view(b, n)
                with torch.cuda.stream(s_in):
                    if in_free[k] is not None:
                        s_in.wait_event(in_free[k])
                    xi.copy_(hin[i], non_blocking=True)
                    ready = torch.cuda.Event()
                    ready.record(s_in)
                stream.wait_event(ready)
                if out_free[k] is not None:
                    stream.wait_event(out_free[k])
                p.exec(xi, yy, -1, stream=stream)
                in_free[k] = torch.cuda.Event()
                in_free[k].record(stream)
                p.exec(yy, zk, +1, stream=stream)
                done = torch.cuda.Event()
                done.record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(done)
                    hout[k][:n * b].view(b, n).copy_(zk, non_blocking=True)
                    out_free[k] = torch.cuda.Event()
                    out_free[k].record(s_out)

        def drain():
            for ev in out_free:
                if ev is not None:
                    stream.wait_event(ev)

        e2e_step()
        drain()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        drain()
        a1.record(stream)
        torch.cuda.synchronize()
        ems = a0.elapsed_time(a1) / args.steps
        # the last size's result really came back: compare it with a device copy
        nl, bl = sizes[-1][1], sizes[-1][2]
        kl = (turn[0] - 1) % 2
        if not torch.equal(hout[kl][:nl * bl].to(dev), zout[kl][:nl * bl]):
            raise RuntimeError("end-to-end result on the host differs from the device result")
        bytes_io = sum(8 * n * b for _, n, b in sizes)
        e2e = {"value": world * fl / (ems * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ems,
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
               "overlap": "copies on two side streams, double-buffered, overlapping the transforms"}

    configs = None
    if rank == 0 and not args.no_configs:
        configs = run_config_keys(args, peak, OracleLeg(not args.no_cpu))
    if world > 1:
        dist.barrier()

    cpu = None
    if rank == 0 and not args.no_cpu:
        gf, secs, threads, desc = oracle_sample(1 << 19 if args.quick else 1 << 21)
        gf1, secs1, _, desc1 = oracle_sample(1 << 15 if args.quick else 1 << 16, threads=1)
        cpu = {"value": gf, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": secs, "one_core": {"value": gf1, "unit": "GFLOP/s", "cores": 1, "sample": desc1,
                                             "seconds": secs1}}

    if rank == 0:
        kname = plans[di].describe()
        traffic = measured_traffic(int(math.log2(dn)), kname) if db << int(math.log2(dn)) == 1 << TOTAL_LOG2 else None
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": sweep_config(args, world),
            "gpu_launches": args.steps * len(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)",
                         "algorithmic_bytes": alg_bytes,
                         "kernel": f"size N=2^{int(math.log2(dn))} kernel #{dk} of [{kname}]",
                         "kernel_time_share": share, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"
                         if "hbm_gbs" in peaks else "fallback 6.4 TB/s"},
            "clocks": clocks,
            "alu_context": {"fp32_fma_tflops_measured": fma_tflops,
                            "sweep_nominal_tflops": value / 1e3, "nominal_frac": value / 1e3 / fma_tflops,
                            "note": "nominal 5N log2 N flops per transform against the measured FP32 FMA "
                                    "rate (probe kernel); the sweep is bounded by HBM, not by this"},
            "per_size_plan": {f"2^{sizes[i][0]}": plans[i].describe() for i in range(len(sizes))},
            "per_size_ms": {f"2^{sizes[i][0]}": sum(statistics.mean(per[(i, kk)]) for kk in
                                                   range(plans[i].kernel_count)) * 2 for i in range(len(sizes))},
        }
        if e2e:
            line["e2e"] = e2e
        if configs:
            line["configs"] = configs
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    if world > 1:
        dist.destroy_process_group()


def _time_stream(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    for _ in range(steps):
        fn()
    a1.record()
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / steps


def _rel_rows(y, ref):
    """Per-row relative L2 distance of y from ref (FP64), along the last axis."""
    y = np.asarray(y, np.complex128)
    ref = np.asarray(ref, np.complex128)
    return np.sqrt(np.sum(np.abs(y - ref) ** 2, -1)) / np.sqrt(np.sum(np.abs(ref) ** 2, -1))


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    i = 2
    while i * i <= n:
        if n % i == 0:
            return False
        i += 1
    return True


class OracleLeg:
    """The CPU-baseline leg's oracle runs beside the other workloads: each
    config's sample is transformed by the FP64 oracle on the host cores (its
    time is that config's CPU baseline) and the GPU result of the same
    transforms is compared with it (relative L2, max over the sample).
    Disabled with --no-cpu, in which case no oracle code runs."""

    def __init__(self, enabled: bool):
        self.enabled = enabled
        self.oracle = None
        if enabled:
            import oracle
            oracle.build()
            self.oracle = oracle

    def run(self, fn):
        """(result, seconds) of fn(oracle), or (None, None) when disabled."""
        if not self.enabled:
            return None, None
        t0 = time.perf_counter()
        r = fn(self.oracle)
        return r, time.perf_counter() - t0


def _ragged_errors(orc, lengths, offsets, data, y, sign):
    """Max per-transform relative L2 error of the ragged result y: the full
    oracle FFT for composite lengths, the definition for primes up to 4096
    points, 24 bins of the definition for longer primes."""
    groups = {}
    for t, n in enumerate(lengths):
        groups.setdefault(int(n), []).append(t)
    worst, sampled = 0.0, 0
    for n, ts in groups.items():
        xs = np.stack([data[offsets[t]:offsets[t + 1]] for t in ts])
        ys = np.stack([y[offsets[t]:offsets[t + 1]] for t in ts])
        if _is_prime(n) and n > 4096:
            ks = np.unique(np.concatenate([[0, 1, n - 1, n // 2], np.random.default_rng(n).integers(0, n, 20)]))
            for j in range(len(ts)):
                vals = orc.dft_bins(xs[j], ks, sign)
                worst = max(worst, float(np.linalg.norm(ys[j][ks] - vals) / np.linalg.norm(vals)))
                sampled += 1
            continue
        ref = orc.dft_naive(xs, sign) if _is_prime(n) else orc.fft(xs, sign)
        worst = max(worst, float(_rel_rows(ys, ref).max()))
    return worst, sampled


def run_config_keys(args, peak: float, leg: OracleLeg) -> dict:
    """The other four workloads, each timed on the GPU (CUDA events on the
    current stream, inputs resident in HBM) and, through the CPU-baseline leg,
    compared with the FP64 oracle:
      small      N=1024 x 64, uniform[-1,1] seed 0, forward (1000 execs per
                 CUDA graph replay: launch-latency bound), every transform;
      image2d    1 x 4096^2 and 16 x 2048^2 image-shaped, seed 2, forward then
                 inverse; oracle on the 4096^2 image and two 2048^2 images,
                 round trip on all;
      precision  4096 x 4096 and 256 x 65536, normal(0,1) seed 3, forward, in
                 every mode (FP32 and the four tensor-core modes); oracle on
                 the first, middle and last transforms;
      ragged     10,000 uneven lengths, seed 4, forward and inverse, one
                 persistent graph launch vs launches per (stage, length);
                 oracle on every transform."""
    import torch
    from paper_1203_4938_b300 import fft as F
    steps, warm = max(3, min(args.steps, 10)), 3
    out = {}

    def hbm(bytes_, ms):
        gbs = bytes_ / (ms * 1e-3) / 1e9
        return {"algorithmic_gbs": gbs, "roofline_frac": gbs / peak}

    # --- small
    n, bt, reps = 1024, 64, 1000
    xh = inputs.uniform_batch(bt, n, seed=0)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    with F.Plan((n,), bt) as p:
        p.forward(x, y)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            p.forward(x, y)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                for _ in range(reps):
                    p.forward(x, y)
        ms = _time_stream(g.replay, 3, 2) / reps
        p.forward(x, y)
        torch.cuda.synchronize()
        p.check()
        yh = y.cpu().numpy()
        plan = p.describe()
    ref, secs = leg.run(lambda o: o.fft(xh, -1))
    out["small"] = {"workload": "N=1024 x 64 forward, uniform[-1,1] seed 0", "us_per_exec": ms * 1e3,
                    "gflops": 5.0 * n * math.log2(n) * bt / (ms * 1e-3) / 1e9, **hbm(16.0 * n * bt, ms),
                    "note": "launch-latency bound (graph replay of 1000 execs); 1 MiB per exec stays in L2",
                    "rel_l2_vs_oracle_max": None if ref is None else float(_rel_rows(yh, ref).max()),
                    "oracle_sample": "all 64 transforms", "oracle_seconds": secs, "plan": plan}
    del x, y

    # --- image2d
    a, b = inputs.image_workload(seed=2)
    parts = {}
    for name, arr, samp in (("4096x4096", a, [0]), ("16x2048x2048", b, [0, 15])):
        bt, h, w = arr.shape
        x = torch.from_numpy(arr).cuda()
        y, z = torch.empty_like(x), torch.empty_like(x)
        with F.Plan((h, w), bt) as p:
            def step():
                p.forward(x, y)
                p.inverse(y, z)
            ms = _time_stream(step, steps, warm)
            step()
            torch.cuda.synchronize()
            p.check()
            plan = p.describe()
        ys = y[samp].cpu().numpy().reshape(len(samp), -1)
        rt = (z.reshape(bt, -1) / (h * w) - x.reshape(bt, -1)).norm(dim=-1) / x.reshape(bt, -1).norm(dim=-1)
        ref, secs = leg.run(lambda o: o.fft2(arr[samp], -1).reshape(len(samp), -1))
        part = {"ms_fwd_inv": ms, "gflops": 2 * bt * 5.0 * h * w * math.log2(h * w) / (ms * 1e-3) / 1e9,
                **hbm(2 * 16.0 * bt * h * w, ms), "round_trip_rel_l2_max": float(rt.max().item()), "plan": plan,
                "oracle_sample": f"forward of image(s) {samp}", "oracle_seconds": secs}
        if ref is not None:
            part["rel_l2_vs_oracle_max"] = float(_rel_rows(ys, ref).max())
            ref_nodc, ys_nodc = ref.copy(), ys.copy()
            ref_nodc[:, 0] = 0
            ys_nodc[:, 0] = 0
            part["rel_l2_vs_oracle_max_without_dc"] = float(_rel_rows(ys_nodc, ref_nodc).max())
        parts[name] = part
        del x, y, z
    tot_ms = sum(v["ms_fwd_inv"] for v in parts.values())
    tot_gf = sum(v["gflops"] * v["ms_fwd_inv"] for v in parts.values()) / tot_ms
    out["image2d"] = {"workload": "1x4096^2 + 16x2048^2 image-shaped, seed 2, forward + inverse",
                      "ms_fwd_inv": tot_ms, "gflops": tot_gf, "parts": parts}

    # --- precision
    parts = {}
    for n, bt in ((4096, 4096), (65536, 256)):
        xh = inputs.normal_batch(bt, n, seed=3)
        samp = [0, bt // 2, bt - 1]
        x = torch.from_numpy(xh).cuda()
        y = torch.empty_like(x)
        ref, secs = leg.run(lambda o: o.fft(xh[samp], -1))
        for mode in ("fp32", "tc_fp16", "tc_bf16", "tc_fp16_plain", "tc_bf16_plain"):
            with F.Plan((n,), bt, mode) as p:
                ms = _time_stream(lambda: p.forward(x, y), steps, warm)
                p.forward(x, y)
                torch.cuda.synchronize()
                p.check()
                yh = y[samp].cpu().numpy()
                parts[f"{bt}x{n} {mode}"] = {
                    "us": ms * 1e3, "gflops": bt * 5.0 * n * math.log2(n) / (ms * 1e-3) / 1e9,
                    **hbm(16.0 * bt * n, ms), "plan": p.describe(),
                    "rel_l2_vs_oracle_max": None if ref is None else float(_rel_rows(yh, ref).max())}
        parts[f"{bt}x{n} oracle"] = {"oracle_sample": "transforms 0, B/2, B-1", "oracle_seconds": secs}
        del x, y
    out["precision"] = {"workload": "4096x4096 and 256x65536, normal(0,1) seed 3, forward", "parts": parts}

    # --- ragged
    lengths, offsets, data = inputs.ragged_workload(10000, seed=4)
    lens = [int(v) for v in lengths]
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    fl = sum(5.0 * n * math.log2(n) for n in lens if n > 1)
    with F.Ragged(lens) as p:
        ms_p = _time_stream(lambda: p.exec(x, y), steps, warm)
        ms_s = _time_stream(lambda: p.exec_per_size(x, y), steps, warm)
        errs, secs_tot = {}, 0.0
        for sign in (-1, +1):
            p.exec(x, y, sign)
            torch.cuda.synchronize()
            p.check()
            if leg.enabled:
                yh = y.cpu().numpy()
                r, secs = leg.run(lambda o: _ragged_errors(o, lens, offsets, data, yh, sign))
                errs["forward" if sign < 0 else "inverse"] = r[0]
                secs_tot += secs
        plan = p.describe()
    out["ragged"] = {"workload": "10,000 lengths (2^6..2^16, 3/5/7*2^k, ~1% primes), seed 4, forward",
                     "elements": int(offsets[-1]), "ms_persistent_graph": ms_p, "ms_per_size_launches": ms_s,
                     "gflops": fl / (ms_p * 1e-3) / 1e9, "gflops_per_size_launches": fl / (ms_s * 1e-3) / 1e9,
                     "persistent_over_per_size": ms_s / ms_p, **hbm(16.0 * offsets[-1], ms_p), "plan": plan,
                     "rel_l2_vs_oracle_max": errs or None,
                     "oracle_sample": "all 10,000 transforms (24 bins for primes above 4096)",
                     "oracle_seconds": secs_tot if leg.enabled else None}
    del x, y
    torch.cuda.synchronize()
    return out


def run_ragged(args):
    """Ragged batch: 10,000 1-D transforms, lengths log-uniform over 2^6..2^16
    mixed with 3/5/7 * 2^k and ~1 % primes (seed 4), forward; the single
    persistent graph-captured launch against one launch per (stage, length)."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    lengths, offsets, data = inputs.ragged_workload(args.count, seed=4)
    lens = [int(v) for v in lengths]
    if not args.no_tune:
        os.environ["FFT_AUTOTUNE"] = "1"  # measured tile shapes per length
    t0 = time.perf_counter()
    p = F.Ragged(lens)
    plan_s = time.perf_counter() - t0
    os.environ.pop("FFT_AUTOTUNE", None)
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    fl = sum(5.0 * n * math.log2(n) for n in lens if n > 1)
    ms_p = _time_stream(lambda: p.exec(x, y), args.steps, args.warmup)
    ms_s = _time_stream(lambda: p.exec_per_size(x, y), args.steps, args.warmup)
    ngroups = None
    line = {"metric": "ragged C2C FFT GFLOP/s (5N*log2N/t), 10,000 uneven lengths",
            "value": fl / (ms_p * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_p, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"ragged count={args.count} seed 4, forward",
                                            "elements": int(offsets[-1]), "plan": p.describe(),
                                            "autotuned": not args.no_tune, "plan_seconds": plan_s},
            "per_size_launches": {"value": fl / (ms_s * 1e-3) / 1e9, "ms_per_step": ms_s},
            "persistent_over_per_size": ms_s / ms_p,
            "effective_gbs": 16.0 * offsets[-1] / (ms_p * 1e-3) / 1e9}
    del ngroups
    print(json.dumps(line), flush=True)
    p.close()


def run_image2d(args):
    """Image-shaped 2-D transforms: one 4096x4096 and 16 x 2048x2048, real
    part uint8-range integers plus a smooth sinusoid, forward then inverse."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    a, b = inputs.image_workload(seed=2)
    res = {}
    for name, arr in (("4096x4096", a), ("16x2048x2048", b)):
        bt, h, w = arr.shape
        p = F.Plan((h, w), bt)
        x = torch.from_numpy(arr).cuda()
        y = torch.empty_like(x)
        z = torch.empty_like(x)

        def step():
            p.forward(x, y)
            p.inverse(y, z)

        ms = _time_stream(step, args.steps, args.warmup)
        fl = 2 * bt * 5.0 * h * w * math.log2(h * w)
        res[name] = {"ms_fwd_inv": ms, "gflops": fl / (ms * 1e-3) / 1e9,
                     "effective_gbs_per_direction": 16.0 * bt * h * w / (ms / 2 * 1e-3) / 1e9,
                     "plan": p.describe()}
        p.close()
    tot_ms = sum(v["ms_fwd_inv"] for v in res.values())
    tot_fl = sum(v["gflops"] * v["ms_fwd_inv"] for v in res.values())
    line = {"metric": "2-D C2C FFT GFLOP/s (5HW*log2(HW)/t), fwd+inv", "value": tot_fl / tot_ms, "unit": "GFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1x4096^2 + 16x2048^2 image-shaped, seed 2"}, "parts": res}
    print(json.dumps(line), flush=True)


def run_image_steps(args):
    """Image example steps 1-3 (Sec. III-B), fused: RGB -> YCbCr, chroma 2x2
    means, directional derivative of Y along (1, 1)/sqrt(2); RGB images of
    the 2-D workload's shapes (one 4096^2, 16 x 2048^2), seed 2.  HBM bytes
    per pixel: 3 in, 4 (Y) + 4 (derivative) + 2 (Cb, Cr at a quarter) out."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    a, b = inputs.rgb_workload(seed=2)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6400.0))
    u = 1.0 / math.sqrt(2.0)
    devs = [(name, torch.from_numpy(arr).cuda()) for name, arr in (("4096x4096", a), ("16x2048x2048", b))]
    outs = {name: (torch.empty(x.shape[:3], device="cuda"), torch.empty((x.shape[0], x.shape[1] // 2, x.shape[2] // 2),
                                                                      device="cuda"),
                   torch.empty((x.shape[0], x.shape[1] // 2, x.shape[2] // 2), device="cuda"),
                   torch.empty(x.shape[:3], device="cuda")) for name, x in devs}
    parts, tot_ms, tot_px = {}, 0.0, 0
    for name, x in devs:
        px = x.shape[0] * x.shape[1] * x.shape[2]
        ms = _time_stream(lambda: F.image_steps(x, u, u, outs[name]), args.steps, args.warmup)
        parts[name] = {"ms": ms, "mpix_per_s": px / (ms * 1e-3) / 1e6, "effective_gbs": 13.0 * px / (ms * 1e-3) / 1e9}
        tot_ms += ms
        tot_px += px
    achieved = 13.0 * tot_px / (tot_ms * 1e-3) / 1e9
    # end to end: pinned host RGB -> device, kernel, all four outputs -> pinned host
    hin = [torch.from_numpy(arr).pin_memory() for arr in (a, b)]
    hout = {name: tuple(torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs[name]) for name, _ in devs}

    def e2e_step():
        for (name, x), h in zip(devs, hin):
            x.copy_(h, non_blocking=True)
            F.image_steps(x, u, u, outs[name])
            for t, ht in zip(outs[name], hout[name]):
                ht.copy_(t, non_blocking=True)

    ems = _time_stream(e2e_step, max(1, args.steps // 4), 1)
    line = {"metric": "image steps 1-3 (YCbCr, chroma 2x2, directional derivative) Mpixel/s",
            "value": tot_px / (tot_ms * 1e-3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "RGB 1x4096^2 + 16x2048^2, seed 2", "direction": "(1,1)/sqrt(2)"},
            "gpu_launches": args.steps * len(devs),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_bytes_per_pixel": 13,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                         else "fallback 6.4 TB/s"},
            "e2e": {"value": tot_px / (ems * 1e-3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ems,
                    "h2d_bytes_per_step": 3 * tot_px, "d2h_bytes_per_step": 10 * tot_px},
            "parts": parts}
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Precision forms: batch 4096 x N=4096 and 256 x N=65536, normal(0,1)
    seed 3; FP32 Stockham vs tensor-core radix-16 (FP16/BF16, hi+lo and
    plain), forward; time, and each tensor-core mode's relative L2 distance
    from the FP32 path on sampled transforms (the FP32 path itself is within
    ~2e-7 of the FP64 oracle; every mode's error against the oracle on these
    same inputs is asserted in the tests)."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    parts = {}
    for n, bt in ((4096, 4096), (65536, 256)):
        xh = inputs.normal_batch(bt, n, seed=3)
        x = torch.from_numpy(xh).cuda()
        y = torch.empty_like(x)
        sample = [0, bt // 2, bt - 1]
        ref = None
        for mode in ("fp32", "tc_fp16", "tc_bf16", "tc_fp16_plain", "tc_bf16_plain"):
            p = F.Plan((n,), bt, mode)
            ms = _time_stream(lambda: p.forward(x, y), args.steps, args.warmup)
            p.check()
            yh = y[sample].cpu().numpy().astype(np.complex128)
            if ref is None:
                ref = yh
            d = np.sqrt(np.sum(np.abs(yh - ref) ** 2, -1)) / np.sqrt(np.sum(np.abs(ref) ** 2, -1))
            parts[f"{bt}x{n} {mode}"] = {"us": ms * 1e3, "gflops": bt * 5.0 * n * math.log2(n) / (ms * 1e-3) / 1e9,
                                         "effective_gbs": 16.0 * bt * n / (ms * 1e-3) / 1e9,
                                         "rel_l2_vs_fp32_max": float(d.max()), "plan": p.describe()}
            p.close()
    line = {"metric": "precision forms: us per forward exec and rel-L2 distance from the FP32 path", "unit": "us",
            "config": {"workload": "4096x4096 and 256x65536, normal(0,1) seed 3"}, "parts": parts,
            "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)


def run_real_conv(args):
    """Real transforms and convolution: R2C then C2R of 2^27 real floats
    (512 MiB) at N = 2^12, 2^16, 2^20, and FFT convolution of 2^14 signals of
    4096 with one filter (forward, spectrum product, inverse); inputs normal(0,1)
    from numpy seed 5."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    parts = {}
    rng = np.random.default_rng(5)
    for lg in (12, 16, 20):
        n = 1 << lg
        bt = (1 << 27) // n
        x = torch.from_numpy(rng.standard_normal((bt, n), dtype=np.float32)).cuda()
        p = F.RealPlan(n, bt)
        X = torch.empty((bt, n // 2 + 1), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        ms_f = _time_stream(lambda: p.forward(x, X), args.steps, args.warmup)
        ms_i = _time_stream(lambda: p.inverse(X, y), args.steps, args.warmup)
        # real input 4 B + half-spectrum output 8 B per (n/2+1) bins
        byts = 4.0 * bt * n + 8.0 * bt * (n // 2 + 1)
        parts[f"r2c N=2^{lg} x {bt}"] = {"us_fwd": ms_f * 1e3, "us_inv": ms_i * 1e3,
                                          "gflops_fwd": bt * 2.5 * n * lg / (ms_f * 1e-3) / 1e9,
                                          "effective_gbs_fwd": byts / (ms_f * 1e-3) / 1e9, "plan": p.describe()}
        p.close()
        del x, X, y
    n, bt = 4096, 1 << 14
    xs = torch.from_numpy(inputs.normal_batch(bt, n, seed=5)).cuda()
    h = torch.from_numpy(inputs.normal_batch(1, n, seed=6)[0]).cuda()
    px, ph = F.Plan((n,), bt), F.Plan((n,), 1)
    H = ph.forward(h.reshape(1, n))
    Xs = torch.empty_like(xs)
    out = torch.empty_like(xs)

    def conv():
        px.forward(xs, Xs)
        F.fft_spectrum_product(Xs.data_ptr(), H.data_ptr(), Xs.data_ptr(), n, bt, 1.0 / n, False,
                               torch.cuda.current_stream().cuda_stream)
        px.inverse(Xs, out)

    ms = _time_stream(conv, args.steps, args.warmup)
    parts[f"conv 1-D {bt} x {n} (three calls)"] = {"us": ms * 1e3,
                                                  "effective_gbs_3_passes": 3 * 16.0 * bt * n / (ms * 1e-3) / 1e9}

    def conv_one_call():
        F.fft_convolve(px.handle, xs.data_ptr(), H.data_ptr(), out.data_ptr(), 1.0 / n, False,
                       torch.cuda.current_stream().cuda_stream)

    ms1 = _time_stream(conv_one_call, args.steps, args.warmup)
    parts[f"conv 1-D {bt} x {n} (fft_convolve)"] = {"us": ms1 * 1e3,
                                                    "effective_gbs": 16.0 * bt * n / (ms1 * 1e-3) / 1e9}
    px.close()
    ph.close()
    print(json.dumps({"metric": "real transforms and FFT convolution", "parts": parts, "steps": args.steps,
                      "warmup": args.warmup, "config": {"workload": "r2c/c2r 2^27 floats; conv 2^14 x 4096"}}),
          flush=True)


def run_small(args):
    """The small parity case (N = 1024, batch 64, uniform[-1, 1] from seed 0,
    512 KiB, forward; its oracle parity is in the tests and smoke()), timed
    as back-to-back launches on a stream and as 1000 execs replayed from one
    CUDA graph (the case is bound by launch latency, not by HBM).  The line
    carries the round-trip error inverse(forward(x)) / N against x."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    n, batch, reps = 1024, 64, 1000
    xh = inputs.uniform_batch(batch, n, seed=0)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    with F.Plan((n,), batch) as p:
        z = p.inverse(p.forward(x, y)) / n
        torch.cuda.synchronize()
        p.check()
        err = float((torch.linalg.vector_norm(z - x, dim=-1) / torch.linalg.vector_norm(x, dim=-1)).max().item())
        stream_ms = _time_stream(lambda: p.forward(x, y), max(reps, args.steps), args.warmup)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            p.forward(x, y)  # warm-up on the capture stream
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                for _ in range(reps):
                    p.forward(x, y)
        graph_ms = _time_stream(g.replay, max(1, args.steps // 10), args.warmup) / reps
        p.check()
    fl = 5.0 * n * math.log2(n) * batch
    line = {"workload": "small", "metric": "C2C FFT GFLOP/s (5N*log2N/t), N=1024 x 64 forward", "unit": "GFLOP/s",
            "value": fl / (graph_ms * 1e-3) / 1e9, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "us_per_exec_graph": graph_ms * 1e3, "us_per_exec_stream": stream_ms * 1e3,
            "gflops_stream": fl / (stream_ms * 1e-3) / 1e9, "round_trip_rel_l2_max": err,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "N=1024, batch 64, uniform[-1,1] seed 0 (512 KiB), forward; "
                                   f"{reps} execs per CUDA graph replay; L2-resident (no flush)"},
            "plan": "rows N=2^10"}
    print(json.dumps(line), flush=True)


def run_case(args):
    """One plan run `steps` times (the small cases profiled with ncu):
    --case 1d|2d|ragged, --n (length, 2-D side, or ragged count), --batch,
    --precision.  Input: normal(0,1) complex64 from torch's generator (1d,
    2d) or the ragged workload (seed 4)."""
    import torch
    from paper_1203_4938_b300 import build as B
    from paper_1203_4938_b300 import fft as F
    B.build()
    if args.case == "ragged":
        lengths, _, data = inputs.ragged_workload(args.n, seed=4)
        p = F.Ragged([int(v) for v in lengths])
        x = torch.from_numpy(data).cuda()
    else:
        shape = (args.n, args.n) if args.case == "2d" else (args.n,)
        p = F.Plan(shape, args.batch, args.precision)
        x = torch.randn(p.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    ms = _time_stream(lambda: p.forward(x, y), max(1, args.steps), args.warmup)
    p.check()
    print(json.dumps({"case": args.case, "n": args.n, "batch": args.batch, "precision": args.precision,
                      "plan": p.describe(), "ms_per_exec": ms,
                      "effective_gbs": 16.0 * x.numel() / (ms * 1e-3) / 1e9}), flush=True)
    p.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "ragged", "image2d", "imagesteps", "precision", "realconv", "case", "small"])
    ap.add_argument("--case", default="1d", choices=["1d", "2d", "ragged"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--count", type=int, default=10000)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lo", type=int, default=LO)
    ap.add_argument("--hi", type=int, default=HI)
    ap.add_argument("--quick", action="store_true", help="1/16 of the batch (smoke runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="sweep only (no small/image2d/precision/ragged keys)")
    ap.add_argument("--no-tune", action="store_true", help="ragged: planner defaults instead of measured tiles")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged":
        run_ragged(args)
    elif args.workload == "image2d":
        run_image2d(args)
    elif args.workload == "imagesteps":
        run_image_steps(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "case":
        run_case(args)
    elif args.workload == "small":
        run_small(args)
    elif args.workload == "realconv":
        run_real_conv(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
