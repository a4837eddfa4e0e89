#!/usr/bin/env python
"""GEMM throughput on GB300: C = 1.5 * A @ B + 0.5 * C at M = N = K = 8192.

One step is one pass of the whole GEMM path through the C ABI: the BF16
hi/lo split of A and of B, then the tensor-core 3xBF16 GEMM with its
alpha/beta epilogue (or the selected --mode).  Inputs are seeded synthetic
FP32 matrices, U[-1, 1] (A, B and the initial C), resident in HBM before
timing; each of A, B, C is 268 MB, larger than the 129 MB L2, so no flush is
needed between steps.

Prints ONE JSON line (rank 0).  `value` is effective TFLOP/s = 2MNK / t
summed over all ranks; `e2e` is the same metric through gemm_from_host
(pinned host buffers, copies inside the timed region); `roofline` rates the
tensor-core kernel against the measured dense BF16 peak; `cpu_baseline` is
the FP64 CPU oracle timed on the host cores on sampled rows; `compare`
holds the FP32 SIMT kernel's throughput on the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode bf16x3]
    python bench.py --impl reference     # the CPU oracle arm
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GEMM TFLOP/s & % of peak at 8192^3: 3xBF16 TC vs FP32 SIMT, err<=1e-6"
ALPHA, BETA = 1.5, 0.5
SEED = 0x5EED


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="bf16x3", choices=["bf16x3", "bf16", "f32_simt"])
    p.add_argument("--size", type=int, default=8192)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-compare", action="store_true", help="skip the FP32 SIMT comparison")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--operand-layout", default="auto", choices=["auto", "as_stored", "k_major"],
                   help="auto: library choice; as_stored: operands stored K x rows are split "
                        "without transposing and read as MN-major tiles; k_major: every operand "
                        "made K-contiguous first")
    p.add_argument("--split-place", default="auto",
                   choices=["auto", "prepass", "in_kernel", "in_kernel_a", "in_kernel_b"],
                   help="3xBF16: where FP32 operands are split into hi/lo BF16 -- library "
                        "choice, a split pass before the kernel, or inside the kernel")
    p.add_argument("--shape", type=int, nargs=3, metavar=("M", "N", "K"),
                   default=[128, 8192, 8192], help="--workload shape: the GEMM's M N K")
    p.add_argument("--inputs", default="fp32", choices=["fp32", "bf16"],
                   help="--workload shape: FP32 operands through gemm() in --mode, or BF16 "
                        "operands through gemm_bf16")
    p.add_argument("--workload", default="square",
                   choices=["square", "rect", "grouped", "chain", "syr2k", "sweep", "shape"],
                   help="square: the 8192^3 headline; rect: BF16-input rectangular shapes; "
                        "grouped: 512 uneven problems; chain: Y = X W forward + backward; "
                        "syr2k: the rank-2k update of Section 5.1 at N = K = --size; "
                        "sweep: sizes 1024..8192 x transposes x distributions x modes; "
                        "shape: one NN GEMM of --shape M N K (alpha 1, beta 0), e.g. for a "
                        "profiler")
    return p.parse_args()


def load_traffic():
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu
    summary, or None once the kernel sources differ from the captured ones."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", "tc_gemm_bf16x3_8192_dram_traffic.md")
    src = [os.path.join(ROOT, "paper_2305_18236_gb300", "csrc", f) for f in ("tc_gemm.cu", "ptx.cuh")]
    try:
        text = open(prof).read()
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in src)).hexdigest()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("traffic_bytes_per_launch: ", "source_sha256: ")))
    if fields.get("source_sha256", "").strip() != h:
        return None
    return int(fields["traffic_bytes_per_launch"])


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- clocks
_REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the
    driver): SM clock, maximum SM clock, power draw and clock-event reasons
    of one GPU, found by UUID.  Nothing is set."""

    def __init__(self, uuid):
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        if not uuid or self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev)) != 0:
            raise OSError("no NVML handle for %s" % uuid)
        v = ctypes.c_uint()
        self.max_mhz = (float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(
            self.dev, 1, ctypes.byref(v)) == 0 else None)

    class _Field(ctypes.Structure):
        # nvmlFieldValue_t: field id, scope id, timestamp, latency, value
        # type, return code, 8-byte value union
        _fields_ = [("fieldId", ctypes.c_uint), ("scopeId", ctypes.c_uint),
                    ("timestamp", ctypes.c_longlong), ("latencyUsec", ctypes.c_longlong),
                    ("valueType", ctypes.c_int), ("nvmlReturn", ctypes.c_int),
                    ("value", ctypes.c_ulonglong)]

    POWER_INSTANT = 186  # NVML_FI_DEV_POWER_INSTANT (milliwatts, unsigned int)

    def sample(self):
        ct = self.ct
        mhz, r = ct.c_uint(), ct.c_ulonglong()
        ok = self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ct.byref(mhz)) == 0
        rs = self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.dev, ct.byref(r)) == 0
        f = self._Field(fieldId=self.POWER_INSTANT)
        watts = None
        if self.lib.nvmlDeviceGetFieldValues(self.dev, 1, ct.byref(f)) == 0 and f.nvmlReturn == 0:
            watts = (f.value & 0xFFFFFFFF) / 1000.0
        else:
            mw = ct.c_uint()
            if self.lib.nvmlDeviceGetPowerUsage(self.dev, ct.byref(mw)) == 0:
                watts = mw.value / 1000.0
        return (float(mhz.value) if ok else None, watts, int(r.value) if rs else 0)

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clock, power and clock-event reasons DURING a timed region.

    In-process NVML sampling every `period_s` (2 ms) on a background thread;
    where NVML is unavailable, nvidia-smi at its 100 ms floor.  Every sample
    is taken between start() (called just before the region's first launch)
    and stop() (called after its final synchronise), while the GPU works
    through the queued steps, so all samples count as under load."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid, period_s=0.002):
        self.uuid = uuid
        self.period = period_s
        self.nvml = None
        self.proc = None
        self.path = None
        self.thread = None
        self.rows = []
        try:
            self.nvml = _Nvml(uuid)
        except (OSError, AttributeError):
            self.nvml = None

    def start(self):
        self.rows = []
        if self.nvml is not None:
            import threading

            self._stop = threading.Event()

            def run():
                while not self._stop.is_set():
                    self.rows.append(self.nvml.sample())
                    self._stop.wait(self.period)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.nvml is not None and self.thread is not None:
            self._stop.set()
            self.thread.join()
            self.thread = None
            rows = self.rows
            if not rows:
                return None
            mhz = [r[0] for r in rows if r[0] is not None]
            watts = [r[1] for r in rows if r[1] is not None]
            reasons = sorted({name for r in rows for bit, name in _REASON_BITS.items()
                              if r[2] & bit})
            return {"sm_mhz": statistics.median(mhz) if mhz else None,
                    "sm_mhz_min": min(mhz) if mhz else None,
                    "sm_mhz_max": max(mhz) if mhz else None,
                    "sm_max_mhz": self.nvml.max_mhz, "reasons": reasons,
                    "power_w_median": statistics.median(watts) if watts else None,
                    "power_w_max": max(watts) if watts else None,
                    "samples": len(rows), "samples_under_load": len(rows),
                    "source": "NVML in-process, every %g ms" % (1e3 * self.period)}
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and parts[0] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        maxmhz = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        # samples taken while the GPU was busy (the clocks that matter)
        busy = [float(r[1]) for r in rows
                if r[3].replace(".", "").isdigit() and float(r[3]) > 250.0] or mhz
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": maxmhz,
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(busy),
                "source": "nvidia-smi every 100 ms"}


def median_ci(xs):
    """Median of a sample with its distribution-free 95 % confidence interval:
    the order statistics of (1-based) ranks floor(n/2 - 0.98 sqrt(n)) + 1 and
    ceil(n/2 + 0.98 sqrt(n)), the normal approximation of the binomial count
    of samples below the median (n = 20 gives ranks 6 and 15)."""
    import math

    x = sorted(xs)
    n = len(x)
    if n == 0:
        return None
    lo = max(0, int(math.floor(n / 2.0 - 0.98 * math.sqrt(n))))
    hi = min(n - 1, int(math.ceil(n / 2.0 + 0.98 * math.sqrt(n))) - 1)
    return {"median": statistics.median(x), "ci95": [x[lo], x[hi]], "mean": sum(x) / n,
            "min": x[0], "max": x[-1], "n": n}


# --------------------------------------------------------------- helpers
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """The largest of the ranks' values (the slowest replica's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_replicas(world, record):
    """Every rank's record, in rank order (each replica's device and time)."""
    if world == 1:
        return [record]
    import torch.distributed as dist

    out = [None] * world
    dist.all_gather_object(out, record)
    return out


def replica_tflops(flops_per_step, steps, ms_max, world):
    """Whole-job throughput of `world` independent replicas: every rank did
    `steps` steps of `flops_per_step` in at most `ms_max` milliseconds."""
    return world * flops_per_step * steps / (ms_max / 1e3) / 1e12


def square_config(n, mode, world, layout=None, split_place=None):
    """The workload description shared by both arms of the headline line."""
    cfg = {"workload": "sgemm %dx%dx%d NN alpha=1.5 beta=0.5, A,B,C0 U[-1,1] seeded"
                       % (n, n, n),
           "mode": mode, "M": n, "N": n, "K": n, "parallelism": "replicas x%d" % world,
           "l2": "inputs larger than L2 (A, B, C 268 MB each); no flush"}
    if layout is not None:
        cfg["operand_layout"] = layout
    if split_place is not None:
        cfg["split_place"] = split_place
    return cfg


def make_inputs(n):
    from paper_2305_18236_gb300 import inputs

    A = inputs.uniform((n, n), SEED)
    B = inputs.uniform((n, n), SEED + 1)
    C0 = inputs.uniform((n, n), SEED + 2)
    return A, B, C0


def time_steps(fn, steps, warmup, world, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    time_steps.per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[steps])


# --------------------------------------------------------------- CPU oracle
def oracle_rows_timed(A, B, C0, n, seconds, max_rows=4096):
    """Time the FP64 oracle on evenly spaced rows of the workload, sized to
    take about `seconds`.  Returns (rows, C64, D, elapsed, threads)."""
    import numpy as np

    import oracle

    probe = np.linspace(0, n - 1, 4).astype(np.int64)
    t0 = time.perf_counter()
    oracle.gemm(A, B, ALPHA, BETA, C0, rows=probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    nrows = int(max(8, min(max_rows, seconds / max(per_row, 1e-6))))
    rows = np.linspace(0, n - 1, nrows).astype(np.int64)
    t0 = time.perf_counter()
    C64, D, threads = oracle.gemm(A, B, ALPHA, BETA, C0, rows=rows)
    el = time.perf_counter() - t0
    return rows, C64, D, el, threads


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, each step a
    bounded sample of rows of the same 8192^3 workload."""
    import numpy as np

    import oracle

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.size
    A, B, C0 = make_inputs(n)
    probe = np.linspace(0, n - 1, 4).astype(np.int64)
    t0 = time.perf_counter()
    _, _, threads = oracle.gemm(A, B, ALPHA, BETA, C0, rows=probe)
    per_row = (time.perf_counter() - t0) / 4
    budget = 150.0 / max(1, args.steps + args.warmup)
    rows_per_step = int(max(1, min(256, budget / max(per_row, 1e-6))))
    times = []
    for s in range(args.warmup + args.steps):
        rows = (np.arange(rows_per_step) * 7919 + s * 104729) % n
        t0 = time.perf_counter()
        oracle.gemm(A, B, ALPHA, BETA, C0, rows=rows)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times)
    flops = 2.0 * rows_per_step * n * n * args.steps
    value = flops / t / 1e12
    sample = "%d rows x %d cols x K=%d per step (FP64 triple loop, C and |A||B| sums)" % (
        rows_per_step, n, n)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": square_config(n, args.mode, world, args.operand_layout, args.split_place),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    uuid = "GPU-" + str(props.uuid) if hasattr(props, "uuid") else None
    n = args.size
    M = N = K = n
    A, B, C0 = make_inputs(n)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    dC = torch.from_numpy(C0).to(dev)
    h = g.Gemm(dev)
    h.set_config(operand_layout=args.operand_layout, split_place=args.split_place)
    stream = torch.cuda.current_stream(dev)
    mode = args.mode
    mcode = g.MODES[mode]
    h.ensure_workspace(h.workspace_size(mcode, 0, 0, M, N, K))

    def step(md=mcode):
        st = h.gemm(0, 0, M, N, K, ALPHA, dA.data_ptr(), n, dB.data_ptr(), n, BETA,
                    dC.data_ptr(), n, md)
        if st != 0:
            raise RuntimeError("gemm failed: %d" % st)

    # launches per step, from the library's own count
    step()
    torch.cuda.synchronize()
    launches_per_step = h.last_launch_count()

    sampler = ClockSampler(uuid)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    h.lib.gemm_profile_enable(h.h, 1)
    sampler.start()
    ms = time_steps(step, args.steps, 0, world, stream)
    clocks = sampler.stop()
    step_stats = median_ci(time_steps.per_step)
    kern = (ctypes.c_float * args.steps)()
    main_n = ctypes.c_int()
    h.lib.gemm_profile_read_each(h.h, kern, args.steps, ctypes.byref(main_n))
    h.lib.gemm_profile_enable(h.h, 0)
    kern_stats = median_ci(list(kern)[:min(args.steps, main_n.value)])
    if h.sync() != 0:
        raise RuntimeError("kernel reported a bounded-wait timeout")
    ms_max = max_over_ranks(ms, world)
    flops = 2.0 * M * N * K
    value = replica_tflops(flops, args.steps, ms_max, world)
    kernel_ms = kern_stats["mean"] if kern_stats else float("nan")

    peaks, peak_src = load_peaks()
    # A timed region under a second is a burst: the kernel is rated against
    # the burst peak; a seconds-long region settles under the power cap and
    # is rated against the sustained one.
    region_s = ms / 1e3
    sustained = region_s >= 1.0
    sms = props.multi_processor_count
    if mode == "f32_simt":
        peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (kernel_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "%d SMs x 128 FP32 lanes x 2 x max clock" % sms}
    else:
        tensor_flops = flops * (3 if mode == "bf16x3" else 1)
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        peak = peaks.get(key, peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": tensor_flops / (kernel_ms / 1e3) / 1e12,
                "peak": peak, "unit": "TFLOP/s",
                "peak_source": "%s dense BF16 (cuBLAS, %s): the timed region lasted %.3f s"
                               % (peak_src, "sustained" if sustained else "burst", region_s)}
        mhz = clocks.get("sm_mhz") if clocks else None
        if mhz:
            # tensor work per SM per clock at the clock the kernel ran at,
            # against the dense rate of 4096 BF16 multiply-adds (8192 flops)
            # per SM per clock (one 128 x 256 x 16 MMA every 128 cycles)
            per_clk = tensor_flops / (kernel_ms / 1e3) / (mhz * 1e6) / sms
            roof["per_clock"] = {"flop_per_clk_per_sm": per_clk, "frac_of_8192": per_clk / 8192.0,
                                 "sm_mhz": mhz}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = load_traffic() if (mode == "bf16x3" and n == 8192) else None
    roof["kernel_ms"] = kernel_ms
    roof["kernel_ms_stats"] = kern_stats

    # FP32 SIMT comparison on the same workload: the two variants one call
    # at a time in randomised order (each timed with its own events), then
    # medians and 95 % intervals per variant
    compare = None
    if not args.no_compare and mode != "f32_simt":
        import random

        rounds = max(3, min(10, args.steps))
        h.ensure_workspace(h.workspace_size(g.MODES["f32_simt"], 0, 0, M, N, K))
        for _ in range(2):
            step(g.MODES["f32_simt"])
        torch.cuda.synchronize()
        order = [mode, "f32_simt"] * rounds
        random.Random(SEED).shuffle(order)
        evs = []
        simt_clocks = ClockSampler(uuid)
        simt_clocks.start()
        for md in order:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(g.MODES[md])
            e1.record(stream)
            evs.append((md, e0, e1))
        torch.cuda.synchronize()
        sclk = simt_clocks.stop()
        per = {mode: [], "f32_simt": []}
        for md, e0, e1 in evs:
            per[md].append(e0.elapsed_time(e1))
        simt_stats = median_ci(per["f32_simt"])
        ours_stats = median_ci(per[mode])
        ms_s = max_over_ranks(simt_stats["median"], world)
        simt = world * flops / (ms_s / 1e3) / 1e12
        compare = {"f32_simt_tflops": simt, "speedup_vs_f32_simt": value / simt,
                   "f32_simt_ms_per_step": ms_s, "order": "randomised, %d calls each" % rounds,
                   "f32_simt_ms_stats": simt_stats, "%s_ms_stats" % mode: ours_stats,
                   "speedup_of_medians": simt_stats["median"] / ours_stats["median"],
                   "clocks": sclk}
        if sclk and sclk.get("sm_mhz"):
            # FP32 peak at the clock the SIMT kernel actually ran at
            peak_at_clock = sms * 128 * 2 * sclk["sm_mhz"] * 1e6 / 1e12
            compare["f32_simt_frac_of_peak_at_clock"] = simt / world / peak_at_clock

    # end to end through the public API with pinned host buffers
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.from_numpy(C0.copy()).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    for _ in range(2):
        g.gemm_from_host(hA, hB, C=hC, alpha=ALPHA, beta=BETA, mode=mode, h=h)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.gemm_from_host(hA, hB, C=hC, alpha=ALPHA, beta=BETA, mode=mode, h=h)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * flops * e2e_steps / e2e_s / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": 3 * n * n * 4, "d2h_bytes_per_step": n * n * 4,
           "ms_per_step": 1000.0 * e2e_s / e2e_steps}
    del hA, hB, hC

    # CPU oracle baseline on sampled rows; the same rows give the error of a
    # fresh GEMM (C = 1.5 A B + 0.5 C0) at this size
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rows, C64, D, el, threads = oracle_rows_timed(A, B, C0, n, args.cpu_seconds)
        cpu = {"value": 2.0 * len(rows) * N * K / el / 1e12, "unit": "TFLOP/s",
               "cores": threads, "kind": "oracle",
               "sample": "%d evenly spaced rows of C (all %d columns, K=%d), FP64 triple loop"
                         % (len(rows), N, K)}
        # the same oracle on one thread (a few rows, about a second)
        import oracle

        one = rows[:: max(1, len(rows) // 8)][:8]
        t0 = time.perf_counter()
        oracle.gemm(A, B, ALPHA, BETA, C0, rows=one, threads=1)
        el1 = time.perf_counter() - t0
        cpu["single_thread"] = {"value": 2.0 * len(one) * N * K / el1 / 1e12, "cores": 1,
                                "sample": "%d of the same rows" % len(one)}
        import oracle

        errs = {}
        for md in ([mode] + (["f32_simt"] if mode != "f32_simt" else [])):
            dC.copy_(torch.from_numpy(C0))
            step(g.MODES[md])
            torch.cuda.synchronize()
            out = dC[torch.from_numpy(rows).to(dev)].cpu().numpy()
            errs[md] = oracle.normwise_error(out, C64, D)
        err = errs

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16x3 (bf16 hi/lo products, f32 accumulate)",
                  "bf16": "bf16 (f32 accumulate)", "f32_simt": "f32"}[mode],
        "data": "synthetic",
        "config": square_config(n, mode, world, args.operand_layout, args.split_place),
        "launches_per_step": launches_per_step,
        "step_ms_stats": step_stats,
        "roofline": roof,
        "gpu_launches": launches_per_step * args.steps,
        "e2e": e2e,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "compare": compare,
        "normwise_error": err,
        "peaks_source": peak_src,
    }
    if world > 1:  # which GPU each replica ran on (distinct UUIDs: distinct devices)
        line["replicas"] = gather_replicas(world, {"rank": rank, "local_rank": local,
                                                   "uuid": uuid, "ms": ms})
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# --------------------------------------------------------------- other workloads
def _events_ms(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_rect(args):
    """BF16-input rectangular/skinny GEMMs (FP32 accumulate and output),
    entries N(0, 1/sqrt(K)), alpha = 1, beta = 0, through gemm_bf16; and the
    3xBF16 mode through gemm() on FP32 copies of the same inputs."""
    import numpy as np
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g

    torch.cuda.set_device(0)
    peaks, src = load_peaks()
    stream = torch.cuda.current_stream()
    h = g.Gemm()
    h.set_config(operand_layout=args.operand_layout)
    out = []
    for (M, N, K) in [(16384, 4096, 1024), (4096, 16384, 4096), (128, 8192, 8192),
                      (8192, 8192, 64)]:
        gen = torch.Generator(device="cuda").manual_seed(SEED)
        A = (torch.randn((M, K), device="cuda", generator=gen) / np.sqrt(K)).to(torch.bfloat16)
        B = (torch.randn((K, N), device="cuda", generator=gen) / np.sqrt(K)).to(torch.bfloat16)
        Bt = B.t().contiguous()
        C = torch.empty((M, N), device="cuda")
        # NN: B stored K x N is read in place as MN-major tiles (as_stored), or
        # packed K-contiguous first (k_major); NT (B stored N x K) for comparison
        ms = _events_ms(lambda: g.matmul_bf16(A, B, C=C, h=h), args.steps, args.warmup, stream)
        launches = h.last_launch_count()
        ms_nt = _events_ms(lambda: g.matmul_bf16(A, Bt, C=C, transB=True, h=h), args.steps,
                           args.warmup, stream)
        flops = 2.0 * M * N * K
        nbytes = 2.0 * (M * K + N * K) + 4.0 * M * N
        row = {"M": M, "N": N, "K": K, "ms": ms, "tflops": flops / ms / 1e9,
               "gbs": nbytes / ms / 1e6,
               "frac_tensor": flops / ms / 1e9 / peaks["bf16_tflops"],
               "frac_hbm": nbytes / ms / 1e6 / peaks["hbm_gbs"],
               "launches": launches, "nt_ms": ms_nt}
        # the 3xBF16 leg: the same values as FP32 copies through gemm()
        # (split precision on FP32 operands); its bytes are the FP32 inputs
        # and the FP32 output, and sampled rows give its error
        A32, B32 = A.float(), B.float()
        ms3 = _events_ms(lambda: g.matmul(A32, B32, C=C, mode="bf16x3", h=h), args.steps,
                         args.warmup, stream)
        launches3 = h.last_launch_count()
        places = {}
        for place in ("prepass", "in_kernel", "in_kernel_a", "in_kernel_b"):
            hx = g.Gemm()
            hx.set_config(split_place=place)
            places[place] = _events_ms(lambda: g.matmul(A32, B32, C=C, mode="bf16x3", h=hx),
                                       args.steps, args.warmup, stream)
            hx.close()
        nbytes3 = 4.0 * (M * K + N * K + M * N)
        rows = np.linspace(0, M - 1, 4).astype(np.int64)
        g.matmul(A32, B32, C=C, mode="bf16x3", h=h)
        torch.cuda.synchronize()
        import oracle

        C64, D, _ = oracle.gemm(A32.cpu().numpy(), B32.cpu().numpy(), rows=rows)
        row["bf16x3"] = {"ms": ms3, "tflops": flops / ms3 / 1e9, "gbs": nbytes3 / ms3 / 1e6,
                         "frac_hbm": nbytes3 / ms3 / 1e6 / peaks["hbm_gbs"],
                         "frac_tensor_div3": 3 * flops / ms3 / 1e9 / peaks["bf16_tflops"],
                         "launches": launches3,
                         "ms_by_split_place": places,
                         "normwise_error": oracle.normwise_error(C[torch.from_numpy(rows).cuda()]
                                                                 .cpu().numpy(), C64, D)}
        out.append(row)
        del A, B, Bt, C, A32, B32
    h.close()
    tot_flops = sum(2.0 * r["M"] * r["N"] * r["K"] for r in out)
    tot_ms = sum(r["ms"] for r in out)
    print(json.dumps({"metric": "rectangular BF16-input GEMM TFLOP/s (sum over 4 shapes)",
                      "value": tot_flops / tot_ms / 1e9, "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": "bf16 in, f32 accumulate/out", "data": "synthetic",
                      "config": {"workload": "bf16 NN shapes, N(0,1/sqrt(K))",
                                 "operand_layout": args.operand_layout},
                      "shapes": out, "peaks_source": src}), flush=True)


def run_grouped(args):
    """512 problems, M, N, K uniform multiples of 32 in [64, 2048], FP32,
    3xBF16, alpha = 1, beta = 0: the library's plan (cost model) eager and
    graph-captured, one CTA per tile, the split pass or the in-kernel split
    forced, and the autotuned plan; then a five-problem straggler set whose
    long-K problems the plans split along K, against the set kept whole."""
    import numpy as np
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g

    torch.cuda.set_device(0)
    rng = np.random.default_rng(SEED)
    shapes = [tuple(int(x) * 32 for x in rng.integers(2, 65, size=3)) for _ in range(512)]
    probs = []
    for i, (M, N, K) in enumerate(shapes):
        gen = torch.Generator(device="cuda").manual_seed(SEED + i)
        probs.append(dict(A=torch.rand((M, K), device="cuda", generator=gen) * 2 - 1,
                          B=torch.rand((K, N), device="cuda", generator=gen) * 2 - 1,
                          C=torch.empty((M, N), device="cuda")))
    flops = sum(2.0 * M * N * K for (M, N, K) in shapes)
    stream = torch.cuda.Stream()
    h = g.Gemm()
    h.set_config(operand_layout=args.operand_layout)
    res = {}
    with torch.cuda.stream(stream):
        hp = g.Gemm()
        hp.set_config(operand_layout=args.operand_layout, cta_group=1)
        hf = g.Gemm()
        hf.set_config(operand_layout=args.operand_layout, split_place="in_kernel")
        hs = g.Gemm()
        hs.set_config(operand_layout=args.operand_layout, split_place="prepass")
        for name, kw, hh in [("model_eager", dict(), h), ("model_graph", dict(graph=True), h),
                             ("one_cta_graph", dict(graph=True), hp),
                             ("prepass_model_graph", dict(graph=True), hs),
                             ("in_kernel_graph", dict(graph=True), hf),
                             ("tuned_graph", dict(autotune=True, graph=True), h)]:
            t0 = time.perf_counter()
            plan = g.GroupedPlan(probs, mode=args.mode, h=hh, **kw)
            create_s = time.perf_counter() - t0
            ms = _events_ms(plan.run, args.steps, args.warmup, stream)
            res[name] = {"ms": ms, "tflops": flops / ms / 1e9, "config": plan.config(),
                         "plan_create_s": create_s}
            plan.close()
        hp.close()
        hf.close()
        hs.close()
        # a straggler set: three long-K problems with one or a few tiles among
        # small ones; the plans split them along K per problem (cost model or
        # autotuner) -- against the same set kept whole (handle split_k 1)
        st_shapes = [(128, 512, 8192), (64, 256, 4096), (256, 768, 6144), (96, 96, 64),
                     (64, 160, 96)]
        st_probs = []
        for i, (M, N, K) in enumerate(st_shapes):
            gen = torch.Generator(device="cuda").manual_seed(SEED + 1000 + i)
            st_probs.append(dict(A=torch.rand((M, K), device="cuda", generator=gen) * 2 - 1,
                                 B=torch.rand((K, N), device="cuda", generator=gen) * 2 - 1,
                                 C=torch.empty((M, N), device="cuda")))
        st_flops = sum(2.0 * M * N * K for (M, N, K) in st_shapes)
        hw = g.Gemm()
        hw.set_config(operand_layout=args.operand_layout, split_k=1)
        stragglers = {}
        for name, kw, hh in [("model_graph", dict(graph=True), h),
                             ("tuned_graph", dict(autotune=True, graph=True), h),
                             ("whole_graph", dict(graph=True), hw)]:
            plan = g.GroupedPlan(st_probs, mode=args.mode, h=hh, **kw)
            ms = _events_ms(plan.run, args.steps, args.warmup, stream)
            stragglers[name] = {"ms": ms, "tflops": st_flops / ms / 1e9,
                                "config": plan.config()}
            plan.close()
        hw.close()
    best = res["tuned_graph"]
    print(json.dumps({"metric": "grouped GEMM TFLOP/s, 512 problems (2MNK summed)",
                      "value": best["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"],
                      "higher_is_better": True, "dtype": args.mode, "data": "synthetic",
                      "config": {"workload": "512 problems, M,N,K ~ 32*U{2..64}, FP32 U[-1,1]",
                                 "flops_per_step": flops,
                                 "operand_layout": args.operand_layout},
                      "variants": res,
                      "straggler_set": {"shapes": st_shapes, "variants": stragglers}}),
          flush=True)


def run_chain(args):
    """Y = X W, loss = sum(Y * G), forward + backward through GemmFn:
    X 8192x4096, W 4096x4096, G 8192x4096, FP32 N(0, 1/sqrt(4096))."""
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g

    torch.cuda.set_device(0)
    gen = torch.Generator(device="cuda").manual_seed(SEED)
    X = (torch.randn((8192, 4096), device="cuda", generator=gen) / 64.0).requires_grad_(True)
    W = (torch.randn((4096, 4096), device="cuda", generator=gen) / 64.0).requires_grad_(True)
    G = torch.randn((8192, 4096), device="cuda", generator=gen) / 64.0

    def step():
        X.grad = None
        W.grad = None
        Y = g.GemmFn.apply(X, W, args.mode)
        Y.backward(G)

    ms = _events_ms(step, args.steps, args.warmup, torch.cuda.current_stream())
    flops = 3 * 2.0 * 8192 * 4096 * 4096
    print(json.dumps({"metric": "differentiable GEMM chain TFLOP/s (forward + backward)",
                      "value": flops / ms / 1e9, "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": args.mode, "data": "synthetic",
                      "config": {"workload": "X 8192x4096, W 4096x4096, dY = G; fwd + dX + dW"}}),
          flush=True)


def run_syr2k(args):
    """SYR2K (Section 5.1): lower triangle of C <- 1.5 (A B^T + B A^T) + 0.5 C,
    A, B FP32 N x K U[-1, 1], N = K = --size; the chosen mode against the
    FP32 SIMT variant, sampled rows against the FP64 oracle."""
    import ctypes

    import numpy as np
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g

    torch.cuda.set_device(0)
    n = args.size
    gen = torch.Generator(device="cuda").manual_seed(SEED)
    A = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    B = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    C0 = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    C = C0.clone()
    h = g.Gemm()
    h.set_config(operand_layout=args.operand_layout)
    stream = torch.cuda.current_stream()
    peaks, src = load_peaks()
    flops = 2.0 * n * n * n  # useful flops of one triangle: 2 N^2 K

    def timed(mode, steps, warmup):
        run = lambda: g.syr2k(A, B, C=C, alpha=ALPHA, beta=BETA, uplo="lower", mode=mode, h=h)
        run()
        torch.cuda.synchronize()
        launches = h.last_launch_count()
        h.lib.gemm_profile_enable(h.h, 1)
        ms = _events_ms(run, steps, warmup, stream)
        main_ms, main_n = ctypes.c_double(), ctypes.c_int()
        h.lib.gemm_profile_read(h.h, ctypes.byref(main_ms), ctypes.byref(main_n))
        h.lib.gemm_profile_enable(h.h, 0)
        return ms, main_ms.value / max(1, main_n.value), launches

    ms, kernel_ms, launches = timed(args.mode, args.steps, args.warmup)
    # tensor work of the kernel: every 128 x BN tile that meets the triangle,
    # in full, over both products (3 BF16 products each in the split mode)
    bn = 256
    tiles = sum(min(-(-n // bn), (128 * mt + 127) // bn + 1) for mt in range(-(-n // 128)))
    tensor_flops = tiles * 128 * bn * 2.0 * (2 * n) * (3 if args.mode == "bf16x3" else 1)
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    line = {"metric": "SYR2K TFLOP/s (2 N^2 K) at N = K = %d" % n, "value": flops / ms / 1e9,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": args.mode, "data": "synthetic",
            "config": {"workload": "syr2k lower, A,B %dx%d U[-1,1], alpha 1.5 beta 0.5" % (n, n),
                       "operand_layout": args.operand_layout},
            "launches_per_step": launches, "peaks_source": src}
    if args.mode != "f32_simt":
        line["roofline"] = {"bound": "tensor", "achieved": tensor_flops / kernel_ms / 1e9,
                            "peak": peak, "unit": "TFLOP/s", "frac": tensor_flops / kernel_ms / 1e9 / peak,
                            "kernel_ms": kernel_ms, "tiles": tiles}
    if not args.no_compare:
        sms, sk, _ = timed("f32_simt", max(2, args.steps // 10), 1)
        line["compare"] = {"f32_simt_ms": sms, "f32_simt_tflops": flops / sms / 1e9,
                           "speedup_vs_f32_simt": sms / ms}
    if not args.no_cpu:
        # CPU baseline: the FP64 oracle on sampled rows of the triangle; the
        # same rows give the error of a fresh GPU call
        C.copy_(C0)
        g.syr2k(A, B, C=C, alpha=ALPHA, beta=BETA, uplo="lower", mode=args.mode, h=h)
        torch.cuda.synchronize()
        import oracle

        rows = np.linspace(0, n - 1, 6).astype(np.int64)
        hA, hB, hC0 = A.cpu().numpy(), B.cpu().numpy(), C0.cpu().numpy()
        t0 = time.perf_counter()
        C64, D, used = oracle.syr2k(hA, hB, ALPHA, BETA, hC0, uplo="lower", rows=rows)
        cpu_s = time.perf_counter() - t0
        row_flops = sum(2.0 * 2 * (int(r) + 1) * n for r in rows)
        line["cpu_baseline"] = {"value": row_flops / cpu_s / 1e12, "unit": "TFLOP/s",
                                "cores": used, "kind": "oracle",
                                "sample": "%d evenly spaced rows of the lower triangle, FP64"
                                          % len(rows)}
        line["normwise_error"] = oracle.normwise_error(C.cpu().numpy()[rows], C64, D)
    h.close()
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """The square-size sweep: M = N = K in {1024, 2048, 4096, 8192} x {NN, NT,
    TN, TT} x {U[-1, 1], sign-random 2^U[-10, 10]} x every mode, alpha 1.5,
    beta 0.5, C0 U[-1, 1].  Each case is timed with CUDA events around each
    call (L2 flushed with a 256 MB write between calls for sizes <= 2048);
    its CPU baseline is the FP64 oracle on 8 sampled rows, which also gives
    the case's normwise error."""
    import numpy as np
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    import oracle
    from paper_2305_18236_gb300 import gemm as g
    from paper_2305_18236_gb300 import inputs

    torch.cuda.set_device(0)
    peaks, src = load_peaks()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    flush = torch.empty(256 << 18, device="cuda")  # 256 MB
    h = g.Gemm()
    cases = []
    for n in (1024, 2048, 4096, 8192):
        for dist in ("uniform", "log_uniform"):
            for tA, tB in ((False, False), (False, True), (True, False), (True, True)):
                A = inputs.make(dist, (n, n), SEED + n, k=n)
                B = inputs.make(dist, (n, n), SEED + n + 1, k=n)
                C0 = inputs.uniform((n, n), SEED + n + 2)
                rows = np.linspace(0, n - 1, 8).astype(np.int64)
                t0 = time.perf_counter()
                C64, D, used = oracle.gemm(A, B, ALPHA, BETA, C0, transA=tA, transB=tB, rows=rows)
                cpu_s = time.perf_counter() - t0
                dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
                dC0 = torch.from_numpy(C0).cuda()
                for mode in ("f32_simt", "bf16", "bf16x3"):
                    C = dC0.clone()
                    g.matmul(dA, dB, C=C, alpha=ALPHA, beta=BETA, transA=tA, transB=tB,
                             mode=mode, h=h)
                    torch.cuda.synchronize()
                    err = oracle.normwise_error(C.cpu().numpy()[rows], C64, D)
                    steps = max(2, args.steps // (1 if n <= 4096 else 4)) if mode != "f32_simt" \
                        else max(2, args.steps // (4 if n <= 4096 else 16))
                    times = []
                    for it in range(args.warmup + steps):
                        if n <= 2048:
                            flush.zero_()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        g.matmul(dA, dB, C=C, alpha=ALPHA, beta=BETA, transA=tA, transB=tB,
                                 mode=mode, h=h)
                        e1.record()
                        torch.cuda.synchronize()
                        if it >= args.warmup:
                            times.append(e0.elapsed_time(e1))
                    ms = statistics.median(times)
                    tflops = 2.0 * n ** 3 / ms / 1e9
                    peak = fp32_peak if mode == "f32_simt" else bf16_peak / (3 if mode == "bf16x3" else 1)
                    cases.append({"n": n, "trans": ("T" if tA else "N") + ("T" if tB else "N"),
                                  "dist": dist, "mode": mode, "ms": round(ms, 5),
                                  "tflops": round(tflops, 2), "pct_of_peak": round(100 * tflops / peak, 1),
                                  "normwise_error": err,
                                  "cpu_oracle_tflops": round(2.0 * len(rows) * n * n / cpu_s / 1e12, 5)})
                    print(json.dumps(cases[-1]), file=sys.stderr, flush=True)
                del dA, dB, dC0
    h.close()
    print(json.dumps({"metric": "square sweep: TFLOP/s and % of the mode's peak (FP32 SIMT: FP32 "
                                "peak; BF16: BF16 peak; 3xBF16: BF16 peak / 3)",
                      "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "M=N=K in {1024..8192} x 4 transposes x 2 "
                                             "distributions x 3 modes, alpha 1.5 beta 0.5",
                                 "l2": "flushed between calls for n <= 2048"},
                      "peaks": {"fp32_tflops": fp32_peak, "bf16_tflops": bf16_peak, "source": src},
                      "cpu_baseline": {"kind": "oracle", "sample": "8 evenly spaced rows per case",
                                       "cores": oracle.host_cores()},
                      "cases": cases}), flush=True)


def run_shape(args):
    """One NN GEMM of shape M x N x K, alpha = 1, beta = 0, N(0, 1/sqrt(K))
    operands: FP32 through gemm() in --mode (with --split-place), or BF16
    through gemm_bf16.  Times --steps back-to-back calls after --warmup and
    prints one JSON line (a small, self-contained case for ncu captures)."""
    import torch

    from paper_2305_18236_gb300 import build as pbuild

    pbuild.build()
    from paper_2305_18236_gb300 import gemm as g
    from paper_2305_18236_gb300 import inputs

    torch.cuda.set_device(0)
    M, N, K = args.shape
    peaks, src = load_peaks()
    A = torch.from_numpy(inputs.normal((M, K), SEED, 1.0 / K ** 0.5)).cuda()
    B = torch.from_numpy(inputs.normal((K, N), SEED + 1, 1.0 / K ** 0.5)).cuda()
    C = torch.empty((M, N), device="cuda")
    h = g.Gemm()
    h.set_config(operand_layout=args.operand_layout, split_place=args.split_place)
    if args.inputs == "bf16":
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
        call = lambda: g.matmul_bf16(A, B, C=C, h=h)
        nbytes = 2.0 * (M * K + K * N) + 4.0 * M * N
        mode = "bf16"
    else:
        call = lambda: g.matmul(A, B, C=C, mode=args.mode, h=h)
        nbytes = 4.0 * (M * K + K * N + M * N)
        mode = args.mode
    ms = _events_ms(call, args.steps, args.warmup, torch.cuda.current_stream())
    if h.sync() != 0:
        raise RuntimeError("kernel reported a bounded-wait timeout")
    flops = 2.0 * M * N * K
    print(json.dumps({"metric": "GEMM %dx%dx%d %s inputs, %s" % (M, N, K, args.inputs, mode),
                      "value": flops / ms / 1e9, "unit": "TFLOP/s", "ms": ms,
                      "gbs": nbytes / ms / 1e6, "frac_hbm": nbytes / ms / 1e6 / peaks["hbm_gbs"],
                      "launches": h.last_launch_count(), "steps": args.steps,
                      "warmup": args.warmup, "split_place": args.split_place,
                      "data": "synthetic", "peaks_source": src}), flush=True)
    h.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "rect":
        run_rect(args)
    elif args.workload == "grouped":
        run_grouped(args)
    elif args.workload == "chain":
        run_chain(args)
    elif args.workload == "syr2k":
        run_syr2k(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "shape":
        run_shape(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
