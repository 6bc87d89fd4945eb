"""Benchmark: integrand samples/s of batched multi-function direct Monte Carlo.

Default workload (N=1): the paper's GPU test (Eq. 1, Fig. 1) at its stated
size, 100 four-dimensional harmonics x 10^6 samples, with the paper's 10
independent evaluations (Philox keys 0..9) in one table: 10^9 samples per step.
One step = one pass of the whole path over that table: reset the work counter,
the persistent FP32 sampling launch over all (integrand, chunk) items, the FP64
merge.  Inputs (the precomputed descriptor table) are resident on the device
when the timed region starts.

Also reported on the same line: the plain form (one FP64 launch per integrand)
on the same table, the 10^4-integrand mixed table (batched and plain), the end-
to-end rate through zmc_integrate with host buffers, a short serving run
(p50/p99 job latency), the roofline of the dominant kernel and the FP64 oracle
on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2104_10073_gb300 import workloads as W  # noqa: E402

METRIC = "integrand samples/s (G/s) batched vs plain on 1 GB300; p50/p99 job latency"
UNIT = "Gsamples/s"
WORKLOAD = "fig1-harmonics-100x1e6-x10-repeats"

# Algorithmic 32-bit operations per sample of a d-dimensional harmonic (the
# dominant kernel of the default workload), counted from the minimal steps of
# the kernel's method: Philox4x32-10 = 10 rounds x (2 widening multiplies + 2
# three-way XORs) per block of five 23-bit coordinates -> 8 d, and the four shifts
# that split a block into its fields -> 0.8 d; per coordinate: 23-bit mask, the
# high-word phase multiply-add, the low-word FMA and the add of its bits -> 4 d;
# the phase carry, |x|, 1/4 - |x|, the integer -> float conversion and its scaling
# -> 5; t^2, the degree-4 polynomial in t^2 with the amplitude in its
# coefficients (4) and the product with t -> 6; shifted sums -> 3.
# Rows whose dimensions all advance the phase at the same rate (k_i (hi_i - lo_i)
# equal, d >= 2) take the equal-rate form: the 23-bit integers are summed
# (mask + add per coordinate -> 2 d) and the phase is one widening multiply-add
# and one multiply-add (2); then |x|, 1/4 - |x|, the conversion and its scaling
# (4).
def harmonic_ops_per_sample(d: int, equal_rates: bool = False) -> float:
    if equal_rates:
        return 8 * d + 0.8 * d + 2 * d + 2 + 4 + 6 + 3
    return 8 * d + 0.8 * d + 4 * d + 5 + 6 + 3


# Algorithmic work of a d-dimensional harmonic sample on the fmaheavy pipe (the
# pipe that executes integer multiplies), in 32-bit multiply-add lane-operations:
# a widening 32 x 32 -> 64 multiply counts 2 (it takes the pipe twice as long as
# a 32-bit one).  Philox: 16 widening multiplies per block once the products
# shared by a chunk are formed once, d / 5 blocks per sample -> 6.4 d; the
# fixed-point phase: one 32-bit multiply-add per coordinate -> d, or for the
# equal-rate form one widening and one 32-bit multiply-add -> 3.
def harmonic_heavy_ops_per_sample(d: int, equal_rates: bool = False) -> float:
    return 2 * 16 * d / 5 + (3 if equal_rates else d)


def equal_rate_rows(table) -> np.ndarray:
    """Harmonic rows the library evaluates in the equal-rate form: d >= 2 and
    k_i (hi_i - lo_i) identical in every dimension (exact equality implies the
    library's test, equal rates after rounding to 2^-41 turn)."""
    out = np.zeros(len(table), dtype=bool)
    for i, row in enumerate(table):
        d = int(row["dim"])
        if int(row["family"]) != W.HARMONIC or d < 2:
            continue
        rate = row["p"][2:2 + d] * (row["hi"][:d] - row["lo"][:d])
        out[i] = bool(np.all(rate == rate[0]))
    return out


def table_mean(table, fn) -> float:
    """Sample-weighted mean of fn(dim, equal_rates) over a table's rows."""
    n = table["n_samples"].astype(np.float64)
    eq = equal_rate_rows(table)
    per = np.array([fn(int(d), bool(e)) for d, e in zip(table["dim"], eq)])
    return float(np.sum(n * per) / np.sum(n))


# Sources of the dominant kernel (zmc_batched_kernel<HARMONIC>).
KERNEL_SOURCES = ["paper_2104_10073_gb300/csrc/zmc_fam_harmonic.cu",
                  "paper_2104_10073_gb300/csrc/zmc_device.cuh",
                  "paper_2104_10073_gb300/csrc/zmc_internal.h",
                  "paper_2104_10073_gb300/csrc/zmc_coeffs.h"]
PROFILE = os.path.join(ROOT, "profiles", "zmc_batched_harmonic_fig1x10.md")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_counters():
    """DRAM traffic and pipe utilisation of the dominant kernel from the committed
    ncu summary, only if it was taken from the current kernel source."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    start = text.find("```json")
    if start < 0:
        return None
    end = text.find("```", start + 7)
    prof = json.loads(text[start + 7:end])
    if prof.get("kernel_source_sha256") != kernel_source_hash():
        return None
    return prof


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml, by
    ctypes; read-only queries) every ``period`` seconds on a thread while the
    timed region runs: a ~50 ms region still gets dozens of samples."""

    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap"}

    def __init__(self, device: int, period: float = 0.001):
        import ctypes

        self.period = period
        self.samples = []
        self.stop_flag = threading.Event()
        self.thread = None
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.nv = nv
        self.h = ctypes.c_void_p()
        uuid = None
        try:
            import torch

            uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
        except Exception:  # noqa: BLE001 - older torch: fall back to the index
            uuid = None
        rc = 1
        if uuid:
            rc = nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device), ctypes.byref(self.h))
        if rc != 0:
            raise OSError("no NVML handle")
        self.get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        self.max_mhz = None
        if nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) == 0:
            self.max_mhz = float(v.value)

    def _read(self):
        import ctypes

        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            if (self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) == 0 and
                    self.get_reasons(self.h, ctypes.byref(rs)) == 0):
                self.samples.append((float(mhz.value), int(rs.value)))
            time.sleep(self.period)

    def start(self):
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag.set()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [m for m, _ in self.samples]
        reasons = sorted({nm for _, r in self.samples for bit, nm in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(sm), "sm_mhz_min": min(sm) if sm else None,
                "source": f"NVML every {1e3 * self.period:.0f} ms"}


def clock_sampler(device: int):
    """The NVML sampler where libnvidia-ml loads, else the nvidia-smi one."""
    try:
        return NvmlClockSampler(device)
    except (OSError, AttributeError):
        return ClockSampler(device)


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi -lms 100"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(world, v: float, op: str) -> float:
    """All-reduce one float over the ranks (NCCL on the GPU; gloo on the CPU when
    the process group runs gloo, as in the host-side tests)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(world, v: float) -> float:
    return _reduce(world, v, "max")


def sum_over_ranks(world, v: float) -> float:
    return _reduce(world, v, "sum")


def oracle_rate(rows, threads=0):
    """FP64 oracle samples/s over ``rows`` on the host cores."""
    import oracle

    t0 = time.perf_counter()
    _, used = oracle.integrate(rows, threads=threads)
    dt = time.perf_counter() - t0
    return W.total_samples(rows) / dt, used, dt


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (else the machine type)."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def fig1_table(rank: int):
    # weak scaling: rank r evaluates its own 10 repeats (keys 10r .. 10r+9)
    return W.harmonic_fig1(10**6, seeds=range(10 * rank, 10 * rank + 10))


def run_reference(args, world, rank):
    """The FP64 CPU oracle on the host cores, on a bounded sample of the workload."""
    if rank != 0:
        return
    sample = W.harmonic_fig1(10**5, seeds=[0])  # 100 integrands x 10^5 samples per step
    for _ in range(args.warmup):
        oracle_rate(sample)
    times = []
    used = 0
    for _ in range(args.steps):
        _, used, dt = oracle_rate(sample)
        times.append(dt)
    n = W.total_samples(sample)
    value = n * len(times) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "100 integrands x 1e5 samples per step",
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": "Fig. 1 harmonics, key 0, 100 x 1e5 samples per step",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_plan(zmc, torch, ctx, plan, steps, flush):
    """Device time per step and of the sampling stage, CUDA events on ctx.stream."""
    s = ctx.stream
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(s):
            flush.zero_()  # write > L2 between steps
        ev[k][0].record(s)
        zmc.zmc_plan_run(plan, zmc.ZMC_STAGE_SAMPLE)
        ev[k][1].record(s)
        zmc.zmc_plan_run(plan, zmc.ZMC_STAGE_MERGE)
        ev[k][2].record(s)
    s.synchronize()
    step = [ev[k][0].elapsed_time(ev[k][2]) for k in range(steps)]
    kern = [ev[k][0].elapsed_time(ev[k][1]) for k in range(steps)]
    return step, kern


def run_native(args, world, rank, local):
    import torch

    from paper_2104_10073_gb300 import build
    from paper_2104_10073_gb300 import zmc

    # one rank per node compiles (if the sources changed); the others wait
    if local == 0:
        build.build()
    barrier(world)
    torch.cuda.set_device(local)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))

    # CPU baseline first (host threads only; no process is forked after CUDA init)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        sample = W.harmonic_fig1(10**6, seeds=range(args.cpu_repeats))
        rate, used, dt = oracle_rate(sample)
        one = W.harmonic_fig1(10**5, seeds=[0])
        rate1, _, dt1 = oracle_rate(one, threads=1)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"Fig. 1 harmonics, keys 0..{args.cpu_repeats - 1}, "
                         f"{len(sample)} x 1e6 samples ({dt:.1f} s wall)",
               "cpu_model": cpu_model(),
               "one_core": {"value": rate1 / 1e9, "unit": UNIT,
                            "sample": f"Fig. 1 harmonics, key 0, 100 x 1e5 samples "
                                      f"({dt1:.1f} s wall)"}}

    import tempfile

    tune_path = os.path.join(tempfile.gettempdir(), f"zmc_tune_{os.getuid()}_{local}.json")
    # the autotuner picks the launch geometry, the chunk length and the unroll
    # (cached per GPU and table shape; --no-autotune: --quints-per-lane, unroll 1)
    tune = 0 if args.no_autotune else zmc.ZMC_TUNE_GEOMETRY | zmc.ZMC_TUNE_CHUNK
    ctx = zmc.Context(arena_bytes=2 << 30, device=local, autotune=tune,
                      tune_cache_path=tune_path, quints_per_lane=args.quints_per_lane)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    tab = fig1_table(rank)
    n_samples = W.total_samples(tab)
    plan = zmc.zmc_plan_create(ctx.handle, tab)
    info = zmc.zmc_plan_info_get(plan)
    for _ in range(max(args.warmup, 3)):
        zmc.zmc_plan_run(plan)
    ctx.stream.synchronize()

    clocks = clock_sampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    step_ms, kern_ms = time_plan(zmc, torch, ctx, plan, args.steps, flush)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = max_over_ranks(world, sum(step_ms) / len(step_ms))
    kms = sum(kern_ms) / len(kern_ms)
    total = sum_over_ranks(world, float(n_samples))
    value = total / (ms / 1e3) / 1e9
    res = zmc.zmc_plan_results(plan, len(tab))
    assert np.all(res["status"] == 0)

    # plain FP64 form, same table, one launch per integrand
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_ms = None
    if not args.skip_plain:
        plain_steps = max(1, min(args.steps, 3))
        zmc.zmc_plan_run_plain(plan)
        ctx.stream.synchronize()
        e0.record(ctx.stream)
        for _ in range(plain_steps):
            zmc.zmc_plan_run_plain(plan)
        e1.record(ctx.stream)
        ctx.stream.synchronize()
        plain_ms = e0.elapsed_time(e1) / plain_steps
    zmc.zmc_plan_destroy(plan)

    # the same FP32 sampling kernels launched one integrand at a time (a plan per
    # row, replayed as a graph): what batching itself gains, at equal arithmetic
    per_row_ms = None
    if not args.skip_plain and rank == 0:
        rows = [zmc.zmc_plan_create(ctx.handle, tab[i:i + 1]) for i in range(len(tab))]
        for pr in rows:
            zmc.zmc_plan_run(pr)
        ctx.stream.synchronize()
        e0.record(ctx.stream)
        for pr in rows:
            zmc.zmc_plan_run(pr)
        e1.record(ctx.stream)
        ctx.stream.synchronize()
        per_row_ms = e0.elapsed_time(e1)
        for pr in rows:
            zmc.zmc_plan_destroy(pr)

    # end to end through the public blocking call: host table in, host results out
    e2e_s = None
    if not args.skip_e2e:
        e2e_t = []
        for k in range(args.steps + 1):
            t0 = time.perf_counter()
            out = zmc.zmc_integrate(ctx.handle, tab)
            if k > 0:
                e2e_t.append(time.perf_counter() - t0)
        assert np.all(out["status"] == 0)
        e2e_s = max_over_ranks(world, sum(e2e_t) / len(e2e_t))

    # The same workload through the general harmonic form: the Fig. 1 wave
    # vectors are isotropic on the unit cube, so every dimension advances the
    # phase at the same rate and the library takes its cheaper equal-rate form;
    # stretching k_4 by 1e-9 (a phase change below 1e-8 rad) makes the rates
    # differ and shows what a general wave vector costs.
    general = None
    if rank == 0 and not args.skip_mixed:
        gt = tab.copy()
        gt["p"][:, 5] *= 1.0 + 1e-9
        general = batched_and_plain(zmc, torch, ctx, gt, flush,
                                    "fig1-harmonics-100x1e6-x10, k_4 x (1 + 1e-9)", 20, False)

    # the 10^4-integrand mix and the Eq. 2 abs-linear set (batched and plain),
    # rank 0 only
    mixed = eq2 = None
    if rank == 0 and not args.skip_mixed:
        mixed = batched_and_plain(zmc, torch, ctx, W.mixed(10**4), flush,
                                  "mixed-1e4-integrands-d1..7-logN4..7", 5, not args.skip_plain)
        eq2 = batched_and_plain(zmc, torch, ctx, W.abslin_eq2(10**6), flush,
                                "eq2-abslin-49x2d-51x3d-x1e6", 20, not args.skip_plain)

    # the generator alone: Philox4x32-10 blocks/s, the ceiling of any sampling
    # kernel (a 4-D sample draws 4/5 of a block); measured after the timed region
    generator = None
    if rank == 0:
        rate = zmc.zmc_philox_rate(ctx.handle, 1 << 35) / 1e9
        generator = {"philox_blocks_per_s": rate, "unit": "G blocks/s",
                     "ceiling_4d_samples_per_s": rate * 5 / 4,
                     "kernel": "zmc_philox_rate_kernel (2 x 256-thread blocks per SM)",
                     "harmonic_over_ceiling": n_samples / (kms / 1e3) / 1e9 / (rate * 5 / 4)}

    functional = checkpoint = udf = normal = None
    if rank == 0 and not args.skip_modes:
        functional = run_functional(zmc, ctx)
        checkpoint = run_checkpoint(zmc, local, ctx)
        udf = run_udf(zmc, ctx)
        udf["mixed"] = run_udf_mixed(zmc, ctx)
        normal = run_normal(zmc, ctx)

    serving = None
    if rank == 0 and not args.skip_serving:
        serving = run_serving(zmc, local, args.serving_rate, args.serving_seconds)
        if serving:
            serving.pop("_stream")
    ctx.close()

    if rank != 0:
        return
    # Roofline of the dominant kernel (the harmonic family's persistent launch).
    # The binding resource is the busiest pipe in the committed ncu summary of
    # this kernel source; achieved = the algorithmic work on that pipe per launch
    # / the launch's CUDA-event time.  The issue-slot figure (every algorithmic
    # operation against 1 instruction per scheduler per cycle) and the measured
    # generator ceiling are given beside it.
    sm_clock = peaks.get("sm_max_mhz", 2070.0)
    sms = info["sms"]
    sched_ghz = sms * 4 * sm_clock * 1e6 / 1e9  # schedulers x clock, G cycles/s
    ops_ps = table_mean(tab, harmonic_ops_per_sample)
    heavy_ps = table_mean(tab, harmonic_heavy_ops_per_sample)
    issue_peak = sched_ghz * 32  # G lane-instructions/s
    issue_ach = ops_ps * n_samples / (kms / 1e3) / 1e9
    heavy_peak = sched_ghz * 16  # G 32-bit multiply-add lane-ops/s (16 lanes per scheduler)
    heavy_ach = heavy_ps * n_samples / (kms / 1e3) / 1e9
    prof = profile_counters()
    pipes = prof["pipes"] if prof else None
    busiest = None
    if pipes:
        busiest = max((k for k in pipes if k != "issue_active"), key=lambda k: pipes[k])
    roofline = {
        "bound": busiest or "alu", "bound_class": "alu",
        "achieved": heavy_ach, "peak": heavy_peak,
        "unit": "G fmaheavy lane-ops/s (32-bit multiply-add = 1, widening = 2)",
        "frac": heavy_ach / heavy_peak,
        "traffic": prof["dram_bytes_per_launch"] if prof else None,
        "kernel": "zmc_batched_kernel<HARMONIC>", "kernel_ms": kms,
        "peak_basis": f"{sms} SMs x 4 schedulers x 16 lanes x {sm_clock:.0f} MHz (measured max)",
        "heavy_ops_per_sample": heavy_ps,
        "issue_slots": {"achieved": issue_ach, "peak": issue_peak, "unit": "G lane-op/s",
                        "frac": issue_ach / issue_peak, "ops_per_sample": ops_ps},
        "ncu_pipes": pipes,
        "ncu_profile": os.path.relpath(PROFILE, ROOT) if prof else "stale (kernel source changed)",
        "generator_ceiling_frac": generator["harmonic_over_ceiling"] if generator else None,
    }
    bop = None if plain_ms is None else plain_ms / (sum(step_ms) / len(step_ms))
    summary = {
        "batched_gsps": sig(value), "plain_fp64_gsps": sig(n_samples / (plain_ms / 1e3) / 1e9)
        if plain_ms else None, "batched_over_plain": sig(bop),
        "per_integrand_fp32_gsps": sig(n_samples / (per_row_ms / 1e3) / 1e9) if per_row_ms else None,
        "batching_alone_x": sig(per_row_ms / (sum(step_ms) / len(step_ms))) if per_row_ms else None,
        "e2e_gsps": sig(total / e2e_s / 1e9) if e2e_s else None,
        "fmaheavy_frac": sig(roofline["frac"], 3),
        "issue_frac": sig(roofline["issue_slots"]["frac"], 3),
    }
    if general:
        summary["fig1_general_phase_gsps"] = sig(general["batched_gsps"])
    for key, leg in (("mix1e4", mixed), ("eq2_abslin", eq2)):
        if leg:
            summary[key] = {"batched_gsps": sig(leg["batched_gsps"]),
                            "plain_fp64_gsps": sig(leg.get("plain_gsps")),
                            "batched_over_plain": sig(leg.get("batched_over_plain"))}
    if serving:
        summary["serving"] = {"jobs_per_s": serving["rate_jobs_per_s"],
                              "p50_ms": sig(serving["p50_ms"], 3), "p99_ms": sig(serving["p99_ms"], 3),
                              "gsps": sig(serving["samples_per_s"], 3)}
    # Long per-mode records first; the contract keys and the metric summary last,
    # so that a reader of the line's tail sees them.
    line = {
        "functional": functional, "checkpoint": checkpoint, "udf": udf, "normal": normal,
        "generator": generator,
        "plain": None if plain_ms is None else {
            "value": n_samples / (plain_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": plain_ms,
            "dtype": "f64", "form": "one FP64 kernel launch per integrand + merge"},
        "per_integrand_fp32": None if per_row_ms is None else {
            "value": n_samples / (per_row_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": per_row_ms,
            "form": "the batched FP32 kernels, one launch (graph) per integrand"},
        "fig1_general_phase": general, "mixed": mixed, "eq2_abslin": eq2, "serving": serving,
        "wall_s_timed": wall,
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "integrands": len(tab), "samples_per_step": n_samples,
                   "quints_per_lane": info["quints_per_lane"], "chunks": info["n_chunks"],
                   "unroll": info["family_unroll"][0],
                   "grid": info["family_grid"][0], "block": info["family_block"][0],
                   "autotune": ["default", "measured", "cached"][info["tune_source"][0]],
                   "chunk_tune": ["default", "measured", "cached"][info["chunk_tune_source"]],
                   "l2": "flushed between steps (256 MiB write, outside the timed events)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": None if e2e_s is None else {
            "value": total / e2e_s / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": len(tab) * W.DESC_DTYPE.itemsize,
            "d2h_bytes_per_step": len(tab) * 32,
            "path": "zmc_integrate (host table in, host results out)"},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "batched_over_plain": bop,
        "summary": summary,
    }
    print(json.dumps(line), flush=True)


def batched_and_plain(zmc, torch, ctx, table, flush, name, steps, plain):
    """Batched rate (median of ``steps`` device-timed plan replays, L2 flushed
    before each) and plain FP64 rate (one pass, one launch per integrand) of one
    table."""
    plan = zmc.zmc_plan_create(ctx.handle, table)
    zmc.zmc_plan_run(plan)
    ctx.stream.synchronize()
    st, _ = time_plan(zmc, torch, ctx, plan, steps, flush)
    ns = W.total_samples(table)
    out = {"workload": name, "integrands": len(table), "samples": ns,
           "batched_gsps": ns / (statistics.median(st) / 1e3) / 1e9,
           "batched_ms": statistics.median(st)}
    res = zmc.zmc_plan_results(plan, len(table))
    assert np.all(res["status"] == 0)
    pi = zmc.zmc_plan_info_get(plan)
    out["plan"] = {"quints_per_lane": pi["quints_per_lane"],
                   "unroll": list(pi["family_unroll"]),
                   "chunk_tune": {0: "default", 1: "measured", 2: "cached"}.get(
                       pi["chunk_tune_source"], pi["chunk_tune_source"])}
    if plain:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        zmc.zmc_plan_run_plain(plan)
        ctx.stream.synchronize()
        e0.record(ctx.stream)
        zmc.zmc_plan_run_plain(plan)
        e1.record(ctx.stream)
        ctx.stream.synchronize()
        pms = e0.elapsed_time(e1)
        out["plain_gsps"] = ns / (pms / 1e3) / 1e9
        out["plain_ms"] = pms
        out["batched_over_plain"] = out["batched_gsps"] / out["plain_gsps"]
    zmc.zmc_plan_destroy(plan)
    return out


def sig(x, digits=4):
    """x rounded to ``digits`` significant digits (None stays None)."""
    if x is None:
        return None
    return float(f"{x:.{digits}g}")


def run_serving(zmc, device, rate_hz, seconds, quints_per_lane=0, chunks_per_iter=0, share=0):
    """Poisson job stream through zmc_submit; a collector thread takes finished
    ids from zmc_poll_any and the results from zmc_poll.  Latency = submit call
    to results collected."""
    jobs = W.serving_stream(rate_hz, seconds, max_fns=1000)
    ctx = zmc.Context(arena_bytes=8 << 30, device=device, serving=True,
                      quints_per_lane=quints_per_lane, max_chunks_per_iter=chunks_per_iter,
                      serving_share=share)
    submitted = {}
    done = {}
    lock = threading.Lock()
    n_total = len(jobs)

    def collector():
        while len(done) < n_total:
            st, ids = zmc.zmc_poll_any(ctx.handle, 4096, 200)
            for jid in ids:
                with lock:
                    ts, n = submitted[jid]
                st2, _ = zmc.zmc_poll(ctx.handle, jid, n, wait_ms=0)
                if st2 == zmc.ZMC_OK:
                    done[jid] = time.perf_counter() - ts

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    samples = 0
    for at, tab in jobs:
        while time.perf_counter() - t0 < at:
            time.sleep(0.0002)
        ts = time.perf_counter()
        with lock:
            jid = zmc.zmc_submit(ctx.handle, tab)
            submitted[jid] = (ts, len(tab))
        samples += W.total_samples(tab)
    th.join()
    wall = time.perf_counter() - t0
    ctx.close()
    lat = sorted(done.values())
    if not lat:
        return None
    return {"rate_jobs_per_s": rate_hz, "jobs": len(lat), "seconds": wall,
            "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "samples_per_s": samples / wall / 1e9, "unit": "Gsamples/s",
            "_stream": [(at, W.total_samples(tab)) for at, tab in jobs]}


def fifo_bound(stream, capacity_gsps):
    """p50 / p99 latency of an ideal server on the same job stream: jobs served
    one at a time, oldest first, at capacity_gsps, with no launch granularity
    (a job's latency is its wait plus its samples / capacity)."""
    t, lat = 0.0, []
    for at, n in stream:
        t = max(t, at) + n / (capacity_gsps * 1e9)
        lat.append(t - at)
    lat.sort()
    return {"capacity_gsps": capacity_gsps, "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


def launch_model(jobs, capacity_gsps, chunk_samples=4160, budget_samples=2**31,
                 cut_backlog=2**34, fixed_s=52e-6, build_s=30e-6, slots=2):
    """p50 / p99 latency of a model of the serving loop on a job stream of
    (arrival_s, samples, chunks): each launch holds at most budget_samples'
    worth of chunks, filled oldest job first and ended at the first job it
    completes while fewer than cut_backlog samples are left to issue (the
    library's rule); a launch runs for fixed_s plus its samples at the kernels'
    rate, which is set so that full launches deliver capacity_gsps; at most
    `slots` launches are in flight, the next one built (build_s) as soon as a
    slot is free and work is waiting; a job completes when the launch with its
    last chunks ends.  It leaves out the merge, the copies and the host threads."""
    budget = max(1, budget_samples // chunk_samples)
    full_s = budget * chunk_samples / (capacity_gsps * 1e9)
    if full_s <= fixed_s:
        raise ValueError("a full launch must take longer than its fixed cost")
    rate = budget * chunk_samples / (full_s - fixed_s)  # samples/s
    n = len(jobs)
    rem = [c for _, _, c in jobs]
    per_chunk = [s / c if c else 0.0 for _, s, c in jobs]
    lat = [0.0] * n
    live, inflight = [], []  # inflight: (end_s, finished job indices), in order
    arrived, t, gpu_free = 0, 0.0, 0.0
    while True:
        while inflight and inflight[0][0] <= t:
            end, fin = inflight.pop(0)
            for j in fin:
                lat[j] = end - jobs[j][0]
        while arrived < n and jobs[arrived][0] <= t:
            if rem[arrived] == 0:
                lat[arrived] = 0.0
            else:
                live.append(arrived)
            arrived += 1
        if live and len(inflight) < slots:
            cut = sum(rem[j] * chunk_samples for j in live) < cut_backlog
            left, samples, fin, keep = budget, 0.0, [], []
            for j in live:
                if left == 0:
                    keep.append(j)
                    continue
                take = min(rem[j], left)
                rem[j] -= take
                left -= take
                samples += take * per_chunk[j]
                if rem[j] == 0:
                    fin.append(j)
                    if cut:
                        left = 0
                else:
                    keep.append(j)
            live = keep
            gpu_free = max(t + build_s, gpu_free) + fixed_s + samples / rate
            inflight.append((gpu_free, fin))
            continue
        nxt = [x for x in ((jobs[arrived][0] if arrived < n else None),
                           (inflight[0][0] if inflight else None)) if x is not None]
        if not nxt:
            break
        t = max(t, min(nxt))
    lat.sort()
    return {"capacity_gsps": capacity_gsps, "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]} if lat else None


def run_functional(zmc, ctx):
    """Functional mode: one 4-D harmonic over a 1000-point lattice of its wave
    vector (k_1 = k_2 = k_3 = k_4 = kappa, kappa from 8.1 to 23.9, the Fig. 1
    range), 10^6 samples per point, common random numbers; end to end through
    zmc_integrate_functional (lattice in from the host, results out)."""
    base = W.harmonic_fig1(10**6)[0]
    kappa = np.linspace(51.0 / (2 * np.pi), 150.0 / (2 * np.pi), 1000)
    values = np.repeat(kappa[:, None], 4, axis=1)
    slots = [zmc.slot_p(2 + i) for i in range(4)]
    zmc.zmc_integrate_functional(ctx.handle, base, slots, values, False)
    t = []
    for _ in range(5):
        t0 = time.perf_counter()
        out = zmc.zmc_integrate_functional(ctx.handle, base, slots, values, False)
        t.append(time.perf_counter() - t0)
    assert np.all(out["status"] == 0)
    sec = statistics.median(t)
    n = len(values) * 10**6
    return {"workload": "harmonic-4d-1000-kappa-points-x1e6-common-streams", "samples": n,
            "value": n / sec / 1e9, "unit": UNIT, "ms": 1e3 * sec,
            "path": "zmc_integrate_functional (host lattice in, host results out)"}


def run_checkpoint(zmc, device, ref_ctx):
    """Preemption of a serving job: 1000 Fig. 1 harmonics x 10^7 samples
    (10^10 samples) submitted, checkpointed after ~10 ms, resumed; reports the
    checkpoint call's latency, the time of the interrupted + resumed run against
    an uninterrupted one, and the largest difference of the final estimates from
    the uninterrupted run in units of their standard error."""
    tab = W.harmonic_fig1(10**7, seeds=range(10))
    ctx = zmc.Context(arena_bytes=2 << 30, device=device, serving=True)
    jid = zmc.zmc_submit(ctx.handle, tab)  # warm-up: graphs, pinned areas
    zmc.zmc_poll(ctx.handle, jid, len(tab), wait_ms=-1)
    t0 = time.perf_counter()
    jid = zmc.zmc_submit(ctx.handle, tab)
    st, whole = zmc.zmc_poll(ctx.handle, jid, len(tab), wait_ms=-1)
    t_whole = time.perf_counter() - t0
    t0 = time.perf_counter()
    jid = zmc.zmc_submit(ctx.handle, tab)
    time.sleep(0.010)
    tc = time.perf_counter()
    st, ck = zmc.zmc_checkpoint(ctx.handle, jid, len(tab), wait_ms=-1)
    t_ckpt = time.perf_counter() - tc
    if st != zmc.ZMC_OK:
        ctx.close()
        return {"status": int(st)}
    rid = zmc.zmc_submit_resume(ctx.handle, tab, ck)
    st, res = zmc.zmc_poll(ctx.handle, rid, len(tab), wait_ms=-1)
    t_both = time.perf_counter() - t0
    ctx.close()
    dev = np.abs(res["estimate"] - whole["estimate"]) / whole["stderr"]
    return {"workload": "fig1-harmonics-100x1e7-x10-keys-one-job", "samples": W.total_samples(tab),
            "checkpoint_ms": 1e3 * t_ckpt,
            "done_at_checkpoint": float(ck["n"].sum() / W.total_samples(tab)),
            "rows_partial_at_checkpoint": int(np.sum((ck["n"] > 0) & (ck["n"] < tab["n_samples"]))),
            "uninterrupted_ms": 1e3 * t_whole, "checkpoint_resume_ms": 1e3 * t_both,
            "max_abs_diff_in_stderr": float(dev.max())}


def run_udf_mixed(zmc, ctx):
    """The 10^4-integrand mix written as user code: one run-time compiled module
    of 28 functions (the four forms x dimensions 1..7; the polynomial degree in
    p[39]), every row selecting its function, one call; FP32 user arithmetic."""
    forms = {
        W.HARMONIC: "float ph = 0.0f;\n  for (int i = 0; i < ZMC_UDF_DIM; ++i) ph = fmaf(p[2 + i], x[i], ph);\n"
                    "  float s, c; sincosf(ph, &s, &c); return p[0] * c + p[1] * s;",
        W.ABSLIN: "float s = 0.0f;\n  for (int i = 0; i < ZMC_UDF_DIM; ++i) s = fmaf(p[1 + i], x[i], s);\n"
                  "  return p[0] * fabsf(s);",
        W.GAUSS: "float r2 = 0.0f;\n  for (int i = 0; i < ZMC_UDF_DIM; ++i) { float t = x[i] - p[2 + i]; r2 = fmaf(t, t, r2); }\n"
                 "  return p[0] * expf(-r2 / (2.0f * p[1] * p[1]));",
        W.POLY: "const int g = (int)p[39]; float prod = 1.0f;\n"
                "  for (int i = 0; i < ZMC_UDF_DIM; ++i) { float q = p[5 * i + 4];\n"
                "    for (int j = 3; j >= 0; --j) q = (j < g) ? fmaf(q, x[i], p[5 * i + j]) : (j == g ? p[5 * i + j] : q);\n"
                "    prod *= q; }\n  return prod;",
    }
    srcs, dims, index = [], [], {}
    for fam in (W.HARMONIC, W.ABSLIN, W.GAUSS, W.POLY):
        for d in range(1, 8):
            index[(fam, d)] = len(srcs)
            srcs.append("__device__ float zmc_user_f(const float *x, const float *p) {\n  "
                        + forms[fam] + "\n}\n")
            dims.append(d)
    t0 = time.perf_counter()
    u = zmc.Udf(srcs, dims, zmc.ZMC_UDF_F32, 0.0)
    compile_s = time.perf_counter() - t0
    tab = W.mixed(10**4)
    fam = tab["family"].copy()
    tab["p"][:, 39] = tab["deg"]
    tab["deg"] = [index[(int(f), int(d))] for f, d in zip(fam, tab["dim"])]
    tab["family"] = W.USER
    u.integrate(ctx.handle, tab)  # load + warm-up
    t = []
    for _ in range(3):
        t0 = time.perf_counter()
        res = u.integrate(ctx.handle, tab)
        t.append(time.perf_counter() - t0)
    assert np.all(res["status"] == 0)
    u.close()
    sec = statistics.median(t)
    n = W.total_samples(tab)
    return {"workload": "mixed-1e4-integrands as 28 user functions, one call", "samples": n,
            "value": n / sec / 1e9, "unit": UNIT, "ms": 1e3 * sec, "compile_s": compile_s,
            "path": "zmc_udf_integrate (host table in, host results out)"}


def run_udf(zmc, ctx):
    """User-defined integrands compiled at run time: the Fig. 1 x 10 table
    (10^9 samples) with Eq. 1 written as user code, FP32 (sincosf) and FP64
    (cos, sin), end to end through Udf.integrate; compile time reported apart."""
    tab = W.harmonic_fig1(10**6, seeds=range(10))
    tab["family"] = W.USER
    srcs = {
        "f32": ("__device__ float zmc_user_f(const float *x, const float *p) {\n"
                "  float ph = 0.0f;\n"
                "  for (int i = 0; i < ZMC_UDF_DIM; ++i) ph = fmaf(p[2 + i], x[i], ph);\n"
                "  float s, c; sincosf(ph, &s, &c); return p[0] * c + p[1] * s;\n}\n",
                zmc.ZMC_UDF_F32),
        "f64": ("__device__ double zmc_user_f(const double *x, const double *p) {\n"
                "  double ph = 0.0;\n"
                "  for (int i = 0; i < ZMC_UDF_DIM; ++i) ph = fma(p[2 + i], x[i], ph);\n"
                "  return p[0] * cos(ph) + p[1] * sin(ph);\n}\n", zmc.ZMC_UDF_F64),
    }
    out = {"workload": "fig1-harmonics-100x1e6-x10-repeats as user code", "samples": 10**9}
    for name, (src, prec) in srcs.items():
        t0 = time.perf_counter()
        u = zmc.Udf(src, 4, prec, amplitude=2.0)
        compile_s = time.perf_counter() - t0
        u.integrate(ctx.handle, tab)  # load + warm-up
        t = []
        for _ in range(3):
            t0 = time.perf_counter()
            res = u.integrate(ctx.handle, tab)
            t.append(time.perf_counter() - t0)
        assert np.all(res["status"] == 0)
        sec = statistics.median(t)
        out[name] = {"value": 1e9 / sec / 1e9, "unit": UNIT, "ms": 1e3 * sec,
                     "compile_s": compile_s}
        u.close()
    return out


def run_normal(zmc, ctx):
    """Stratified sampling with tree refinement (the paper's normal mode, for 8 to
    12 dimensions) on the case it is meant for, a localised integrand: a 10-D
    Gaussian peak (sigma 0.1 at (0.25, ..., 0.25)) as run-time compiled user code
    on [0, 1]^10; 2^10 level-0 cells x 2^14 samples, up to two refinement
    rounds; against plain direct MC with the same number of samples (one cell)."""
    src = ("__device__ float zmc_user_f(const float *x, const float *p) {\n"
           "  float r2 = 0.0f;\n"
           "  for (int i = 0; i < ZMC_UDF_DIM; ++i) r2 = fmaf(x[i] - p[0], x[i] - p[0], r2);\n"
           "  return expf(-r2 / (2.0f * p[1] * p[1]));\n}\n")
    u = zmc.Udf(src, 10, zmc.ZMC_UDF_F32, amplitude=1.0)
    lo, hi, p = np.zeros(10), np.ones(10), np.array([0.25, 0.1])
    opts = zmc.normal_options(divisions=2, depth=2, samples_per_cell=1 << 14, sigma_mult=3.0,
                              seed=1, max_leaves=8 << 10)
    u.normal_integrate(ctx.handle, lo, hi, p, opts)  # load + warm-up
    t0 = time.perf_counter()
    r = u.normal_integrate(ctx.handle, lo, hi, p, opts)
    sec = time.perf_counter() - t0
    plain = u.normal_integrate(ctx.handle, lo, hi, p, zmc.normal_options(
        divisions=1, depth=0, samples_per_cell=r["n_samples"], seed=1, stream_base=1 << 20))
    u.close()
    return {"workload": "gauss-peak-10d-user-code, 2^10 cells x 2^14, depth 2",
            "value": r["n_samples"] / sec / 1e9, "unit": UNIT, "ms": 1e3 * sec,
            "samples": r["n_samples"], "cells": r["n_cells"], "leaves": r["n_leaves"],
            "rounds": r["rounds"], "estimate": r["estimate"], "stderr": r["stderr"],
            "plain_estimate": plain["estimate"], "plain_stderr": plain["stderr"],
            "variance_reduction": (plain["stderr"] / r["stderr"]) ** 2}


def run_serving_sweep(args):
    """p50/p99 job latency and throughput over a sweep of Poisson arrival rates
    (rank 0, one GPU); one JSON object on stdout."""
    from paper_2104_10073_gb300 import build
    from paper_2104_10073_gb300 import zmc

    build.build()
    out = []
    for rate in args.serving_rates:
        r = run_serving(zmc, 0, rate, args.serving_seconds, args.serving_quints,
                        args.serving_chunks, args.serving_share)
        if r is not None:
            r["demand_gsps"] = rate * 500.5 * 1.444e6 / 1e9  # E[jobs/s x rows x N]
        out.append(r)
        print(json.dumps({"serving_point": {k: v for k, v in (r or {}).items() if k != "_stream"}}),
              file=sys.stderr, flush=True)
    # the bound at the highest rate the sweep delivered (the capacity, when the
    # sweep holds a point above it)
    cap = max((r["samples_per_s"] for r in out if r), default=0.0)
    chunk = 160 * (args.serving_quints or 26)
    for rate, r in zip(args.serving_rates, out):
        if r:
            stream = r.pop("_stream")
            if cap > 0:
                r["fifo_bound"] = fifo_bound(stream, cap)
                # the same stream through a model of the launch loop (default
                # launch rules only)
                if not (args.serving_chunks or args.serving_share):
                    jobs = [(at, W.total_samples(tab),
                             int(np.sum((tab["n_samples"].astype(np.int64) + chunk - 1) // chunk)))
                            for at, tab in W.serving_stream(rate, args.serving_seconds,
                                                            max_fns=1000)]
                    r["launch_model"] = launch_model(jobs, cap, chunk_samples=chunk)
    print(json.dumps({"serving_sweep": out, "seconds_per_rate": args.serving_seconds,
                      "job": "U{1..1000} mixed-style integrands, N ~ 10^U[4,7]"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-modes", action="store_true",
                    help="skip the functional, checkpoint/resume, user-integrand and "
                         "stratified (normal-mode) legs")
    ap.add_argument("--cpu-repeats", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--quints-per-lane", type=int, default=104,
                    help="chunk length = 160 x this many samples (with --no-autotune)")
    ap.add_argument("--serving-sweep", action="store_true")
    ap.add_argument("--serving-rates", type=float, nargs="+",
                    default=[10.0, 30.0, 100.0, 300.0, 1000.0])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--serving-rate", type=float, default=100.0)
    ap.add_argument("--serving-seconds", type=float, default=10.0)
    ap.add_argument("--serving-quints", type=int, default=0,
                    help="chunk length of the serving context (0: library default)")
    ap.add_argument("--serving-chunks", type=int, default=0,
                    help="chunks per serving iteration (0: library default)")
    ap.add_argument("--serving-share", type=int, default=0,
                    help="serving launches: 0 oldest job first (library default), > 0 equal "
                         "shares of at least this many chunks")
    args = ap.parse_args()
    world, rank, local = (int(os.environ.get("WORLD_SIZE", "1")),
                          int(os.environ.get("RANK", "0")),
                          int(os.environ.get("LOCAL_RANK", "0")))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.serving_sweep:
        run_serving_sweep(args)
        return
    world, rank, local = dist_setup()
    run_native(args, world, rank, local)


if __name__ == "__main__":
    main()
