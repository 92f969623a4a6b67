#!/usr/bin/env python3
"""Throughput of the FFT matched-filter search of arXiv:1708.01609 on GB300.

One step is one pass of the whole hot path over one synthetic segment:
  S1     segment spectrum of an N = 2^16 strain segment resident in HBM,
  S2-S6  the fused correlate kernel over all 2^20 chirp templates (template
         spectrum, spectral product, Parseval sigma, inverse FFT, kappa-sigma
         threshold, tail compaction), kappa = 5.5,
  S7     fetch of the tail count and records to host memory.
The metric is chirp correlations per second (templates x segments / s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torch.distributed.run, one rank per GPU, each rank
searching its own segment against the full bank (weak scaling; no collective
on the data path, only the barrier and the max-over-ranks time), or with
``--shard`` one segment against the bank split into one contiguous row range
per rank (strong scaling).  Rank 0 prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402
from paper_1708_01609_gb300 import metrics  # noqa: E402

N_SAMPLES = 1 << 16
KAPPA = 5.5
METRIC = "chirp correlations/s at N=2^16"
UNIT = "correlations/s"
PRECISIONS = {"fp32": 0, "bf16x3": 1, "fp16x3": 2}


def workload_config(templates: int, world: int, shard: bool = False) -> dict:
    return {
        "workload": (f"N=2^16 band-limited (350-2000 Hz) strain segment x {templates} chirp "
                     "templates (1024 f0 x 1024 fdot grid, tau 1 s, 5% taper), kappa 5.5, "
                     "32 injections SNR 8-30"),
        "segment_len": N_SAMPLES,
        "templates": templates,
        "kappa": KAPPA,
        "fs_hz": 4096.0,
        "l2": "inputs larger than L2: the 17.2 GB FP32 bank is streamed from HBM every step",
        "parallelism": (f"bank split into {world} contiguous row range(s), one per GPU, the "
                        "same segment on every GPU; tails stay on each rank's host"
                        if shard else
                        f"{world} independent replica(s), one segment per GPU per step"),
    }


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands
# ---------------------------------------------------------------------------
def oracle_sample(seconds: float, max_templates: int, batch: int = 8):
    """Time the oracle on the first templates of the benchmark bank until
    ``seconds`` of CPU work or ``max_templates`` are done."""
    import oracle as O
    seg, params = S.paper_case()
    y = seg.y
    done = 0
    t0 = time.perf_counter()
    while done < max_templates:
        bank = O.chirp_bank(params[done:done + batch], 4096.0, 4096, 0.05)
        O.search(y, bank, KAPPA, k0=done, batch=batch)
        done += len(bank)
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done, dt


def _oracle_worker(args):
    """One process of the all-cores baseline: the oracle on its own slice of
    the bank for about ``seconds``."""
    first, seconds, batch = args
    import oracle as O
    seg, params = S.paper_case()
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        k = first + done
        bank = O.chirp_bank(params[k:k + batch], 4096.0, 4096, 0.05)
        O.search(seg.y, bank, KAPPA, k0=k, batch=batch)
        done += len(bank)
    return done, time.perf_counter() - t0


def oracle_parity_case_rate() -> dict:
    """The oracle on the N = 2^14 parity case (64 chirps, kappa 5), one
    process: the small configuration beside the benchmark's."""
    import oracle as O
    seg, params = S.small_case()
    t0 = time.perf_counter()
    bank = O.chirp_bank(params, 4096.0, 4096, 0.05)
    O.search(seg.y, bank, 5.0, batch=8)
    dt = time.perf_counter() - t0
    return {"value": len(params) / dt, "unit": UNIT, "cores": 1,
            "sample": f"N=2^14 segment x 64 chirps (8 f0 x 8 fdot), one process, {dt:.2f} s"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline(seconds: float = 15.0) -> dict:
    """The oracle as it stands on the host cores: one process, then one
    process per core on disjoint slices of the bank (spawned: the parent has
    already used the GPU)."""
    import multiprocessing as mp
    done, dt = oracle_sample(seconds / 2, 4096)
    single = done / dt
    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(4096 * i, seconds / 2, 8) for i in range(cores)])
    total = sum(d for d, _ in res)
    rate = sum(d / t for d, t in res)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": (f"FP64 oracle (own radix-2 FFT, numpy) against the N=2^16 segment: "
                       f"{cores} processes, one per core, on disjoint slices of the 2^20 bank "
                       f"({total} templates, ~{seconds / 2:.0f} s each)"),
            "single_process": {"value": single, "cores": 1,
                               "sample": f"the first {done} templates, {dt:.1f} s"},
            "parity_case": oracle_parity_case_rate()}


# ---------------------------------------------------------------------------
# reference arm: the oracle timed as the reference implementation
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    per_step = args.ref_templates
    for _ in range(args.warmup):
        oracle_sample(0.0, per_step, batch=per_step)
    times = []
    for _ in range(args.steps):
        done, dt = oracle_sample(0.0, per_step, batch=per_step)
        times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(1 << 20, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": (f"each step: FP64 oracle on {per_step} templates of the "
                                    "2^20 bank against the N=2^16 segment, one process")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# the sources the N = 2^16 FP32 correlate kernel is compiled from
CORRELATE_SOURCES = ("bege_corr.cuh", "bege_fft.cuh", "bege_corr_s8.cu", "bege_internal.h")


def correlate_source_hash() -> str:
    src = os.path.join(ROOT, "paper_1708_01609_gb300", "csrc")
    h = hashlib.sha256()
    for name in CORRELATE_SOURCES:
        with open(os.path.join(src, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _counter_record():
    """The committed ncu record of the correlate kernel, if its source is
    unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get("correlate_kernel")
    if not rec or rec.get("source_sha256") != correlate_source_hash():
        return None
    return rec


def traffic_record(templates: int):
    """DRAM bytes per correlate launch from the committed ncu summary, if the
    kernel source is unchanged since it was captured; else None."""
    rec = _counter_record()
    return None if rec is None else rec["dram_bytes_per_correlation"] * templates


def ncu_counters():
    """Pipe and issue utilisation of the correlate kernel from the same ncu
    capture (percent of peak), or None when the source has changed."""
    rec = _counter_record()
    if rec is None or "counters" not in rec:
        return None
    return dict(rec["counters"], source="profiles/traffic.json")


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1708_01609_gb300 import binding, build
    build()
    cap = 1 << 25   # all hits of 32 strong injections per segment run to ~1.4e7 records
    prec = PRECISIONS[args.precision]
    ctx = binding.Context(local, tail_capacity=cap, precision=prec)
    templates = args.templates
    seg_data, params = S.paper_case(seed=2017 + (0 if args.shard else rank))
    params = params[:templates]
    # --shard: this rank holds and searches only its own rows of the bank
    from paper_1708_01609_gb300 import shard
    k0, k1 = shard.shard_ranges(templates, world)[rank] if args.shard else (0, templates)
    rows = k1 - k0
    stream_obj = torch.cuda.current_stream()
    stream = stream_obj.cuda_stream
    bank = ctx.bege_define_bank(params[k0:k1], tau=1.0, taper_frac=0.05, stream=stream)
    y_dev = torch.from_numpy(seg_data.y).cuda()
    y_pin = torch.from_numpy(seg_data.y).pin_memory()
    y_host = y_pin.numpy()
    out = torch.empty(cap * 12, dtype=torch.uint8).pin_memory().numpy().view(binding.TAIL_DTYPE)
    torch.cuda.synchronize()

    def step(host: bool):
        if host:
            seg = ctx.bege_load_segment(y_host, 0, stream)
        else:
            seg = ctx.bege_load_segment_device(y_dev.data_ptr(), N_SAMPLES, 0, stream)
        job = ctx.bege_correlate(seg, bank, 0, rows, KAPPA, stream)
        recs, total = ctx.bege_fetch_tails(job, out=out)
        if len(recs) != total:
            raise RuntimeError(f"tail buffer overflow: {total} tails, {len(recs)} copied")
        kms = ctx.bege_job_kernel_ms(job)
        ctx.bege_release(job)
        ctx.bege_release(seg)
        return total, kms

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(host: bool, steps: int, clocks: ClockSampler | None = None):
        barrier()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream_obj)
        tails, kms = [], []
        for _ in range(steps):
            t, k = step(host)
            tails.append(t)
            kms.append(k)
        e1.record(stream_obj)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        barrier()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, tails, kms, clk

    for _ in range(args.warmup):
        step(False)
    ms, tails, kms, clk = timed(False, args.steps, ClockSampler(local))
    for _ in range(max(1, args.warmup // 2)):
        step(True)
    ms_e2e, tails_e2e, _, _ = timed(True, args.steps)

    units = templates * (1 if args.shard else world) * args.steps
    value = units / (ms / 1e3)
    value_e2e = units / (ms_e2e / 1e3)
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    peak = metrics.fp32_peak_flops(props.multi_processor_count, sm_max)
    kernel_ms = statistics.mean(kms)
    flops_launch = rows * metrics.nominal_flops_per_correlation(N_SAMPLES)
    achieved = flops_launch / (kernel_ms / 1e3)
    traffic = traffic_record(rows)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(templates, world, args.shard),
        "roofline": {
            "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "correlate_kernel<4096,8,2,256>", "kernel_ms": kernel_ms,
            "flops_per_launch": flops_launch,
            "peak_basis": (f"FP32 ALU: {props.multi_processor_count} SMs x 128 lanes x 2 flops x "
                           f"{sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json)"),
            "flop_convention": "5 N log2 N per correlation (Eq. nd)",
            "ncu": ncu_counters(),
        },
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": N_SAMPLES * 4,
                "d2h_bytes_per_step": int(8 + 12 * statistics.mean(tails_e2e))},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "tails_per_step": statistics.mean(tails),
    }
    if rank == 0 and world == 1 and args.precision == "fp32":
        line["fft_normalized"] = fft_normalized(kernel_ms, templates)
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_precision_form:
        line["max_projection"] = max_projection_form(ctx, bank, y_dev, templates, args, value,
                                                     stream_obj)
        line["multi_segment"] = multi_segment_form(ctx, bank, templates, value)
        ctx.close()
        ctx = None
        line["precision_form"] = {
            name: precision_form(PRECISIONS[name], seg_data, params, templates, args, value, local)
            for name in ("bf16x3", "fp16x3")}
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_serving:
        if ctx is not None:
            ctx.close()
            ctx = None
        line["serving"] = serving_form(args, local)
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_batch:
        if ctx is not None:
            ctx.close()
            ctx = None
        line["batch"] = batch_form(args, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def fft_normalized(kernel_ms: float, templates: int, batch: int = 2048, reps: int = 10) -> dict:
    """The paper's efficiency measure (Sec. 4: ~65%, 'normalised to FFT
    alone'): the time the vendor FFT library needs for one correlation's
    transforms, a forward and an inverse real FFT of N = 2^16 (cuFFT through
    torch.fft, batched, device-resident), divided by the correlate kernel's
    time per correlation.  Context for the roofline, not a replacement."""
    import torch
    x = torch.randn(batch, N_SAMPLES, device="cuda", dtype=torch.float32)
    spec = torch.fft.rfft(x)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / batch * 1e3  # us per transform

    # unnormalised in both directions, so no scaling kernel follows the FFT
    t_r2c = timed(lambda: torch.fft.rfft(x, norm="backward"))
    t_c2r = timed(lambda: torch.fft.irfft(spec, n=N_SAMPLES, norm="forward"))
    t_corr = kernel_ms / templates * 1e3
    del x, spec
    torch.cuda.empty_cache()
    return {"cufft_rfft_us": t_r2c, "cufft_irfft_us": t_c2r, "correlation_us": t_corr,
            "efficiency": (t_r2c + t_c2r) / t_corr,
            "basis": "cuFFT R2C + C2R of N=2^16 (batch 2048, FP32, device-resident, no "
                     "normalisation pass; the C2R time includes the library's copy of its "
                     "input) per correlation / correlate kernel time per correlation (the "
                     "paper's 'efficiency normalised to FFT alone', Sec. 4)"}


def multi_segment_form(ctx, bank: int, templates: int, fp32_value: float, m: int = 8,
                       reps: int = 3) -> dict:
    """The paper's block of segments per template (Sec. 3.2): m segments of
    N = 2^16 against the whole bank in one bege_correlate_multi launch, the
    template transforms shared; kernel time per launch (CUDA events around it)."""
    segs = [ctx.bege_load_segment(S.band_limited_noise(N_SAMPLES, 4000 + i)) for i in range(m)]
    times = []
    for r in range(reps + 1):
        jobs = ctx.bege_correlate_multi(segs, bank, 0, templates, KAPPA)
        for j in jobs:
            ctx.bege_fetch_tails(j, capacity=0)
        if r > 0:
            times.append(ctx.bege_job_kernel_ms(jobs[0]))
        for j in jobs:
            ctx.bege_release(j)
    for sg in segs:
        ctx.bege_release(sg)
    ms = statistics.median(times)
    value = m * templates / (ms / 1e3)
    return {"segments": m, "value": value, "unit": UNIT, "kernel_ms": ms,
            "vs_fp32_path": value / fp32_value,
            "note": "one launch for m segments: forward template transforms once, product, "
                    "inverse and tails per segment; results bitwise those of single searches"}


def max_projection_form(ctx, bank: int, y_dev, templates: int, args, fp32_value: float,
                        stream_obj) -> dict:
    """The per-lag maximum over the bank (bege_correlate_max, Eq. Ak / BA) on
    the same workload: a step is S1 + the correlate kernel with the
    projection epilogue + the projection (N lags) read back to the host."""
    import torch
    stream = stream_obj.cuda_stream

    def step():
        seg = ctx.bege_load_segment_device(y_dev.data_ptr(), N_SAMPLES, 0, stream)
        job = ctx.bege_correlate_max(seg, bank, 0, templates, KAPPA, stream)
        snr, tmpl = ctx.bege_fetch_max(job, N_SAMPLES)
        ctx.bege_release(job)
        ctx.bege_release(seg)
        return int((tmpl >= 0).sum())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream_obj)
    lags = [step() for _ in range(args.steps)]
    e1.record(stream_obj)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = templates * args.steps / (ms / 1e3)
    return {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
            "vs_fp32_path": value / fp32_value, "lags_with_a_hit": statistics.mean(lags),
            "d2h_bytes_per_step": N_SAMPLES * 8,
            "note": "FP32 path with the Eq. Ak projection epilogue (64-bit atomic maximum per "
                    "lag); all-hit records are still collected on the device"}


def tc_flops_per_template(n: int) -> float:
    """Dense MMA flops of the precision form per template: S/2 groups of two
    4096-point columns, four GEMMs of M = N = 128 with K = 64 (half-zero
    template input) and 3 x 128, times the three split terms (both forms)."""
    s_cols = max(1, (n // 2) // 4096)
    terms = 3
    per_group = terms * (64 + 3 * 128) * 128 * 128 * 2
    return (s_cols // 2 if s_cols >= 2 else 1) * per_group


def precision_form(prec: int, seg_data, params, templates: int, args, fp32_value: float,
                   device: int) -> dict:
    """The precision form on the same workload: device-resident steps timed
    like the FP32 path's (CUDA events on the launching stream)."""
    import torch
    from paper_1708_01609_gb300 import binding
    ctx = binding.Context(device, tail_capacity=1 << 25, precision=prec)
    stream_obj = torch.cuda.current_stream()
    stream = stream_obj.cuda_stream
    bank = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05, stream=stream)
    y_dev = torch.from_numpy(seg_data.y).cuda()
    out = torch.empty((1 << 25) * 12, dtype=torch.uint8).pin_memory().numpy().view(binding.TAIL_DTYPE)

    def step():
        seg = ctx.bege_load_segment_device(y_dev.data_ptr(), N_SAMPLES, 0, stream)
        job = ctx.bege_correlate(seg, bank, 0, templates, KAPPA, stream)
        recs, total = ctx.bege_fetch_tails(job, out=out)
        kms = ctx.bege_job_kernel_ms(job)
        ctx.bege_release(job)
        ctx.bege_release(seg)
        return total, kms

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream_obj)
    res = [step() for _ in range(args.steps)]
    e1.record(stream_obj)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    value = templates * args.steps / (ms / 1e3)
    kernel_ms = statistics.mean(r[1] for r in res)
    peaks = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops_sustained") or 1700.0
    fp32_peak = metrics.fp32_peak_flops(torch.cuda.get_device_properties(device).multi_processor_count,
                                        peaks.get("sm_max_mhz") or 2070.0) / 1e12
    method = templates * metrics.nominal_flops_per_correlation(N_SAMPLES) / (kernel_ms / 1e3) / 1e12
    mma = templates * tc_flops_per_template(N_SAMPLES) / (kernel_ms / 1e3) / 1e12
    return {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps, "kernel_ms": kernel_ms,
            "vs_fp32_path": value / fp32_value, "tails_per_step": statistics.mean(r[0] for r in res),
            "method_work": {"achieved": method, "unit": "TFLOP/s",
                            "frac_of_fp32_peak": method / fp32_peak,
                            "frac_of_bf16_peak": method / bf16_peak,
                            "fp32_peak": fp32_peak, "bf16_peak": bf16_peak,
                            "basis": "the method's nominal 5 N log2 N flops per correlation "
                                     "(Eq. nd) over the kernel's CUDA-event time; peaks: FP32 "
                                     "ALU (SMs x 128 x 2 x max SM clock) and the measured "
                                     "sustained bf16 of MEASURED_PEAKS.json"},
            "mma_pipe": {"achieved": mma, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": mma / bf16_peak,
                         "basis": "diagnostic: dense MMA flops issued, including the three "
                                  "split terms, against the measured sustained bf16 peak (FP16 "
                                  "has the same dense rate)"},
            "error_bar_sigma": 2e-3}


def batch_form(args, device: int = 0) -> dict:
    """Batching form: 64 segments, N uniform over 2^14..2^17, each against
    its own sub-bank of 2^12..2^16 chirps (tau 0.5 s or 1 s), 8 injections
    each; one persistent launch in a CUDA graph per step, plan chosen by the
    batch autotuner.  Graph launches timed with CUDA events on the launching
    stream, with the clocks sampled meanwhile."""
    import torch
    from paper_1708_01609_gb300 import binding
    ctx = binding.Context(device, tail_capacity=1 << 22)
    entries, grids = S.batch_case()
    stream_obj = torch.cuda.current_stream()
    stream = stream_obj.cuda_stream
    banks = {tau: ctx.bege_define_bank(grids[tau], tau=tau, taper_frac=0.05, stream=stream)
             for tau in grids}
    spec = [(e.seg.y, banks[e.tau], e.k0, e.k1, KAPPA) for e in entries]
    batch = ctx.bege_batch_create(spec, stream=stream)
    tuned_ms = ctx.bege_batch_autotune(batch, reps=2, stream=stream)
    plan = ctx.bege_batch_get_plan(batch)
    steps = max(3, min(args.steps, 10))
    for _ in range(max(3, args.warmup)):
        ctx.bege_batch_run(batch, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream_obj)
    for _ in range(steps):
        ctx.bege_batch_run(batch, stream)
    e1.record(stream_obj)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    corr = sum(e.k1 - e.k0 for e in entries)
    flops = sum((e.k1 - e.k0) * metrics.nominal_flops_per_correlation(e.seg.n) for e in entries)
    tails = sum(ctx.bege_batch_fetch_tails(batch, i, capacity=0)[1] for i in range(len(entries)))
    ctx.close()
    return {
        "value": corr * steps / (ms / 1e3), "unit": UNIT, "graph_launches": steps,
        "ms_per_graph_launch": ms / steps,
        "workload": (f"{len(entries)} segments, N uniform over 2^14..2^17, sub-banks of "
                     "2^12..2^16 chirps (log-uniform), tau 0.5 or 1 s, 8 injections each, "
                     "kappa 5.5; one CUDA graph launch per step"),
        "correlations_per_graph_launch": corr,
        "segment_lengths": sorted({e.seg.n for e in entries}),
        "nominal_tflops": flops * steps / (ms / 1e3) / 1e12,
        "autotuned": {"plan": ["persistent", "per-segment"][plan[0]], "chunk": plan[1],
                      "order": ["longest-first", "interleaved"][plan[2]],
                      "radix": plan_radix(plan), "autotuned_ms": tuned_ms},
        "tails_per_graph_launch": tails,
        "clocks": clk,
    }


def plan_radix(plan) -> str:
    """The column FFT plan the batch runs (the autotuner's radix axis)."""
    return plan[3] if len(plan) > 3 else "16x16x16"


def run_batch_form(args):
    """``--form batch``: the batching form alone, as its own JSON line."""
    import torch
    from paper_1708_01609_gb300 import build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    build()
    b = batch_form(args)
    line = {"form": "batch", "metric": "chirp correlations/s, batching form", "value": b["value"],
            "unit": UNIT, "n_gpus": 1, "steps": b["graph_launches"], "warmup": args.warmup,
            "ms_per_step": b["ms_per_graph_launch"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": b["workload"]}, "batch": b}
    print(json.dumps(line), flush=True)
    return 0


def serving_form(args, device: int = 0) -> dict:
    """Serving form: two channels of band-limited noise emit 8, 16 and 32 s
    segments with Poisson arrivals at 2x real time; every request searches the
    resident 2^20-chirp bank at kappa 5.5 under a 120 GB device budget.
    Paced run: latency (p50/p99), throughput, real-time factor.  Saturated
    run (every request submitted at once): capacity.  Clocks are sampled
    during each run."""
    import threading

    from paper_1708_01609_gb300 import binding
    budget = 120 * 10**9
    ctx = binding.Context(device, tail_capacity=1 << 21, hbm_budget_bytes=budget)
    params = S.grid_paper()
    bank = ctx.bege_define_bank(params, tau=1.0, taper_frac=0.05)
    count = len(params)
    sv = ctx.bege_serve_create(bank, KAPPA, streams=args.serve_streams,
                               slice_templates=args.serve_slice,
                               hbm_budget_bytes=budget - ctx.bege_device_bytes())
    warm = S.serving_stream(3, seed=1)
    for a in warm:
        ctx.bege_serve_wait(sv, ctx.bege_serve_submit(sv, a.y, a.channel))

    def run(arrivals, paced):
        ids = [None] * len(arrivals)
        clocks = ClockSampler(device)
        clocks.start()
        t0 = time.monotonic()

        def feed():
            for i, a in enumerate(arrivals):
                if paced:
                    delay = t0 + a.t - time.monotonic()
                    if delay > 0:
                        time.sleep(delay)
                ids[i] = ctx.bege_serve_submit(sv, a.y, a.channel)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        infos = []
        for rid in ids:
            ctx.bege_serve_wait(sv, rid)
            infos.append(ctx.bege_serve_info_get(sv, rid))
            ctx.bege_serve_forget(sv, rid)
        clk = clocks.stop()
        lat = np.array([i["t_done"] - i["t_submit"] for i in infos]) * 1e3
        span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
        data_s = sum(a.n for a in arrivals) / S.FS
        return {
            "requests": len(arrivals), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "mean_ms": float(lat.mean()), "wall_s": span,
            "correlations_per_s": len(arrivals) * count / span,
            "real_time_factor": data_s / span / 2.0,
            "tails_per_request_mean": float(np.mean([i["n_tails"] for i in infos])),
            "tails_per_request_max": int(max(i["n_tails"] for i in infos)),
            "segment_lengths": sorted({a.n for a in arrivals}),
            "offered_real_time_factor": (data_s / (max(a.t for a in arrivals) -
                                                   min(a.t for a in arrivals)) / 2.0
                                         if paced and len(arrivals) > 1 else None),
            "clocks": clk,
        }

    paced = run(S.serving_stream(args.serve_requests, seed=2024, speed=2.0), paced=True)
    burst = run(S.serving_stream(args.serve_burst, seed=7, speed=2.0), paced=False)
    ctx.bege_serve_destroy(sv)
    ctx.close()
    return {
        "metric": "served p99 latency, 2x real time, 2^20-chirp bank",
        "p50_ms": paced["p50_ms"], "p99_ms": paced["p99_ms"],
        "correlations_per_s": paced["correlations_per_s"],
        "real_time_factor": paced["real_time_factor"],
        "tails_per_request_mean": paced["tails_per_request_mean"],
        "workload": ("two channels of band-limited noise, 8/16/32 s segments, Poisson "
                     "arrivals at 2x real time per channel, full 2^20 chirp bank per "
                     "request, kappa 5.5, 120 GB device budget"),
        "streams": args.serve_streams, "slice_templates": args.serve_slice,
        "paced": paced,
        "saturated": burst,
    }


def run_serve_form(args):
    """``--form serve``: the serving form alone, as its own JSON line."""
    import torch
    from paper_1708_01609_gb300 import build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    build()
    sv = serving_form(args)
    line = {"form": "serve", "metric": sv["metric"], "value": sv["p99_ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sv["workload"], "streams": sv["streams"],
                       "slice_templates": sv["slice_templates"]},
            "serving": sv}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["search", "batch", "serve"], default="search",
                    help="search: the headline N=2^16 x 2^20 step; batch: the batching form; "
                         "serve: the serving form")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the paced serving run (arrivals at 2x real time)")
    ap.add_argument("--serve-burst", type=int, default=24,
                    help="requests of the saturated serving run")
    ap.add_argument("--serve-streams", type=int, default=3)
    ap.add_argument("--serve-slice", type=int, default=65536)
    ap.add_argument("--templates", type=int, default=1 << 20,
                    help="bank rows per step (the benchmark uses all 2^20)")
    ap.add_argument("--precision", choices=list(PRECISIONS), default="fp32",
                    help="fp32: the plain path; bf16x3 / fp16x3: the precision form "
                         "(column FFTs as split-operand tensor-core GEMMs)")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip timing the BF16x3 / FP16x3 precision form beside the FP32 path")
    ap.add_argument("--shard", action="store_true",
                    help="split the bank over the ranks (one segment, strong scaling) instead "
                         "of one replica per rank")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the paced serving run (about 80 s) in the default line")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batching form in the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-templates", type=int, default=8,
                    help="templates per reference-arm step (bounded oracle sample)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batch":
        return run_batch_form(args)
    if args.form == "serve":
        return run_serve_form(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
