#!/usr/bin/env python
"""Throughput benchmark: template-seconds filtered per second on B300 (paper Eq. 1, cores = 1 per GPU).

Headline workload (per GPU rank): one production-shaped SVD bin of 1000
templates (60 s Newtonian chirps, chirp mass 1.0-1.5 Msun, six time slices at
4096 ... 128 Hz, SVD truncated at 99.99% of sigma^2) on two detectors (H1, L1:
two units, independent seeded white noise, injections at SNR 8-30).  A step is
one grouped push of ``--push-seconds`` of strain to both units: decimation,
basis FIR, mixing, up-sampling + sum, window maxima, FP32 refinement of the
candidate maxima and trigger hand-off.  Data are synthetic (seeded white
Gaussian noise; random-parameter chirps).

The device-timed value has the strain already resident in HBM; L2 is flushed
(256 MB write) between timed steps, outside the step's events, and a ~2-ms
device spin ahead of each step lets the host enqueue the push before the step's
start event runs (host time belongs to e2e).  ``e2e`` runs
the same steps through the C ABI from host buffers, with the host->device
strain copies and the trigger read-back inside the timed region.

The same run also reports, as sub-results of the metric: the other precisions
(``by_precision``), the production bin with 1-s buffers (``push_1s``), the
grouped batch of uneven bins (``batch``: 200 bins x 2 detectors in one grouped
launch per stage) and the serving loop (``serve``: 1-s buffers of 1000 bins x 2
detectors with Poisson arrivals, p50 / p99 buffer-to-trigger latency).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
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

import synth  # noqa: E402

METRIC = "template-seconds filtered/s on 1 B300 (FP32 vs BF16/FP8 grouped); p99 latency"
UNIT = "template-s/s"
L2_FLUSH_BYTES = 256 << 20
DTYPES = {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}
INTERP_FLOPS_PER_OUTPUT = 32.0      # halfband x2 interpolation: 32 multiply-adds per odd output, none per even
RECORD_BYTES = 32                   # one top-level partial window record (sizeof WinPart)
# With graphs on, a context keeps one executable graph per (group shape, trigger slot, task arena):
# the 8-slot trigger ring cycles through 8 of them, each instantiated on its first use.  The
# warm-up covers the whole ring, so no graph instantiation falls inside the timed steps.
GRAPH_RING = 8
HOST_AHEAD_CYCLES = 4_000_000       # ~2 ms spin before each device-timed step (outside its events)


def warm_pushes(warmup: int, graphs: bool) -> int:
    return max(warmup, GRAPH_RING) if graphs else warmup


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="lloid", choices=["lloid", "reference"])
    p.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16", "fp8"])
    p.add_argument("--compare", default="fp32,fp16,fp8", help="other precisions timed for by_precision ('none': skip)")
    p.add_argument("--push-seconds", type=int, default=16)
    p.add_argument("--templates", type=int, default=1000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--graphs", default="on", choices=["on", "off"],
                   help="capture every push into a CUDA graph (reused per group shape)")
    p.add_argument("--xi2", default="on", choices=["on", "off"],
                   help="production bank: hand the templates' autocorrelation to svdbank_create (xi^2 of every trigger)")
    p.add_argument("--autotune", default="on", choices=["on", "off"],
                   help="time the mixing kernel's pipeline shapes on the first push of each launch shape")
    p.add_argument("--cpu-seconds", type=float, default=4.0, help="strain seconds per oracle worker")
    p.add_argument("--workload", default="production", choices=["production", "batch", "serve"],
                   help="production: one 1000-template bin x 2 detectors (+ sub-results); batch / serve: that "
                        "sub-result alone as the line")
    p.add_argument("--sub", default="push1s,batch,paper,serve",
                   help="sub-results of the production line ('none': skip)")
    p.add_argument("--bins", type=int, default=200, help="batch: uneven bins (x 2 detectors)")
    p.add_argument("--paper-banks", default="1,2,4,8,16,32",
                   help="paper shape: numbers of (1,004-template, 73 s) banks per detector, 3 detectors")
    p.add_argument("--paper-steps", type=int, default=5)
    p.add_argument("--batch-steps", type=int, default=6)
    p.add_argument("--batch-push-seconds", type=int, default=8)
    p.add_argument("--serve-bins", type=int, default=1000)
    p.add_argument("--serve-seconds", type=int, default=20, help="serve: 1-s buffers per stream")
    p.add_argument("--serve-precisions", default="bf16,fp8")
    p.add_argument("--distinct-banks", type=int, default=20, help="serve: distinct banks the bins cycle through")
    p.add_argument("--time-scale", type=float, default=1.0, help="serve: arrival clock speed-up")
    return p.parse_args()


# ----------------------------------------------------------------------------- workload
def production_bank_templates(bin_index: int, n_templates: int):
    spec = synth.scaled_bin(synth.PRODUCTION_BIN, n_templates)
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s,
                               2, bin_index, 0)
    return spec, h


def production_config(spec, basis_counts, push_seconds: int) -> dict:
    """The workload as both arms name it (the reference arm times a bounded sample of it)."""
    return {"workload": f"production bin: {spec.n_templates} templates x 2 detectors, 6 slices 4096-128 Hz, "
                        f"L={list(basis_counts)}, {push_seconds} s pushes",
            "templates": 2 * spec.n_templates, "units_per_gpu": 2, "push_seconds": push_seconds}


def make_strain(bin_index: int, detector: int, seconds: int, f0: float, h, n_templates: int):
    n = int(seconds * f0)
    d = synth.white_noise(n, 2, bin_index, detector + 1)
    for inj in synth.injection_plan(max(1, seconds // 80), n_templates, n, f0, 80.0, 8.0, 30.0, bin_index, detector):
        synth.inject(d, h, inj.template, inj.n_c, inj.amplitude, inj.phi0)
    return d


def _levels(bank):
    f0 = bank.top_rate_hz
    lv = {}
    for s in bank.slices:
        k = int(round(math.log2(f0 / s.rate_hz)))
        lv.setdefault(k, []).append(s)
    return lv


def algorithmic_model(bank, units: int, B_s: float, precision: str = "fp32"):
    """Per-stage algorithmic FLOPs and HBM bytes of one push (all units), and the mix stage's own
    intermediate traffic.

    The method's work (a2-a5): FIR 2 L Q FLOPs per output; mixing 2 L_k FLOPs per output of each
    real filter; the x2 interpolation 32 FLOPs per interpolated output (halfband: 32 odd taps
    on odd outputs, a copy on even ones).  Bytes that must move: weights (re-read per push), the
    basis outputs between the FIR and the mixing, the strain, and the top-level window records (two
    32-byte records per template and 128 samples).  Weights and basis outputs move in the operand
    width of their GEMM (SB_FP8: E4M3 FIR weights, BF16 basis outputs and mixing).  The per-level
    SNR y_k (k >= 1) that one mixing launch writes and the next finer one reads is the design's own
    intermediate, reported separately, not as algorithmic work."""
    w_fir = {"fp32": 4.0, "bf16": 2.0, "fp16": 2.0, "fp8": 1.0}[precision]
    w_mix = {"fp32": 4.0, "bf16": 2.0, "fp16": 2.0, "fp8": 2.0}[precision]
    fused = precision != "fp32"
    yb = 4.0 if precision == "fp16" else 2.0                   # bytes per stored y sample
    f0 = bank.top_rate_hz
    M2 = 2 * bank.n_templates
    levels = _levels(bank)
    kmax = max(levels)
    fl = {k: 0.0 for k in ("fir", "mix", "upsample", "decimate", "trigger")}
    by = {k: 0.0 for k in fl}
    inter = 0.0
    for s in bank.slices:
        L, Q = s.basis.shape
        N = B_s * s.rate_hz
        fl["fir"] += 2.0 * L * Q * N
        by["fir"] += w_fir * L * Q + w_fir * N + w_mix * L * N
    for k, ss in levels.items():
        Lk = sum(s.basis.shape[0] for s in ss)
        N = B_s * f0 / 2 ** k
        fl["mix"] += 2.0 * M2 * Lk * N
        by["mix"] += w_mix * (M2 * Lk + Lk * N)
        if not fused:
            by["mix"] += 4.0 * M2 * N * (2 if k < kmax else 1)
    if fused:
        by["mix"] += (M2 / 2) * (B_s * f0 / 128) * 2 * RECORD_BYTES
        for k in range(1, kmax + 1):                            # every stored level, with a slice or not
            inter += 2 * yb * M2 * B_s * f0 / 2 ** k
    for k in range(0, kmax):
        N = B_s * f0 / 2 ** k                                   # interpolated outputs at level k
        if fused:
            fl["mix"] += M2 * N * INTERP_FLOPS_PER_OUTPUT
        else:
            fl["upsample"] += M2 * N * INTERP_FLOPS_PER_OUTPUT
            by["upsample"] += 4.0 * M2 * (N / 2 + N)
    for k in range(1, kmax + 1):
        N = B_s * f0 / 2 ** k
        fl["decimate"] += 2 * N * 33
        by["decimate"] += 4.0 * (3 * N)
    fl["trigger"] = 3.0 * M2 / 2 * B_s * f0 if not fused else 0.0
    # FP32: the top-rate SNR block is read once; fused modes: the window records the mixing wrote
    by["trigger"] = 4.0 * M2 * B_s * f0 if not fused else (M2 / 2) * (B_s * f0 / 128) * 2 * RECORD_BYTES
    return {k: fl[k] * units for k in fl}, {k: by[k] * units for k in by}, inter * units


def model_sum(banks_units, B_s, precision):
    flops, bytes_, inter = {}, {}, 0.0
    for b, n in banks_units:
        f1, b1, i1 = algorithmic_model(b, n, B_s, precision)
        for k in f1:
            flops[k] = flops.get(k, 0.0) + f1[k]
            bytes_[k] = bytes_.get(k, 0.0) + b1[k]
        inter += i1
    return flops, bytes_, inter


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event reasons of the bench's GPU, sampled every 2 ms by a host thread over
    NVML while the timed steps run (the same counters nvidia-smi's clocks query reads; a timed
    region of a few milliseconds still gets samples).  With no NVML binding, nvidia-smi -lms is
    run instead and waited for until it writes its first row."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None
        self.thread = None
        self.rows = []
        self.nvml_error = None

    def _nvml_handle(self):
        import pynvml
        pynvml.nvmlInit()
        try:
            import torch
            p = torch.cuda.get_device_properties(self.device)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
            return pynvml, pynvml.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.device)

    def start(self):
        import threading
        try:
            nv, h = self._nvml_handle()
            bits = [getattr(nv, "nvmlClocksEventReason" + n, None) for n in
                    ("HwSlowdown", "HwThermalSlowdown", "SwThermalSlowdown", "SwPowerCap")]
            reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = float(nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM))
            self.stop_flag = threading.Event()

            def run():
                while True:
                    r = int(reasons(h))
                    self.rows.append((float(nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)), mx,
                                      [self.NAMES[i] for i, b in enumerate(bits) if b is not None and r & b]))
                    if self.stop_flag.wait(0.002):
                        return
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        except Exception as e:
            self.thread = None
            self.nvml_error = f"{type(e).__name__}: {e}"[:120]
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.time()
            while os.path.getsize(self.path) == 0 and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join()
            rows = self.rows
        elif self.proc is not None:
            time.sleep(0.06)                     # one more row after the timed steps
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            rows = []
            for line in open(self.path):
                r = [p.strip() for p in line.split(",")]
                if len(r) >= 9 and r[1].replace(".", "").isdigit() and r[2].replace(".", "").isdigit():
                    rows.append((float(r[1]), float(r[2]),
                                 [self.NAMES[i] for i in range(4) if r[5 + i].lower() == "active"]))
            os.unlink(self.path)
        else:
            return None
        if not rows:
            return None
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted({n for r in rows for n in r[2]}), "samples": len(rows),
                "source": "nvml" if self.thread is not None else f"nvidia-smi (nvml: {self.nvml_error})"}


# ----------------------------------------------------------------------------- oracle (CPU)
BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


_WORKER_BANK = None


def _init_worker(bank):
    global _WORKER_BANK
    _WORKER_BANK = bank


def _oracle_task(args):
    """One oracle run (FP64): SVD path + window maxima on a seeded strain excerpt."""
    n, seed, win_len, threshold = args
    import oracle
    strain = synth.white_noise(n, 7, *seed)
    t = time.perf_counter()
    x = oracle.lloid_snr(_WORKER_BANK, strain)
    oracle.triggers(x, win_len, threshold, x.shape[1])
    return time.perf_counter() - t


def oracle_bank(h, spec):
    import oracle
    return oracle.build_bank(h, spec.top_rate_hz, spec.slices)


def _available_bytes() -> int:
    try:
        import psutil
        return int(psutil.virtual_memory().available)
    except ImportError:
        return int(os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE"))


def cpu_workers(seconds: float) -> int:
    """All host cores, one oracle process each, as far as host memory holds them (about 0.35 GB per
    second of excerpt per process for the production bin)."""
    cores = os.cpu_count() or 1
    per = 0.5e9 + 0.35e9 * seconds
    return max(1, min(cores, int(0.7 * _available_bytes() / per)))


class OraclePool:
    """`workers` spawned host processes holding the oracle's bank, BLAS pinned to one thread each."""

    def __init__(self, ob, workers: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers
        saved = {k: os.environ.get(k) for k in BLAS_ENV}
        for k in BLAS_ENV:                       # children read these when they import numpy
            os.environ[k] = "1"
        try:
            self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                             initializer=_init_worker, initargs=(ob,))
            list(self.ex.map(abs, range(workers)))          # start every process before timing
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def step(self, n: int, win_len: int, key: int) -> float:
        """Wall time of one round: every process filters its own n-sample excerpt."""
        t = time.perf_counter()
        list(self.ex.map(_oracle_task, [(n, (key, w), win_len, 6.0) for w in range(self.workers)]))
        return time.perf_counter() - t

    def close(self):
        self.ex.shutdown()


def cpu_baseline(ob, spec, seconds: float, workers: int):
    """The oracle as it stands on `workers` host processes, each on its own excerpt."""
    f0 = spec.top_rate_hz
    n = int(seconds * f0) // 32 * 32
    pool = OraclePool(ob, workers)
    try:
        wall = pool.step(n, int(f0), 0)
    finally:
        pool.close()
    value = workers * spec.n_templates * (n / f0) / wall
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "host_cpu_count": os.cpu_count(),
            "sample": f"{workers} processes (host has {os.cpu_count()} cores) x {n / f0:.0f} s excerpt "
                      f"of one unit of the production bin ({spec.n_templates} templates), FP64 SVD path + window "
                      f"maxima, BLAS 1 thread each; wall {wall:.1f} s (processes started before timing)"}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric, workload and config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, h = production_bank_templates(0, args.templates)
    ob = oracle_bank(h, spec)
    del h
    f0 = spec.top_rate_hz
    n = int(min(args.cpu_seconds, 4.0) * f0) // 32 * 32
    workers = cpu_workers(n / f0)
    pool = OraclePool(ob, workers)
    try:
        times = [pool.step(n, int(f0), 1 + step) for step in range(args.warmup + args.steps)][args.warmup:]
    finally:
        pool.close()
    total = sum(times)
    value = args.steps * workers * spec.n_templates * (n / f0) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": production_config(spec, [s.basis.shape[0] for s in ob.slices], args.push_seconds),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "host_cpu_count": os.cpu_count(),
                             "sample": f"each step: {workers} processes x a {n / f0:.0f} s excerpt of one unit "
                                       f"(independent noise), FP64 SVD path + window maxima, BLAS 1 thread each"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def shard_bins(n_bins: int, rank: int, world: int):
    """Bins of one rank: rank, rank + world, ...  Units never cross ranks, so the data path
    needs no collective."""
    return list(range(rank, n_bins, world))


def job_rate(tpl_s_rank: float, secs_rank: float, dist, device):
    """Whole-job throughput: every rank's template-seconds over the slowest rank's time
    (returns the rate and that time).  dist is torch.distributed or None (one process)."""
    if dist is None:
        return tpl_s_rank / secs_rank, secs_rank
    import torch
    t = torch.tensor([tpl_s_rank], dtype=torch.float64, device=device)
    s = torch.tensor([secs_rank], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(t.item()) / float(s.item()), float(s.item())


def measured_traffic(stage: str, workload: str, precision: str):
    """DRAM bytes per step of a stage from a committed ncu capture (profiles/), or None when
    there is none or the kernel source changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_{stage}_{workload}_{precision}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["kernel_source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, KeyError, ValueError):
        return None
    return float(rec["dram_bytes_per_step"]) if sha == rec.get("kernel_source_sha256_16") else None


def roofline_of(stages, flops, bytes_, inter, precision, steps, peaks, workload="production"):
    """Roofline of the stage that takes the most device time among the stages with an
    algorithmic model (the refinement's work depends on the candidates the data produce, so it
    has none and is reported through its time share only).  `achieved` = the stage's
    algorithmic work per push / its mean CUDA-event time per push."""
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12            # FP32 FFMA lanes x 2 FLOP x max clock
    tensor_peak = peaks.get("bf16_tflops", 1800.0)             # dense BF16 = FP16 rate, burst (short steps)
    busy = {k: v[0] for k, v in stages.items() if v[1] > 0 and (flops.get(k, 0.0) > 0 or bytes_.get(k, 0.0) > 0)}
    dom = max(busy, key=busy.get)
    out = {}
    for st in sorted(busy, key=busy.get, reverse=True)[:2]:
        st_ms, _ = stages[st]
        on_tensor = precision != "fp32" and st in ("fir", "mix")
        cpeak = tensor_peak if on_tensor else alu_peak
        # SB_FP8's basis FIR: E4M3 operands (nominal 2x the BF16 rate) with the strain as two terms
        src = "measured bf16_tflops (burst)" if on_tensor else "derived: 148 SM x 128 FP32 lanes x 2 FLOP x max SM clock"
        if precision == "fp8" and st == "fir":
            cpeak, src = 2.0 * tensor_peak, "measured bf16_tflops (burst) x 2 (E4M3 nominal ratio)"
        t_c = flops.get(st, 0.0) / (cpeak * 1e12)
        t_m = bytes_.get(st, 0.0) / (hbm_peak * 1e9)
        secs = st_ms / 1e3 / steps
        kname = {"mix": "tc_mixup_kernel (a3 mixing + a4 interpolation + a5 window partials)",
                 "fir": "tc_fir_kernel (a2 basis FIR)"}.get(st, st) if precision != "fp32" else st
        if t_c >= t_m:
            ach = flops[st] / secs / 1e12
            r = {"bound": "tensor" if on_tensor else "alu", "achieved": ach, "peak": cpeak, "unit": "TFLOP/s",
                 "frac": ach / cpeak, "algorithmic_flops_per_push": flops[st],
                 "algorithmic_bytes_per_push": bytes_.get(st, 0.0), "time_at_peak_us": 1e6 * t_c,
                 "time_us": 1e6 * secs}
        else:
            ach = bytes_[st] / secs / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                 "algorithmic_bytes_per_push": bytes_[st], "time_at_peak_us": 1e6 * t_m, "time_us": 1e6 * secs}
            src = "measured hbm_gbs"
        r["traffic"] = measured_traffic(st, workload, precision)
        if st == "mix" and precision != "fp32":
            r["intermediate_bytes_per_push"] = inter
        r["kernel"] = kname
        r["peak_source"] = src + " (of measured)" if "measured" in src else src
        out[st] = r
    return dom, out


def make_units_for(ctx, banks, precision, B, xi2_on=True, threshold=6.0, refine=5.5):
    """The two detectors of a bin share one copy of the bank's device data (svdbank_create_like)."""
    units = []
    for b in banks:
        if not xi2_on:
            b.autocorr = None
        u0 = ctx.create_unit(b, detector=0, precision=precision, threshold=threshold, refine_threshold=refine,
                             window_s=1.0, max_push_samples=B)
        units += [u0, ctx.create_like(u0, detector=1)]
    return units


def device_arm(lloid, torch, stream, local, banks, precision, B, steps, warmup, dev, graphs, autotune, barrier,
               flush, n_prof=None, make_units=None):
    """Time `steps` grouped pushes of B samples per unit with the strain resident in HBM.
    make_units(ctx) -> (units, detector of each unit); default: each bank on detectors 0 and 1."""
    ctx = lloid.Context(local, stream=stream.cuda_stream)
    ctx.graphs(graphs)
    ctx.autotune(autotune)
    tc0 = time.perf_counter()
    if make_units is None:
        units = make_units_for(ctx, banks, precision, B)
        dets = [det for _ in banks for det in (0, 1)]
    else:
        units, dets = make_units(ctx)
    create_s = time.perf_counter() - tc0
    n_units = len(units)
    n_prof = min(steps, 16) if n_prof is None else n_prof
    t = 0
    for _ in range(warm_pushes(warmup, graphs)):
        ctx.push_group(units, [dev[det][t:t + B] for det in dets], [t] * n_units, True)
        t += B
    ctx.pop_triggers()
    barrier()
    st0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    w0 = time.perf_counter()
    for i in range(steps):
        # a short spin on the device ahead of the step's start event: the host enqueues the push
        # (its graph update and launch) while the GPU spins, so a slow host call lands outside the
        # events (host time is part of e2e, not of the device-timed step)
        if hasattr(torch.cuda, "_sleep"):
            torch.cuda._sleep(HOST_AHEAD_CYCLES)
        flush.zero_()
        ev[i][0].record(stream)
        ctx.push_group(units, [dev[det][t:t + B] for det in dets], [t] * n_units, True)
        ev[i][1].record(stream)
        t += B
    barrier()
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    st1 = ctx.stats()
    # stage split from separate pushes with every launch bracketed by events (not timed above)
    ctx.profile(True)
    for i in range(n_prof):
        flush.zero_()
        ctx.push_group(units, [dev[det][t:t + B] for det in dets], [t] * n_units, True)
        t += B
    stages = ctx.stage_times()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    trig = ctx.pop_triggers()
    tuned = ctx.autotune_choices()
    ctx.close()
    return {"dev_s": dev_s, "wall": wall, "clocks": clk, "create_s": create_s, "stages": stages,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
            "launches": st1["kernel_launches"] - st0["kernel_launches"],
            "autotune": {"choices": tuned, "timed_launches": st1["autotune_launches"],
                         "in_timed_region": st1["autotune_launches"] - st0["autotune_launches"]},
            "refine_candidates": st1["refine_candidates"] - st0["refine_candidates"], "prof_steps": n_prof,
            "triggers": int(len(trig)), "n_units": n_units}


def paper_sweep(lloid, torch, stream, local, args, rank, world, dist, barrier, flush, graphs, autotune, peaks):
    """The paper's benchmark shape (Sec. IV, Fig. 3): one 1,004-template bank of 73 s templates per
    detector, three detectors of white Gaussian noise, the same bank provided n times per detector
    (svdbank_create_like shares its device data), one grouped push of 16 s per step; throughput
    against the number of banks.  Ranks split the bank copies."""
    spec = synth.PAPER_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 5, 0, 0)
    tb = time.perf_counter()
    bank = lloid.decompose(h, spec.top_rate_hz, spec.slices)
    del h
    setup = time.perf_counter() - tb
    f0 = int(spec.top_rate_hz)
    push_s, steps, warmup = 16, args.paper_steps, 2
    B = push_s * f0
    total = (warm_pushes(warmup, graphs) + steps + min(steps, 16)) * push_s
    dev = [torch.from_numpy(synth.white_noise(total * f0, 6, rank, det)).cuda() for det in range(3)]
    curve = []
    for nb in [int(x) for x in args.paper_banks.split(",") if x.strip()]:
        mine = len(shard_bins(nb, rank, world))
        if mine == 0:
            continue

        def make(ctx, mine=mine):
            units, dets = [], []
            for det in range(3):
                u0 = ctx.create_unit(bank, detector=det, precision=args.precision, threshold=6.0,
                                     refine_threshold=5.5, window_s=1.0, max_push_samples=B)
                units.append(u0)
                dets.append(det)
                for _ in range(mine - 1):
                    units.append(ctx.create_like(u0, detector=det))
                    dets.append(det)
            return units, dets

        r = device_arm(lloid, torch, stream, local, [bank], args.precision, B, steps, warmup, dev, graphs, autotune,
                       barrier, flush, make_units=make)
        tpl = 3 * mine * spec.n_templates * push_s * steps
        value, secs = job_rate(tpl, r["dev_s"], dist, "cuda")
        flops, bytes_, inter = model_sum([(bank, 3 * mine)], push_s, args.precision)
        _, roofs = roofline_of(r["stages"], flops, bytes_, inter, args.precision, r["prof_steps"], peaks, "paper")
        curve.append({"banks_per_detector": nb, "units": 3 * nb, "value": value, "ms_per_step": 1e3 * secs / steps,
                      "mix_frac": roofs.get("mix", {}).get("frac"), "fir_frac": roofs.get("fir", {}).get("frac")})
    del dev
    return {"workload": f"{spec.n_templates} templates of {spec.duration_s:.0f} s (6 slices 4096-128 Hz, "
                        f"L={bank.basis_counts()}), 3 detectors of white Gaussian noise, the same bank n times per "
                        f"detector, 16-s grouped pushes, {args.precision}",
            "unit": UNIT, "bank_setup_s": setup, "curve": curve}


def serve_once(lloid, serve, args, precision, rank, world, local):
    """Serving loop (1-s buffers, Poisson arrivals) over this rank's bins; returns the report summary."""
    banks = [synth.production_shape_bank(i) for i in range(args.distinct_banks)]
    g = np.random.default_rng(20241016 + rank)
    reqs = []
    for b in shard_bins(args.serve_bins, rank, world):
        bank = banks[b % len(banks)]
        for det in (0, 1):
            reqs.append(serve.StreamRequest(
                name=f"bin{b}-det{det}", bank=bank, detector=det,
                arrivals=serve.poisson_arrivals(g, args.serve_seconds, float(g.uniform(0.0, 5.0))),
                strain=(lambda j, b=b, det=det: synth.white_noise_block(j, 4096, 9, b, det)),
                unit_kwargs=dict(precision=precision, threshold=6.0, refine_threshold=5.5),
                share_key=f"bank{b % len(banks)}"))
    ctx = lloid.Context(local)
    tl = time.perf_counter()
    anchors = serve.preload(ctx, reqs, 4096)          # banks are loaded before data arrive
    load_s = time.perf_counter() - tl
    rep = serve.run(ctx, reqs, 4096, time_scale=args.time_scale, anchors=anchors)
    st = ctx.stats()
    ctx.close()
    s = rep.summary()
    s["bank_load_s"] = load_s
    s["template_seconds"] = rep.template_seconds
    s["gpu_launches"] = st["kernel_launches"]
    return s


def merge_serve(s, dist):
    """Whole-job serving numbers: template-seconds summed, the slowest rank's wall, the largest p99."""
    if dist is None:
        return s
    import torch
    v = torch.tensor([s["template_seconds"], s["wall_s"], s["p99_latency_s"] or 0.0, s["max_latency_s"] or 0.0],
                     dtype=torch.float64, device="cuda")
    t = v[:1].clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    s = dict(s)
    s["template_seconds"], s["wall_s"], s["p99_latency_s"], s["max_latency_s"] = float(t[0]), float(v[1]), \
        float(v[2]), float(v[3])
    s["template_seconds_per_s"] = s["template_seconds"] / s["wall_s"]
    return s


def serve_line(args, s, world, precision):
    return {"metric": METRIC, "value": s["template_seconds_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": s["pushes"], "warmup": 0, "ms_per_step": 1e3 * s["wall_s"] / max(1, s["pushes"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[precision],
            "data": "synthetic (seeded white noise per (bin, detector, buffer); production-shaped random banks)",
            "config": {"workload": f"serve: {args.serve_bins} bins x 2 detectors, 1-s buffers, Poisson arrivals "
                                   f"(1/s per stream) for {args.serve_seconds} s, banks cycled from "
                                   f"{args.distinct_banks} production-shaped banks (~1000 templates, 6 slices)",
                       "time_scale": args.time_scale, "precision": precision, "bank_load_s": s["bank_load_s"]},
            "latency": {"p50_s": s["p50_latency_s"], "p99_s": s["p99_latency_s"], "max_s": s["max_latency_s"],
                        "buffers": s["buffers"], "definition": "buffer arrival -> its push finished and its "
                                                               "triggers host-visible"},
            "serving": s, "gpu_launches": s["gpu_launches"]}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2410_16416_b300 as lloid
    from paper_2410_16416_b300 import serve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.workload == "serve":                      # the serving loop alone as the line
        s = merge_serve(serve_once(lloid, serve, args, args.precision, rank, world, local), dist)
        if rank == 0:
            print(json.dumps(serve_line(args, s, world, args.precision)), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    # One non-default stream for the library, the L2 flush and the timing events.
    # (torch's default stream has handle 0, which the C ABI reads as "no stream".)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    graphs, autotune = args.graphs == "on", args.autotune == "on"

    def batch_run(precision, n_bins, steps, warmup, push_s):
        banks = [synth.shape_only_bank(b) for b in shard_bins(n_bins, rank, world)]
        f0 = int(banks[0].top_rate_hz)
        B = push_s * f0
        total = (warm_pushes(warmup, graphs) + steps + min(steps, 16)) * push_s
        strains = [synth.white_noise(int(total * f0), 3, rank, det) for det in (0, 1)]
        dev = [torch.from_numpy(s).cuda() for s in strains]
        r = device_arm(lloid, torch, stream, local, banks, precision, B, steps, warmup, dev, graphs, autotune,
                       barrier, flush)
        tpl = sum(2 * b.n_templates for b in banks) * push_s * steps
        r["value"], r["dev_s"] = job_rate(tpl, r["dev_s"], dist, "cuda")
        r["banks"], r["B_s"] = banks, push_s
        r["templates"] = sum(2 * b.n_templates for b in banks)
        return r

    if args.workload == "batch":                      # the grouped batch alone as the line
        r = batch_run(args.precision, args.bins, args.steps, args.warmup, args.push_seconds)
        flops, bytes_, inter = model_sum([(b, 2) for b in r["banks"]], args.push_seconds, args.precision)
        dom, roofs = roofline_of(r["stages"], flops, bytes_, inter, args.precision, r["prof_steps"], peaks, "batch")
        busy = {k: v[0] for k, v in r["stages"].items() if v[1] > 0}
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * r["dev_s"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
                "data": "synthetic (seeded white noise; shape-only random banks)",
                "config": {"workload": f"batch: {args.bins} uneven SVD bins x 2 detectors (M logU[200,2000], "
                                       f"3-8 slices, 2-120 s templates, L logU[50,600]), one grouped push per step, "
                                       f"{args.push_seconds} s pushes", "templates": r["templates"],
                           "units_per_gpu": r["n_units"], "setup_s": r["create_s"]},
                "roofline": roofs[dom], "roofline_stages": roofs, "gpu_launches": r["launches"],
                "clocks": r["clocks"],
                "stages_ms_share": {k: round(v / sum(busy.values()), 4) for k, v in busy.items()}}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- headline: the production bin x 2 detectors
    spec, h = production_bank_templates(rank, args.templates)
    bank = lloid.decompose(h, spec.top_rate_hz, spec.slices)
    if args.xi2 == "off":
        bank.autocorr = None
    f0 = int(spec.top_rate_hz)
    B = args.push_seconds * f0
    n_prof = min(args.steps, 16)
    total_s = (warm_pushes(args.warmup, graphs) + args.steps + n_prof) * args.push_seconds
    strains = [make_strain(rank, det, total_s, f0, h, spec.n_templates) for det in (0, 1)]
    dev = [torch.from_numpy(s).cuda() for s in strains]
    tpl_s_rank = 2 * spec.n_templates * args.push_seconds * args.steps

    def prod_arm(precision, push_s=args.push_seconds, steps=args.steps):
        r = device_arm(lloid, torch, stream, local, [bank], precision, push_s * f0, steps, args.warmup, dev, graphs,
                       autotune, barrier, flush)
        r["value"], r["dev_s"] = job_rate(2 * spec.n_templates * push_s * steps, r["dev_s"], dist, "cuda")
        return r

    prim = prod_arm(args.precision)
    others = {}
    for p in args.compare.split(","):
        p = p.strip()
        if p and p != "none" and p != args.precision:
            others[p] = prod_arm(p)

    # e2e: host strain in, triggers out, through the C ABI
    ctx2 = lloid.Context(local, stream=stream.cuda_stream)
    ctx2.graphs(graphs)
    ctx2.autotune(autotune)
    u2 = make_units_for(ctx2, [bank], args.precision, B)
    t2 = 0
    for _ in range(warm_pushes(args.warmup, graphs)):
        ctx2.push_group(u2, [strains[det][t2:t2 + B] for det in (0, 1)], [t2] * 2, False)
        ctx2.pop_triggers()
        t2 += B
    barrier()
    s0 = ctx2.stats()
    w1 = time.perf_counter()
    for i in range(args.steps):
        ctx2.push_group(u2, [strains[det][t2:t2 + B] for det in (0, 1)], [t2] * 2, False)
        ctx2.pop_triggers()
        t2 += B
    ctx2.sync()
    ctx2.pop_triggers()
    e2e_wall = time.perf_counter() - w1
    s1 = ctx2.stats()
    e2e_value, e2e_wall = job_rate(tpl_s_rank, e2e_wall, dist, "cuda")
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": (s1["h2d_bytes"] - s0["h2d_bytes"]) // args.steps,
           "d2h_bytes_per_step": (s1["d2h_bytes"] - s0["d2h_bytes"]) // args.steps}
    ctx2.close()

    flops, bytes_, inter = model_sum([(bank, 2)], args.push_seconds, args.precision)
    flops["refine"], bytes_["refine"] = 0.0, 0.0          # data-dependent: no fixed algorithmic work
    dom, roofs = roofline_of(prim["stages"], flops, bytes_, inter, args.precision, prim["prof_steps"], peaks)
    busy = {k: v[0] for k, v in prim["stages"].items() if v[1] > 0}
    total_stage_ms = sum(busy.values())
    config = production_config(spec, bank.basis_counts(), args.push_seconds)
    line = {"metric": METRIC, "value": prim["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * prim["dev_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded white noise, random-parameter Newtonian chirp bank, injections)",
            "config": config,
            "run": {"setup_s": prim["create_s"], "precision": args.precision,
                    "parallelism": f"units sharded, {world} GPU(s)", "cuda_graphs": args.graphs,
                    "mix_autotune": args.autotune, "xi2": args.xi2,
                    "l2": "flushed between steps (256 MB write outside the step events)",
                    "host_ahead": "2-ms device spin before each step's start event (host enqueue outside the events)",
                    "warmup_pushes": warm_pushes(args.warmup, graphs), "step_ms": prim["step_ms"]},
            "roofline": roofs[dom], "roofline_stages": roofs, "e2e": e2e, "gpu_launches": prim["launches"],
            "clocks": prim["clocks"],
            "stages_ms_share": {k: round(v / total_stage_ms, 4) for k, v in busy.items()},
            "by_precision": {p: {"value": r["value"], "ms_per_step": 1e3 * r["dev_s"] / args.steps,
                                 "gain_vs_fp32": None}
                             for p, r in [(args.precision, prim), *others.items()]},
            "autotune": prim["autotune"],
            "wall_s": prim["wall"], "triggers": prim["triggers"],
            "refine_candidates_per_step": prim["refine_candidates"] / args.steps}
    if "fp32" in line["by_precision"]:
        ref = line["by_precision"]["fp32"]["value"]
        for p in line["by_precision"]:
            line["by_precision"][p]["gain_vs_fp32"] = line["by_precision"][p]["value"] / ref
    subs = [s.strip() for s in args.sub.split(",") if s.strip() and s.strip() != "none"]
    if "push1s" in subs:                              # the same bin with 1-s buffers (weights re-read per second)
        r1 = prod_arm(args.precision, push_s=1, steps=4 * args.steps)
        f1, b1, i1 = model_sum([(bank, 2)], 1, args.precision)
        _, roof1 = roofline_of(r1["stages"], f1, b1, i1, args.precision, r1["prof_steps"], peaks)
        line["push_1s"] = {"value": r1["value"], "ms_per_step": 1e3 * r1["dev_s"] / (4 * args.steps),
                           "steps": 4 * args.steps, "precision": args.precision,
                           "mix_frac": roof1.get("mix", {}).get("frac"), "clocks": r1["clocks"]}
    if "batch" in subs:                               # grouped batch of uneven bins (one launch per stage)
        tb = time.perf_counter()
        rb = batch_run(args.precision, args.bins, args.batch_steps, 2, args.batch_push_seconds)
        fb, bb, ib = model_sum([(b, 2) for b in rb["banks"]], args.batch_push_seconds, args.precision)
        _, roofb = roofline_of(rb["stages"], fb, bb, ib, args.precision, rb["prof_steps"], peaks, "batch")
        bbusy = {k: v[0] for k, v in rb["stages"].items() if v[1] > 0}
        line["batch"] = {"value": rb["value"], "ms_per_step": 1e3 * rb["dev_s"] / args.batch_steps,
                         "steps": args.batch_steps, "precision": args.precision,
                         "workload": f"{args.bins} uneven SVD bins x 2 detectors ({rb['n_units']} units, "
                                     f"{rb['templates']} templates; M logU[200,2000], 3-8 slices, 2-120 s "
                                     f"templates, L logU[50,600]), one grouped push of {args.batch_push_seconds} s "
                                     f"per step, every stage one launch over all units",
                         "gain_vs_fp32_production": None, "setup_s": rb["create_s"],
                         "run_s": time.perf_counter() - tb, "gpu_launches_per_step": rb["launches"] / args.batch_steps,
                         "roofline_stages": roofb, "clocks": rb["clocks"],
                         "stages_ms_share": {k: round(v / sum(bbusy.values()), 4) for k, v in bbusy.items()}}
        del rb
    if "paper" in subs:                               # the paper's benchmark shape: throughput vs banks
        line["paper_banks"] = paper_sweep(lloid, torch, stream, local, args, rank, world, dist, barrier, flush,
                                          graphs, autotune, peaks)
    if "serve" in subs:                               # the serving loop, 1-s buffers, p50 / p99 latency
        line["serve"] = {}
        for p in [x.strip() for x in args.serve_precisions.split(",") if x.strip()]:
            s = merge_serve(serve_once(lloid, serve, args, p, rank, world, local), dist)
            line["serve"][p] = {"template_s_per_s": s["template_seconds_per_s"], "p50_latency_s": s["p50_latency_s"],
                                "p99_latency_s": s["p99_latency_s"], "max_latency_s": s["max_latency_s"],
                                "buffers": s["buffers"], "pushes": s["pushes"], "wall_s": s["wall_s"],
                                "bank_load_s": s["bank_load_s"], "max_concurrent_streams": s["max_concurrent_streams"],
                                "workload": f"{args.serve_bins} bins x 2 detectors, 1-s buffers, Poisson arrivals "
                                            f"(1/s per stream) for {args.serve_seconds} s, real time"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ob = oracle_bank(h, spec)
        line["cpu_baseline"] = cpu_baseline(ob, spec, args.cpu_seconds, cpu_workers(args.cpu_seconds))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
