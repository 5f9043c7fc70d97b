#!/usr/bin/env python
"""Throughput benchmark: template-seconds filtered per second on B300 (paper Eq. 1, cores = 1 per GPU).

Workload (per GPU rank): one production-shaped SVD bin of 1000 templates
(60 s Newtonian chirps, chirp mass 1.0-1.5 Msun, six time slices at 4096 ...
128 Hz, SVD truncated at 99.99% of sigma^2) on two detectors (H1, L1: two
units, independent seeded white noise, injections at SNR 8-30).  A step is one
grouped push of ``--push-seconds`` of strain to both units: decimation, basis
FIR, mixing, up-sampling + sum, window maxima and trigger hand-off.  Data are
synthetic (seeded white Gaussian noise; random-parameter chirps).

The device-timed value has the strain already resident in HBM; L2 is flushed
(256 MB write) between timed steps, outside the step's events.  ``e2e`` runs
the same steps through the C ABI from host buffers, with the host->device
strain copies and the trigger read-back inside the timed region.

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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=240)       # 240 + 16 pushes of 16 s = 4096 s of strain
    p.add_argument("--warmup", type=int, default=16)
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
    p.add_argument("--cpu-seconds", type=float, default=8.0, help="strain seconds per oracle worker")
    p.add_argument("--workload", default="production", choices=["production", "batch", "serve"],
                   help="production: one 1000-template bin x 2 detectors; batch: --bins uneven bins x 2 detectors")
    p.add_argument("--bins", type=int, default=200)
    p.add_argument("--serve-seconds", type=int, default=30, help="serve: 1-s buffers per stream")
    p.add_argument("--distinct-banks", type=int, default=20, help="serve: distinct banks the bins cycle through")
    p.add_argument("--time-scale", type=float, default=1.0, help="serve: arrival clock speed-up")
    return p.parse_args()


# ----------------------------------------------------------------------------- workload
def production_bank_templates(bin_index: int, n_templates: int):
    spec = synth.scaled_bin(synth.PRODUCTION_BIN, n_templates)
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s,
                               2, bin_index, 0)
    return spec, h


def make_strain(bin_index: int, detector: int, seconds: int, f0: float, h, n_templates: int):
    n = int(seconds * f0)
    d = synth.white_noise(n, 2, bin_index, detector + 1)
    for inj in synth.injection_plan(max(1, seconds // 80), n_templates, n, f0, 80.0, 8.0, 30.0, bin_index, detector):
        synth.inject(d, h, inj.template, inj.n_c, inj.amplitude, inj.phi0)
    return d


def algorithmic_model(bank, units: int, B_s: float, precision: str = "fp32"):
    """Per-stage algorithmic FLOPs and HBM bytes of one push (all units).

    Weights and basis outputs move in the operand width (4 bytes in FP32 mode,
    2 in the 16-bit modes, 1 in E4M3).  FP32 mode: SNR series are FP32, each
    level's is written once and read once by the interpolation stage.  16-bit
    and 8-bit modes: mixing and interpolation are one stage ("mix"); each level
    k >= 1 writes its y once and the next finer level reads it once (2 bytes per
    sample, one FP16 plane, in BF16 and E4M3 modes; 4 bytes, BF16 hi + lo, in
    FP16 mode); the top level writes only per-window partial maxima (two 24-byte
    records per template and 128 samples).  Interpolation FLOPs are
    the halfband filter's own (about 17 per output), however it is executed."""
    w = {"fp32": 4.0, "bf16": 2.0, "fp16": 2.0, "fp8": 1.0}[precision]
    fused = precision != "fp32"
    yb = 4.0 if precision == "fp16" else 2.0                   # bytes per stored y sample
    f0 = bank.top_rate_hz
    M2 = 2 * bank.n_templates
    levels = {}
    for s in bank.slices:
        k = int(round(math.log2(f0 / s.rate_hz)))
        levels.setdefault(k, []).append(s)
    kmax = max(levels)
    fl = {k: 0.0 for k in ("fir", "mix", "upsample", "decimate", "trigger")}
    by = {k: 0.0 for k in fl}
    for s in bank.slices:
        L, Q = s.basis.shape
        N = B_s * s.rate_hz
        fl["fir"] += 2.0 * L * Q * N
        by["fir"] += w * (L * Q + N + L * N)
    for k, ss in levels.items():
        Lk = sum(s.basis.shape[0] for s in ss)
        N = B_s * f0 / 2 ** k
        fl["mix"] += 2.0 * M2 * Lk * N
        if fused:
            by["mix"] += w * (M2 * Lk + Lk * N) + (2 * yb * M2 * N if k >= 1 else 0.0)
        else:
            by["mix"] += w * (M2 * Lk + Lk * N) + 4.0 * M2 * N * (2 if k < kmax else 1)
    if fused:
        by["mix"] += (M2 / 2) * (B_s * f0 / 128) * 2 * 24.0          # top-level window records
    for k in range(1, kmax + 1):
        N = B_s * f0 / 2 ** k
        if fused:
            fl["mix"] += M2 * (2 * N) * 17                            # the halfband filter's own work
        else:
            fl["upsample"] += M2 * (2 * N) * 17
            by["upsample"] += 4.0 * M2 * (N + 2 * N)
        fl["decimate"] += 2 * N * 17
        by["decimate"] += 4.0 * (3 * N)
    fl["trigger"] = 3.0 * M2 / 2 * B_s * f0
    by["trigger"] = 4.0 * M2 * B_s * f0
    return {k: fl[k] * units for k in fl}, {k: by[k] * units for k in by}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle (CPU)
BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_worker(args):
    """One oracle run (FP64): SVD path + window maxima on a strain excerpt."""
    bank, strain, win_len, threshold = args
    import oracle
    t = time.perf_counter()
    x = oracle.lloid_snr(bank, strain)
    oracle.triggers(x, win_len, threshold, x.shape[1])
    return time.perf_counter() - t


def _blas_threads() -> int:
    """Threads numpy's BLAS uses in this process (threadpoolctl when present)."""
    try:
        from threadpoolctl import threadpool_info
        n = [p.get("num_threads", 1) for p in threadpool_info() if p.get("user_api") == "blas"]
        return max(n) if n else 1
    except ImportError:
        v = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
        return int(v) if v else (os.cpu_count() or 1)


def oracle_bank(h, spec):
    import oracle
    return oracle.build_bank(h, spec.top_rate_hz, spec.slices)


def cpu_baseline(h, spec, seconds: float, workers: int):
    """The oracle as it stands on `workers` host processes, each on its own excerpt."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ob = oracle_bank(h, spec)
    f0 = spec.top_rate_hz
    n = int(seconds * f0) // 32 * 32
    jobs = [(ob, synth.white_noise(n, 7, w, 0), int(f0), 6.0) for w in range(workers)]
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in BLAS_ENV}
    for k in BLAS_ENV:                       # children read these when they import numpy
        os.environ[k] = "1"
    try:
        t = time.perf_counter()
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            list(ex.map(_oracle_worker, jobs))
        wall = time.perf_counter() - t
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    value = workers * spec.n_templates * (n / f0) / wall
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} processes x {n / f0:.0f} s excerpt of one unit of the production bin "
                      f"({spec.n_templates} templates), FP64 SVD path + window maxima, BLAS 1 thread each; "
                      f"wall {wall:.1f} s incl. process start"}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric and workload shape."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, h = production_bank_templates(0, args.templates)
    ob = oracle_bank(h, spec)
    f0 = spec.top_rate_hz
    n = int(min(args.cpu_seconds, 4.0) * f0) // 32 * 32
    times = []
    for step in range(args.warmup + args.steps):
        d = synth.white_noise(n, 8, 0, step)
        dt = _oracle_worker((ob, d, int(f0), 6.0))
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * spec.n_templates * (n / f0) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"production bin ({spec.n_templates} templates, 6 slices 4096-128 Hz), "
                                   f"one unit, {n / f0:.0f} s excerpt per step", "templates": spec.n_templates},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                             "sample": f"{n / f0:.0f} s excerpt of one unit per step, one process"},
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


def roofline_of(stages, flops, bytes_, precision, steps, peaks, workload="production"):
    """Bound, achieved and fraction of the stage that takes the most device time among the stages
    with an algorithmic model (the refinement's work depends on how many candidates the data
    produce, so it has none and is reported through its time share only)."""
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12            # FP32 FFMA lanes x 2 FLOP x max clock
    tensor_peak = peaks.get("bf16_tflops", 1800.0)             # dense BF16 = FP16 rate, burst (short steps)
    busy = {k: v[0] for k, v in stages.items() if v[1] > 0 and (flops.get(k, 0.0) > 0 or bytes_.get(k, 0.0) > 0)}
    dom = max(busy, key=busy.get)
    dom_ms, _ = stages[dom]
    on_tensor = precision in ("bf16", "fp16") and dom in ("fir", "mix")
    cpeak = tensor_peak if on_tensor else alu_peak
    t_c = flops.get(dom, 0.0) / (cpeak * 1e12)
    t_m = bytes_.get(dom, 0.0) / (hbm_peak * 1e9)
    secs = dom_ms / 1e3
    if t_c >= t_m:
        ach = flops[dom] * steps / secs / 1e12
        return dom, {"bound": "tensor" if on_tensor else "alu", "achieved": ach, "peak": cpeak, "unit": "TFLOP/s",
                     "frac": ach / cpeak, "traffic": None, "kernel": dom,
                     "peak_source": "measured bf16_tflops (burst)" if on_tensor else
                     "derived: 148 SM x 128 FP32 lanes x 2 FLOP x max SM clock"}
    ach = bytes_[dom] * steps / secs / 1e9
    return dom, {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                 "traffic": measured_traffic(dom, workload, precision), "algorithmic_bytes": bytes_[dom],
                 "kernel": dom, "peak_source": "measured hbm_gbs"}


def run_serve(args):
    """Streaming serving loop: bins x 2 detectors of 1-s buffers arriving as Poisson processes."""
    import torch
    import paper_2410_16416_b300 as lloid
    from paper_2410_16416_b300 import serve
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:                                     # ranks serve disjoint bins; only the report is reduced
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    banks = [synth.production_shape_bank(i) for i in range(args.distinct_banks)]
    g = np.random.default_rng(20241016 + rank)
    reqs = []
    for b in shard_bins(args.bins, rank, world):
        bank = banks[b % len(banks)]
        for det in (0, 1):
            reqs.append(serve.StreamRequest(
                name=f"bin{b}-det{det}", bank=bank, detector=det,
                arrivals=serve.poisson_arrivals(g, args.serve_seconds, float(g.uniform(0.0, 5.0))),
                strain=(lambda j, b=b, det=det: synth.white_noise_block(j, 4096, 9, b, det)),
                unit_kwargs=dict(precision=args.precision, threshold=6.0, refine_threshold=5.5),
                share_key=f"bank{b % len(banks)}"))
    ctx = lloid.Context(int(os.environ.get("LOCAL_RANK", "0")))
    tl = time.perf_counter()
    anchors = serve.preload(ctx, reqs, 4096)          # banks are loaded before data arrive
    load_s = time.perf_counter() - tl
    rep = serve.run(ctx, reqs, 4096, time_scale=args.time_scale, anchors=anchors)
    st = ctx.stats()
    ctx.close()
    s = rep.summary()
    value, wall = job_rate(rep.template_seconds, rep.wall_s, dist, "cuda")
    p99 = s["p99_latency_s"] or 0.0
    if dist is not None:                              # the slowest rank's p99 and max (a conservative merge)
        lat = torch.tensor([p99, s["max_latency_s"] or 0.0], dtype=torch.float64, device="cuda")
        dist.all_reduce(lat, op=dist.ReduceOp.MAX)
        p99, s["max_latency_s"] = float(lat[0]), float(lat[1])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": s["pushes"], "warmup": 0, "ms_per_step": 1e3 * s["wall_s"] / max(1, s["pushes"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}[args.precision],
            "data": "synthetic (seeded white noise per (bin, detector, buffer); production-shaped random banks)",
            "config": {"workload": f"serve: {args.bins} bins x 2 detectors, 1-s buffers, Poisson arrivals "
                                   f"(1/s per stream) for {args.serve_seconds} s, banks cycled from "
                                   f"{len(banks)} production-shaped banks (~1000 templates, 6 slices)",
                       "time_scale": args.time_scale, "precision": args.precision,
                       "bank_load_s": load_s},
            "latency": {"p50_s": s["p50_latency_s"], "p99_s": p99, "max_s": s["max_latency_s"],
                        "buffers": s["buffers"], "definition": "buffer arrival -> its push finished and its "
                                                               "triggers host-visible"},
            "serving": s, "gpu_launches": st["kernel_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    import torch
    import paper_2410_16416_b300 as lloid

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

    if args.workload == "production":
        spec, h = production_bank_templates(rank, args.templates)
        bank = lloid.decompose(h, spec.top_rate_hz, spec.slices)
        if args.xi2 == "off":
            bank.autocorr = None
        banks = [bank]
        f0 = int(spec.top_rate_hz)
    else:                       # uneven shape-only bins; rank r takes bins r, r + world, ...
        banks = [synth.shape_only_bank(b) for b in shard_bins(args.bins, rank, world)]
        spec, h, bank = None, None, banks[0]
        f0 = int(banks[0].top_rate_hz)
    B = args.push_seconds * f0
    n_prof = min(args.steps, 16)                       # profiled pushes after the timed ones (stage split)
    total_s = (args.warmup + args.steps + n_prof) * args.push_seconds
    if spec is not None:
        strains = [make_strain(rank, det, total_s, f0, h, spec.n_templates) for det in (0, 1)]
    else:                       # every bank of a detector filters that detector's strain
        strains = [synth.white_noise(int(total_s * f0), 3, rank, det) for det in (0, 1)]
    dev = [torch.from_numpy(s).cuda() for s in strains]
    unit_specs = [(b, det) for b in banks for det in (0, 1)]
    n_templates_all = sum(b.n_templates for b, _ in unit_specs)
    # One non-default stream for the library, the L2 flush and the timing events.
    # (torch's default stream has handle 0, which the C ABI reads as "no stream".)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    n_units = len(unit_specs)
    tpl_s_rank = n_templates_all * args.push_seconds * args.steps

    def make_units(ctx, precision):
        # the two detectors of a bin share one copy of the bank's device data (svdbank_create_like)
        units = []
        for b in banks:
            u0 = ctx.create_unit(b, detector=0, precision=precision, threshold=6.0, refine_threshold=5.5,
                                 window_s=1.0, max_push_samples=B)
            units += [u0, ctx.create_like(u0, detector=1)]
        return units

    def device_arm(precision):
        ctx = lloid.Context(local, stream=stream.cuda_stream)
        ctx.graphs(args.graphs == "on")
        ctx.autotune(args.autotune == "on")
        tc0 = time.perf_counter()
        units = make_units(ctx, precision)
        create_s = time.perf_counter() - tc0
        dets = [det for _, det in unit_specs]
        t = 0
        for _ in range(args.warmup):
            ctx.push_group(units, [dev[det][t:t + B] for det in dets], [t] * n_units, True)
            t += B
        ctx.pop_triggers()
        barrier()
        st0 = ctx.stats()
        clocks = ClockSampler(local)
        clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        w0 = time.perf_counter()
        for i in range(args.steps):
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
        value, dev_s = job_rate(tpl_s_rank, sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, "cuda")
        trig = ctx.pop_triggers()
        tuned = ctx.autotune_choices()
        ctx.close()
        return {"value": value, "autotune": {"choices": tuned, "timed_launches": st1["autotune_launches"],
                                             "in_timed_region": st1["autotune_launches"] - st0["autotune_launches"]}, "dev_s": dev_s, "wall": wall, "clocks": clk, "create_s": create_s,
                "stages": stages, "launches": st1["kernel_launches"] - st0["kernel_launches"],
                "refine_candidates": st1["refine_candidates"] - st0["refine_candidates"], "prof_steps": n_prof,
                "triggers": int(len(trig))}

    prim = device_arm(args.precision)
    others = {}
    for p in args.compare.split(","):
        p = p.strip()
        if p and p != "none" and p != args.precision:
            others[p] = device_arm(p)

    # e2e: host strain in, triggers out, through the C ABI
    ctx2 = lloid.Context(local, stream=stream.cuda_stream)
    ctx2.graphs(args.graphs == "on")
    ctx2.autotune(args.autotune == "on")
    u2 = make_units(ctx2, args.precision)
    dets = [det for _, det in unit_specs]
    t2 = 0
    for _ in range(args.warmup):
        ctx2.push_group(u2, [strains[det][t2:t2 + B] for det in dets], [t2] * n_units, False)
        ctx2.pop_triggers()
        t2 += B
    barrier()
    s0 = ctx2.stats()
    w1 = time.perf_counter()
    for i in range(args.steps):
        ctx2.push_group(u2, [strains[det][t2:t2 + B] for det in dets], [t2] * n_units, False)
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

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    flops, bytes_ = {}, {}
    for b, _ in unit_specs:
        f1, b1 = algorithmic_model(b, 1, args.push_seconds, args.precision)
        for k in f1:
            flops[k] = flops.get(k, 0.0) + f1[k]
            bytes_[k] = bytes_.get(k, 0.0) + b1[k]
    flops["refine"], bytes_["refine"] = 0.0, 0.0          # data-dependent: no fixed algorithmic work
    dom, roof = roofline_of(prim["stages"], flops, bytes_, args.precision, prim["prof_steps"], peaks, args.workload)
    busy = {k: v[0] for k, v in prim["stages"].items() if v[1] > 0}
    total_stage_ms = sum(busy.values())
    line = {"metric": METRIC, "value": prim["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * prim["dev_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}[args.precision],
            "data": "synthetic (seeded white noise, random-parameter Newtonian chirp bank, injections)",
            "config": {"workload": (f"production bin: {spec.n_templates} templates x 2 detectors, 6 slices "
                                    f"4096-128 Hz, L={bank.basis_counts()}, {args.push_seconds} s pushes")
                       if spec is not None else
                       (f"batch: {len(banks)} uneven SVD bins x 2 detectors ({n_units} units, "
                        f"{n_templates_all} templates; M logU[200,2000], 3-8 slices, 2-120 s templates, "
                        f"L logU[50,600]), one grouped push per step, {args.push_seconds} s pushes"),
                       "templates": n_templates_all, "units_per_gpu": n_units, "setup_s": prim["create_s"],
                       "push_seconds": args.push_seconds, "precision": args.precision,
                       "parallelism": f"units sharded, {world} GPU(s)", "cuda_graphs": args.graphs,
                       "mix_autotune": args.autotune,
                       "xi2": args.xi2 if spec is not None else "off",
                       "l2": "flushed between steps (256 MB write outside the step events)"},
            "roofline": roof, "e2e": e2e, "gpu_launches": prim["launches"], "clocks": prim["clocks"],
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline and spec is not None:
        line["cpu_baseline"] = cpu_baseline(h, spec, args.cpu_seconds, max(1, min(os.cpu_count() or 1, 16)))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
