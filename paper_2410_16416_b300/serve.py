"""Streaming serving loop with continuous batching over the C ABI (host-side scheduler).

Strain arrives as short buffers (1 s by default) for many (SVD bin, detector)
streams.  Every stream is one unit of the library: its FIR histories,
resampler state and open trigger windows stay resident on the device between
buffers.  The loop

* admits a stream when its first buffer is due and the context's HBM budget
  can hold its unit (``svdbank_create`` returns SB_EBUSY otherwise; the stream
  waits and is retried whenever a finished stream frees its unit);
* on every tick pushes the next due buffer of every admitted stream as ONE
  grouped push (``filter_push_group``), so streams that arrived while others
  were on the GPU simply join the next group (continuous batching) and their
  work overlaps on the device;
* records, per buffer, the latency from its arrival to the moment the push that
  carried it has finished and its triggers are host-visible
  (``sb_ctx_progress``), and drains triggers (``triggers_pop``).

Every step of the filter runs in the library; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import _abi


@dataclasses.dataclass
class StreamRequest:
    """One (bin, detector) stream: ``n_buffers`` buffers, buffer j due at ``arrivals[j]`` seconds."""
    name: str
    bank: object
    detector: int
    arrivals: np.ndarray                        # non-decreasing, seconds from the loop's start
    strain: Callable[[int], np.ndarray]         # j -> FP32 buffer j (n samples)
    unit_kwargs: dict = dataclasses.field(default_factory=dict)
    share_key: Optional[str] = None             # streams with the same key share one bank on the device


@dataclasses.dataclass
class ServeReport:
    latencies_s: np.ndarray
    triggers: np.ndarray
    trigger_stream: np.ndarray                  # index of the request each trigger belongs to
    wall_s: float
    template_seconds: float
    pushes: int
    admitted_late: int                          # streams that waited for memory at least once
    max_concurrent: int

    def summary(self) -> dict:
        lat = self.latencies_s
        return {"p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
                "max_latency_s": float(lat.max()) if lat.size else None,
                "buffers": int(lat.size), "pushes": self.pushes, "wall_s": self.wall_s,
                "template_seconds_per_s": self.template_seconds / self.wall_s if self.wall_s else None,
                "streams_admitted_late": self.admitted_late, "max_concurrent_streams": self.max_concurrent,
                "triggers": int(self.triggers.size)}


def poisson_arrivals(rng: np.random.Generator, n: int, start_s: float, rate_hz: float = 1.0) -> np.ndarray:
    """Arrival times of n buffers: a Poisson process of the given rate starting at start_s."""
    return start_s + np.cumsum(rng.exponential(1.0 / rate_hz, n))


def preload(ctx: "_abi.Context", requests: List[StreamRequest], buffer_samples: int) -> Dict[str, "_abi.Unit"]:
    """Load each shared bank once, before serving starts (a resident unit per share_key
    that streams then clone with svdbank_create_like).

    Also switches the context's mixing-kernel autotuner off: timing a new launch shape
    synchronises the stream, and in a serving loop the group shapes keep changing, so the
    tuning would land in the latency tail (measured: p99 0.39 s with it, 0.04 s without, for
    1000 bins x 2 detectors of 1-s buffers).  The built-in pipeline shapes are used."""
    ctx.autotune(False)
    anchors: Dict[str, "_abi.Unit"] = {}
    for req in requests:
        if req.share_key is not None and req.share_key not in anchors:
            anchors[req.share_key] = ctx.create_unit(req.bank, detector=req.detector,
                                                     max_push_samples=buffer_samples, **req.unit_kwargs)
    return anchors


def run(ctx: "_abi.Context", requests: List[StreamRequest], buffer_samples: int,
        time_scale: float = 1.0, on_device: bool = False, idle_sleep_s: float = 0.0005,
        max_wall_s: Optional[float] = None, anchors: Optional[Dict[str, "_abi.Unit"]] = None) -> ServeReport:
    """Serve all requests to completion.  time_scale > 1 replays arrivals faster than real time.
    anchors: preloaded units (see preload) that streams with the same share_key clone."""
    anchors = anchors or {}
    n_req = len(requests)
    units: Dict[int, "_abi.Unit"] = {}
    next_buf = [0] * n_req
    waiting = list(range(n_req))                 # not yet admitted (in arrival order of first buffer)
    waiting.sort(key=lambda r: requests[r].arrivals[0])
    waited = set()
    finished = set()
    inflight: List[tuple] = []                  # (push_seq, [(req, arrival_time)])
    last_push_of: Dict[int, int] = {}
    latencies: List[float] = []
    trig_chunks: List[np.ndarray] = []
    unit_to_req: Dict[int, int] = {}
    shared: Dict[str, List[int]] = {}           # share_key -> admitted requests holding that bank
    pushes = 0
    max_conc = 0
    tpl_s = 0.0
    t0 = time.perf_counter()

    def now() -> float:
        return (time.perf_counter() - t0) * time_scale

    def drain():
        nonlocal inflight
        _, done = ctx.progress()
        keep = []
        tnow = now()
        for seq, bufs in inflight:
            if seq < done:
                latencies.extend((tnow - a) / time_scale for _, a in bufs)
            else:
                keep.append((seq, bufs))
        inflight = keep
        tr = ctx.pop_triggers()
        if tr.size:
            trig_chunks.append(tr)
        return done

    while len(finished) < n_req:
        if max_wall_s is not None and time.perf_counter() - t0 > max_wall_s:
            break
        tnow = now()
        # admission: streams whose first buffer is due, while the budget holds them
        still = []
        for r in waiting:
            if requests[r].arrivals[0] > tnow:
                still.append(r)
                continue
            key = requests[r].share_key
            try:
                if key is not None and key in anchors:
                    u = ctx.create_like(anchors[key], detector=requests[r].detector)
                elif key is not None and shared.get(key):
                    u = ctx.create_like(units[shared[key][0]], detector=requests[r].detector)
                else:
                    u = ctx.create_unit(requests[r].bank, detector=requests[r].detector,
                                        max_push_samples=buffer_samples, **requests[r].unit_kwargs)
            except _abi.LloidError as e:
                if e.code != _abi.SB_EBUSY:
                    raise
                waited.add(r)
                still.append(r)
                continue
            units[r] = u
            unit_to_req[u.info().unit] = r
            if key is not None:
                shared.setdefault(key, []).append(r)
        waiting = still
        max_conc = max(max_conc, len(units))
        # one grouped push of every admitted stream's next due buffer
        group, strains, t0s, bufs = [], [], [], []
        for r, u in units.items():
            j = next_buf[r]
            if j < len(requests[r].arrivals) and requests[r].arrivals[j] <= tnow:
                group.append(u)
                strains.append(requests[r].strain(j))
                t0s.append(j * buffer_samples)
                bufs.append((r, float(requests[r].arrivals[j])))
        if group:
            ctx.push_group(group, strains, t0s, on_device)
            for r, _ in bufs:
                next_buf[r] += 1
                last_push_of[r] = pushes
                tpl_s += requests[r].bank.n_templates * buffer_samples / requests[r].bank.top_rate_hz
            inflight.append((pushes, bufs))
            pushes += 1
        done = drain()
        # retire streams whose last buffer's push has completed: frees their memory
        for r in list(units):
            if next_buf[r] == len(requests[r].arrivals) and last_push_of.get(r, -1) < done:
                units[r].destroy()
                del units[r]
                finished.add(r)
                key = requests[r].share_key
                if key is not None:
                    shared[key].remove(r)
        if not group:
            time.sleep(idle_sleep_s)
    ctx.sync()
    drain()
    wall = time.perf_counter() - t0
    trig = np.concatenate(trig_chunks) if trig_chunks else np.empty(0, dtype=_abi.TRIGGER_DTYPE)
    owner = np.array([unit_to_req.get(int(u), -1) for u in trig["unit"]], dtype=np.int64)
    return ServeReport(np.array(latencies), trig, owner, wall, tpl_s, pushes, len(waited), max_conc)
