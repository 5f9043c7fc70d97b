"""ctypes binding of ``liblloid.so`` (include/lloid.h): argument marshalling only.

Every step of the filter runs in the library's CUDA kernels; this module only
converts Python/numpy/torch arguments into the C structures and pointers the
C ABI takes.  There is no CPU fallback: if the library is missing, importing
this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblloid.so")

SB_OK, SB_EINVAL, SB_ENOMEM, SB_EBUSY, SB_EGAP, SB_ETIMEOUT, SB_ECUDA, SB_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6, -7
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}
SB_FLAG_KEEP_SNR = 1
SB_TRIG_REFINED = 1
SB_TRIG_SUBSAMPLE = 2
SB_TRIG_XI2 = 4
SB_XI2_HALF = 16


class SbSlice(C.Structure):
    _fields_ = [("rate_hz", C.c_double), ("t_start_s", C.c_double), ("t_end_s", C.c_double),
                ("n_basis", C.c_int32), ("n_taps", C.c_int32),
                ("basis", C.POINTER(C.c_double)), ("mixing", C.POINTER(C.c_double))]


class SbDesc(C.Structure):
    _fields_ = [("n_templates", C.c_int32), ("n_slices", C.c_int32), ("top_rate_hz", C.c_double),
                ("slices", C.POINTER(SbSlice)), ("template_ids", C.POINTER(C.c_int64)),
                ("precision", C.c_int32), ("flags", C.c_int32), ("threshold", C.c_float),
                ("refine_threshold", C.c_float), ("window_s", C.c_double), ("max_push_samples", C.c_int64),
                ("autocorr", C.POINTER(C.c_double))]


class SbTrigger(C.Structure):
    _fields_ = [("unit", C.c_int64), ("template_id", C.c_int64), ("sample", C.c_int64), ("window", C.c_int64),
                ("snr", C.c_float), ("phase", C.c_float), ("snr_peak", C.c_float), ("dt_peak", C.c_float),
                ("flags", C.c_int32), ("xi2", C.c_float)]


class SbUnitInfo(C.Structure):
    _fields_ = [("unit", C.c_int64), ("n_templates", C.c_int32), ("n_slices", C.c_int32), ("k_max", C.c_int32),
                ("precision", C.c_int32), ("latency_samples", C.c_int64), ("samples_pushed", C.c_int64),
                ("device_bytes", C.c_int64), ("flops_per_second", C.c_int64)]


class SbCtxStats(C.Structure):
    _fields_ = [("pushes", C.c_int64), ("kernel_launches", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("triggers", C.c_int64), ("refine_candidates", C.c_int64),
                ("refine_dropped", C.c_int64), ("graph_launches", C.c_int64),
                ("autotune_shapes", C.c_int64), ("autotune_launches", C.c_int64)]


STAGES = ["history", "strain", "decimate", "fir", "upsample", "mix", "trigger", "snr_history", "refine"]

TRIGGER_DTYPE = np.dtype([("unit", "<i8"), ("template_id", "<i8"), ("sample", "<i8"), ("window", "<i8"),
                          ("snr", "<f4"), ("phase", "<f4"), ("snr_peak", "<f4"), ("dt_peak", "<f4"),
                          ("flags", "<i4"), ("xi2", "<f4")])
assert TRIGGER_DTYPE.itemsize == C.sizeof(SbTrigger)
COINC_DTYPE = np.dtype([("template_id", "<i8"), ("index_a", "<i8"), ("index_b", "<i8"), ("sample_a", "<i8"),
                        ("sample_b", "<i8"), ("snr_a", "<f4"), ("snr_b", "<f4"), ("network_snr", "<f4"),
                        ("reserved", "<i4")])

# name -> (restype, argtypes): every entry point declared in include/lloid.h
SIGNATURES = {
    "sb_ctx_create": (C.c_int, [C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    "sb_ctx_destroy": (C.c_int, [C.c_void_p]),
    "sb_ctx_sync": (C.c_int, [C.c_void_p]),
    "svdbank_create": (C.c_int, [C.c_void_p, C.POINTER(SbDesc), C.c_int32, C.POINTER(C.c_void_p)]),
    "svdbank_destroy": (C.c_int, [C.c_void_p]),
    "svdbank_create_like": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "sb_unit_query": (C.c_int, [C.c_void_p, C.POINTER(SbUnitInfo)]),
    "svdbank_plan": (C.c_int, [C.POINTER(SbDesc), C.POINTER(SbUnitInfo)]),
    "filter_push": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32]),
    "filter_push_group": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.c_int64, C.POINTER(C.c_int64), C.c_int32]),
    "triggers_pop": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "sb_ctx_progress": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sb_unit_snr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sb_ctx_get_stats": (C.c_int, [C.c_void_p, C.POINTER(SbCtxStats)]),
    "sb_ctx_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "sb_ctx_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "sb_ctx_autotune": (C.c_int, [C.c_void_p, C.c_int32]),
    "sb_ctx_autotune_choices": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "sb_ctx_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "sb_window_triggers_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                                             C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                             C.c_void_p]),
    "sb_coincidences": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_int64)]),
    "sb_cond_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "sb_cond_destroy": (C.c_int, [C.c_void_p]),
    "sb_cond_latency": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "sb_cond_push": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
    "sb_cond_psd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sb_ctx_test_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32]),
    "sb_last_error": (C.c_char_p, []),
}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2410_16416_b300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


class LloidError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.sb_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc != SB_OK:
        raise LloidError(rc, where)
    return rc


def _ptr(a) -> int:
    """Device or host data pointer of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_desc(bank, precision: str = "fp32", threshold: float = 6.0, refine_threshold: float = 0.0,
              window_s: float = 1.0, max_push_samples: int = 0, keep_snr: bool = False,
              template_ids: Optional[Sequence[int]] = None, autocorr=None):
    """(SbDesc, keep-alive list) for a bank; the arrays must outlive the C call.
    autocorr: [M, 2 SB_XI2_HALF + 1] complex (or the bank's `autocorr` attribute) for xi^2."""
    keep = []
    sl = (SbSlice * len(bank.slices))()
    for i, s in enumerate(bank.slices):
        basis = np.ascontiguousarray(s.basis, dtype=np.float64)
        mixing = np.ascontiguousarray(s.mixing, dtype=np.float64)
        keep += [basis, mixing]
        sl[i] = SbSlice(float(s.rate_hz), float(s.t_start_s), float(s.t_end_s), basis.shape[0], basis.shape[1],
                        basis.ctypes.data_as(C.POINTER(C.c_double)), mixing.ctypes.data_as(C.POINTER(C.c_double)))
    keep.append(sl)
    ids = None
    if template_ids is not None:
        ids = np.ascontiguousarray(template_ids, dtype=np.int64)
        keep.append(ids)
    if autocorr is None:
        autocorr = getattr(bank, "autocorr", None)
    ac = None
    if autocorr is not None:
        a = np.asarray(autocorr, dtype=np.complex128)
        if a.shape != (int(bank.n_templates), 2 * SB_XI2_HALF + 1):
            raise ValueError(f"autocorr must be [{bank.n_templates}, {2 * SB_XI2_HALF + 1}] complex")
        ac = np.ascontiguousarray(a).view(np.float64)
        keep.append(ac)
    d = SbDesc(int(bank.n_templates), len(bank.slices), float(bank.top_rate_hz), sl,
               ids.ctypes.data_as(C.POINTER(C.c_int64)) if ids is not None else None,
               PRECISION[precision], SB_FLAG_KEEP_SNR if keep_snr else 0, float(threshold),
               float(refine_threshold), float(window_s), int(max_push_samples),
               ac.ctypes.data_as(C.POINTER(C.c_double)) if ac is not None else None)
    return d, keep


def coincidences(trig_a: np.ndarray, trig_b: np.ndarray, max_dt_samples: int) -> np.ndarray:
    """sb_coincidences: same-template pairs of two detectors' triggers (TRIGGER_DTYPE arrays) within
    max_dt_samples; a COINC_DTYPE array ordered by (template_id, sample_a, sample_b, index_a, index_b)."""
    a = np.ascontiguousarray(trig_a, dtype=TRIGGER_DTYPE)
    b = np.ascontiguousarray(trig_b, dtype=TRIGGER_DTYPE)
    n = C.c_int64()
    cap = 64
    while True:
        out = np.empty(cap, dtype=COINC_DTYPE)
        rc = lib.sb_coincidences(a.ctypes.data if a.size else None, a.size, b.ctypes.data if b.size else None,
                                 b.size, int(max_dt_samples), out.ctypes.data, cap, C.byref(n))
        if rc == SB_EOVERFLOW and n.value > cap:
            cap = n.value
            continue
        _check(rc, "sb_coincidences")
        return out[: n.value]


def plan(bank, **kw) -> SbUnitInfo:
    """svdbank_plan: validate a bank and report latency, bytes and FLOPs (no device needed)."""
    d, keep = make_desc(bank, **kw)
    info = SbUnitInfo()
    _check(lib.svdbank_plan(C.byref(d), C.byref(info)), "svdbank_plan")
    return info


class Context:
    """sb_ctx: one device, one stream, one HBM budget, one trigger queue."""

    def __init__(self, device: int = 0, stream=None, hbm_budget_bytes: int = 0):
        """stream: a cudaStream_t handle (int) the library launches on; None or 0
        (torch's default stream) makes the library create its own stream."""
        h = C.c_void_p()
        s = None if not stream else C.c_void_p(int(stream))
        _check(lib.sb_ctx_create(device, s, int(hbm_budget_bytes), C.byref(h)), "sb_ctx_create")
        self.handle = h
        self.units: List["Unit"] = []

    def close(self):
        if self.handle:
            lib.sb_ctx_destroy(self.handle)       # also destroys the context's units
            self.handle = None
            for u in self.units:
                u.handle = None
            self.units = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        _check(lib.sb_ctx_sync(self.handle), "sb_ctx_sync")

    def progress(self):
        """(pushes issued, pushes completed with triggers host-visible); never blocks."""
        a, b = C.c_int64(), C.c_int64()
        _check(lib.sb_ctx_progress(self.handle, C.byref(a), C.byref(b)), "sb_ctx_progress")
        return a.value, b.value

    def stats(self) -> dict:
        st = SbCtxStats()
        _check(lib.sb_ctx_get_stats(self.handle, C.byref(st)), "sb_ctx_get_stats")
        return {k: getattr(st, k) for k, _ in SbCtxStats._fields_}

    def profile(self, enable: bool):
        _check(lib.sb_ctx_profile(self.handle, int(bool(enable))), "sb_ctx_profile")

    def graphs(self, enable: bool):
        """Capture every push into a CUDA graph (reused per group shape); results are unchanged."""
        _check(lib.sb_ctx_graphs(self.handle, int(bool(enable))), "sb_ctx_graphs")

    def test_wait(self, wait_limit_ns: int, skip_fir_chunk: int) -> None:
        """sb_ctx_test_wait: bound the basis-FIR kernel's waits and skip one K chunk's load (test hook)."""
        _check(lib.sb_ctx_test_wait(self.handle, int(wait_limit_ns), int(skip_fir_chunk)), "sb_ctx_test_wait")

    def autotune(self, enable: bool) -> None:
        """Time the mixing kernel's pipeline shapes on new launch shapes (default on)."""
        _check(lib.sb_ctx_autotune(self.handle, int(bool(enable))), "sb_ctx_autotune")

    def autotune_choices(self) -> list:
        """[{key, mode, store_y, interp, k_chunks, k_bytes, log4_tiles, stages, u_buffers, window_ring}]
        tuned so far."""
        n = lib.sb_ctx_autotune_choices(self.handle, None, 0)
        _check(min(n, 0), "sb_ctx_autotune_choices")
        buf = (C.c_int32 * (4 * max(n, 1)))()
        n = lib.sb_ctx_autotune_choices(self.handle, buf, n)
        _check(min(n, 0), "sb_ctx_autotune_choices")
        out = []
        for i in range(n):
            k = buf[4 * i]
            out.append({"key": k, "mode": ("fp16", "bf16", "?", "?")[k & 3], "store_y": bool(k & 4),
                        "interp": bool(k & 8), "k_chunks": (k >> 4) & 3, "k_bytes": (32, 64, 128, 0)[(k >> 6) & 3],
                        "log4_tiles": k >> 8, "stages": buf[4 * i + 1], "u_buffers": buf[4 * i + 2],
                        "window_ring": buf[4 * i + 3]})
        return out

    def stage_times(self) -> dict:
        """{stage: (ms summed over launches, launches)} since profile(True); blocks."""
        n = len(STAGES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        _check(lib.sb_ctx_stage_times(self.handle, ms, cnt, n), "sb_ctx_stage_times")
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(n)}

    def create_unit(self, bank, detector: int = 0, **kw) -> "Unit":
        """svdbank_create from any bank with n_templates, top_rate_hz and slices
        (rate_hz, t_start_s, t_end_s, basis [L, Q], mixing [2M, L]); keywords as make_desc."""
        d, keep = make_desc(bank, **kw)
        h = C.c_void_p()
        _check(lib.svdbank_create(self.handle, C.byref(d), int(detector), C.byref(h)), "svdbank_create")
        u = Unit(self, h)
        self.units.append(u)
        return u

    def create_like(self, src: "Unit", detector: int = 0) -> "Unit":
        """svdbank_create_like: a unit sharing src's bank data, with its own streaming state."""
        h = C.c_void_p()
        _check(lib.svdbank_create_like(self.handle, src.handle, int(detector), C.byref(h)), "svdbank_create_like")
        u = Unit(self, h)
        self.units.append(u)
        return u

    def push_group(self, units: Sequence["Unit"], strains: Sequence, t0: Sequence[int], on_device: bool):
        n = len(units)
        hs = (C.c_void_p * n)(*[u.handle.value for u in units])
        ps = (C.c_void_p * n)(*[_ptr(s) for s in strains])
        ts = (C.c_int64 * n)(*[int(t) for t in t0])
        ns = int(strains[0].shape[0])
        _check(lib.filter_push_group(self.handle, n, hs, ps, ns, ts, int(bool(on_device))), "filter_push_group")
        for u in units:
            u.last_push_len = ns

    def pop_triggers(self, cap: int = 1 << 16) -> np.ndarray:
        """triggers_pop until empty; returns a structured array (TRIGGER_DTYPE)."""
        chunks = []
        while True:
            buf = np.empty(cap, dtype=TRIGGER_DTYPE)
            n = C.c_int64()
            _check(lib.triggers_pop(self.handle, buf.ctypes.data, cap, C.byref(n)), "triggers_pop")
            chunks.append(buf[: n.value])
            if n.value < cap:
                break
        return np.concatenate(chunks) if chunks else np.empty(0, dtype=TRIGGER_DTYPE)


class SbCondDesc(C.Structure):
    _fields_ = [("rate_hz", C.c_double), ("fft_len", C.c_int32), ("n_avg", C.c_int32),
                ("gate_threshold", C.c_float), ("gate_half", C.c_int32), ("gate_taper", C.c_int32),
                ("max_push_samples", C.c_int64)]


class Conditioner:
    """sb_cond: PSD running average, whitening and gating of one detector's strain on the device.

    push(strain, out) conditions the next buffer (numpy FP32 or a CUDA tensor) into the CUDA
    tensor `out` (FP32, same length), delayed by `latency` samples; out can then be pushed to a
    unit of the same context (on_device)."""

    def __init__(self, ctx: Context, rate_hz: float, fft_len: int, n_avg: int, gate_threshold: float,
                 gate_half: int, gate_taper: int, max_push_samples: int):
        d = SbCondDesc(float(rate_hz), int(fft_len), int(n_avg), float(gate_threshold), int(gate_half),
                       int(gate_taper), int(max_push_samples))
        h = C.c_void_p()
        _check(lib.sb_cond_create(ctx.handle, C.byref(d), C.byref(h)), "sb_cond_create")
        self.ctx, self.handle, self.fft_len = ctx, h, int(fft_len)
        lat = C.c_int64()
        _check(lib.sb_cond_latency(self.handle, C.byref(lat)), "sb_cond_latency")
        self.latency = lat.value
        self.pushed = 0

    def push(self, strain, out):
        on_device = hasattr(strain, "is_cuda") and strain.is_cuda
        if not on_device:
            strain = np.ascontiguousarray(strain, dtype=np.float32)
        n = int(strain.shape[0])
        assert out.is_cuda and out.shape[0] >= n
        _check(lib.sb_cond_push(self.handle, C.c_void_p(_ptr(strain)), n, self.pushed, int(on_device),
                                C.c_void_p(out.data_ptr())), "sb_cond_push")
        self.pushed += n

    def psd(self):
        """(P [N/2 + 1] per-bin variance, segments averaged); blocks."""
        nb, seg = C.c_int64(), C.c_int64()
        _check(lib.sb_cond_psd(self.handle, None, 0, C.byref(nb), C.byref(seg)), "sb_cond_psd")
        buf = np.empty(nb.value, dtype=np.float32)
        _check(lib.sb_cond_psd(self.handle, C.c_void_p(buf.ctypes.data), nb.value, C.byref(nb), C.byref(seg)),
               "sb_cond_psd")
        return buf, seg.value

    def close(self):
        if self.handle:
            lib.sb_cond_destroy(self.handle)
            self.handle = None


class Unit:
    """sb_unit: one SVD bank on one detector."""

    def __init__(self, ctx: Context, handle: C.c_void_p):
        self.ctx = ctx
        self.handle = handle
        self.last_push_len = 0

    def info(self) -> SbUnitInfo:
        i = SbUnitInfo()
        _check(lib.sb_unit_query(self.handle, C.byref(i)), "sb_unit_query")
        return i

    def push(self, strain, t0: Optional[int] = None):
        """filter_push: strain is a numpy FP32 array (host) or a CUDA torch tensor (device)."""
        on_device = hasattr(strain, "is_cuda") and strain.is_cuda
        if not on_device:
            strain = np.ascontiguousarray(strain, dtype=np.float32)
        if t0 is None:
            t0 = self.info().samples_pushed
        _check(lib.filter_push(self.handle, C.c_void_p(_ptr(strain)), int(strain.shape[0]), int(t0),
                               int(on_device)), "filter_push")
        self.last_push_len = int(strain.shape[0])

    def snr(self):
        """(first_sample, x [2M, n]) of the last push (needs keep_snr=True); blocks."""
        M2 = 2 * self.info().n_templates
        first, n = C.c_int64(), C.c_int64()
        buf = np.empty(M2 * max(1, self.last_push_len), dtype=np.float32)
        _check(lib.sb_unit_snr(self.handle, buf.ctypes.data, buf.size, C.byref(first), C.byref(n)), "sb_unit_snr")
        return first.value, buf[: M2 * n.value].reshape(M2, n.value)

    def destroy(self):
        if self.handle and self.ctx.handle:
            lib.svdbank_destroy(self.handle)
            self.ctx.units.remove(self)
        self.handle = None
