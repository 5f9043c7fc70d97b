"""The allocation-free trigger pick (sb_window_triggers_noalloc) against the library's own.

Some callers cannot allocate device memory while they run (CUDA-graph serving
loops, pools they do not own); sb_window_triggers_noalloc keeps its scratch in
a fixed device array instead.  Here its triggers, computed from the SNR block a
push produced, must equal the triggers the normal push path delivered for the
same windows, on two calls in a row (the shared scratch keeps the first call's
contents).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


def _noalloc(lloid, x_dev, first, win_len, threshold, M, cap=4096):
    out = torch.zeros(cap * lloid.TRIGGER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lloid.lib.sb_window_triggers_noalloc(x_dev.data_ptr(), x_dev.shape[1], M, x_dev.shape[1], first, win_len,
                                              threshold, None, out.data_ptr(), cnt.data_ptr(), cap,
                                              C.c_void_p(stream))
    assert rc == 0, lloid.lib.sb_last_error()
    torch.cuda.synchronize()
    n, overflow = cnt.cpu().tolist()
    assert overflow == 0
    rec = np.frombuffer(out.cpu().numpy().tobytes(), dtype=lloid.TRIGGER_DTYPE)[:n]
    return np.sort(rec, order=["window", "template_id"])


def test_noalloc_matches_push_path_twice(has_gpu):
    if not has_gpu:
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as lloid
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 11, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    B = 8 * 2048
    d = synth.white_noise(2 * B, 11, 0, 0)
    synth.inject(d, h, 7, 5 * 2048 + 300, 12.0, 0.2)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, threshold=3.0, max_push_samples=B, keep_snr=True)
    win = 2048
    for call, t0 in enumerate((0, B)):
        u.push(d[t0:t0 + B], t0)
        first, x = u.snr()
        ctx.sync()
        ref = ctx.pop_triggers()
        lo, hi = max(first, 0), first + x.shape[1]
        whole = (ref["window"] * win >= lo) & ((ref["window"] + 1) * win <= hi)
        ref = np.sort(ref[whole], order=["window", "template_id"])
        got = _noalloc(lloid, torch.from_numpy(np.ascontiguousarray(x)).cuda(), first, win, 3.0, bank.n_templates)
        assert len(got) == len(ref) and len(ref) > 0, (call, len(got), len(ref))
        for f in ("template_id", "window", "sample"):
            assert np.array_equal(got[f], ref[f]), (call, f)
        assert np.abs(got["snr"] - ref["snr"]).max() <= TOL_FP32 * max(1.0, float(ref["snr"].max()))
        assert np.abs(np.angle(np.exp(1j * (got["phase"] - ref["phase"])))).max() <= 1e-4
    ctx.close()


def test_noalloc_rejects_oversized_requests(has_gpu):
    if not has_gpu:
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as lloid
    x = torch.zeros((2 * 1024, 1 << 17), dtype=torch.float32, device="cuda")      # 1024 templates x 131072 samples
    out = torch.zeros(lloid.TRIGGER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc = lloid.lib.sb_window_triggers_noalloc(x.data_ptr(), x.shape[1], 1024, x.shape[1], 0, 4096, 6.0, None,
                                              out.data_ptr(), cnt.data_ptr(), 1, None)
    assert rc == lloid.SB_EINVAL
    assert b"exceeds the fixed scratch" in lloid.lib.sb_last_error()
