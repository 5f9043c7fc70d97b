"""The allocation-free trigger pick (sb_window_triggers_noalloc).

Some callers cannot allocate device memory while they run (CUDA-graph serving
loops, pools they do not own); sb_window_triggers_noalloc keeps its scratch in
a fixed device array instead.  Its triggers are checked two ways: against the
oracle's window maxima (oracle.window_maxima, through check_triggers) computed
from the same FP32 SNR values, and against the triggers the normal push path
delivered for the same windows, on two calls in a row (the shared scratch keeps
the first call's contents).  The edge cases are a caller-supplied template_ids
array, a block that starts before sample 0 with a partial first window, a
trigger buffer too small (cap = 1), and the size and window-length rejections.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from helpers import check_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


def _noalloc_raw(lloid, x_dev, first, win_len, threshold, M, cap=4096, ids_dev=None):
    out = torch.zeros(max(cap, 1) * lloid.TRIGGER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.full((2,), -7, dtype=torch.int32, device="cuda")          # the call must zero it
    stream = torch.cuda.current_stream().cuda_stream
    rc = lloid.lib.sb_window_triggers_noalloc(x_dev.data_ptr(), x_dev.shape[1], M, x_dev.shape[1], first, win_len,
                                              threshold, None if ids_dev is None else ids_dev.data_ptr(),
                                              out.data_ptr(), cnt.data_ptr(), cap, C.c_void_p(stream))
    assert rc == 0, lloid.lib.sb_last_error()
    torch.cuda.synchronize()
    n, overflow = cnt.cpu().tolist()
    rec = np.frombuffer(out.cpu().numpy().tobytes(), dtype=lloid.TRIGGER_DTYPE)[:min(n, cap)]
    return rec, n, overflow


def _noalloc(lloid, x_dev, first, win_len, threshold, M, cap=4096, ids_dev=None):
    rec, n, overflow = _noalloc_raw(lloid, x_dev, first, win_len, threshold, M, cap, ids_dev)
    assert overflow == 0 and 0 <= n <= cap
    return np.sort(rec, order=["window", "template_id"])


def _small_bin(seed):
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, seed,
                               0, 0)
    return spec, h, oracle.build_bank(h, spec.top_rate_hz, spec.slices)


def test_noalloc_matches_push_path_twice(has_gpu):
    if not has_gpu:
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as lloid
    spec, h, bank = _small_bin(11)
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


def test_noalloc_matches_oracle_window_maxima(has_gpu):
    """The oracle's SNR (rounded to FP32) in, oracle.window_maxima of the same values out.

    The block starts 300 samples before sample 0 (columns there hold large
    values that must be ignored), template ids come from a device array, and
    the two calls in a row use different thresholds."""
    if not has_gpu:
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as lloid
    spec, h, bank = _small_bin(12)
    n = 12 * 2048 + 700                                   # a ragged last window (ignored: not whole)
    d = synth.white_noise(n, 12, 0, 0)
    synth.inject(d, h, 5, 9 * 2048 + 77, 11.0, 1.1)
    x32 = oracle.lloid_snr(bank, d).astype(np.float32)
    x_orc = x32.astype(np.float64)                        # the exact values the kernel reads
    pre = 300
    block = np.concatenate([np.full((x32.shape[0], pre), 50.0, np.float32), x32], axis=1)
    ids = (1000 + 7 * np.arange(bank.n_templates)).astype(np.int64)
    x_dev = torch.from_numpy(np.ascontiguousarray(block)).cuda()
    ids_dev = torch.from_numpy(ids).cuda()
    win = 2048
    for thr in (2.5, 4.0):
        got = _noalloc(lloid, x_dev, -pre, win, thr, bank.n_templates, ids_dev=ids_dev)
        got = got.copy()
        assert (got["unit"] == -1).all()
        matched = check_triggers(got, x_orc, win, thr, n, TOL_FP32, template_ids=ids)
        assert matched == len(got) and matched > 0
        # every whole window in [0, n) is inside the block, so every window maximum above the
        # threshold is a trigger; the injection's window is one of them
        hit = got[(got["template_id"] == ids[5]) & (got["window"] == 9)]
        assert len(hit) == 1 and abs(float(hit["snr"][0]) - 11.0) < 1.5


def test_noalloc_overflow_keeps_count_at_cap(has_gpu):
    if not has_gpu:
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as lloid
    rng = np.random.default_rng(3)
    M, n, win = 8, 4 * 1024, 1024
    x = rng.standard_normal((2 * M, n)).astype(np.float32) * 4.0
    x_dev = torch.from_numpy(x).cuda()
    full = _noalloc(lloid, x_dev, 0, win, 1.0, M)
    assert len(full) == M * (n // win)                    # every window qualifies at threshold 1
    for cap in (1, 5):
        rec, cnt, overflow = _noalloc_raw(lloid, x_dev, 0, win, 1.0, M, cap=cap)
        assert overflow == 1 and cnt == cap, (cap, cnt, overflow)
        # the stored records are valid triggers of the full set
        keys = {(int(t["template_id"]), int(t["window"])): t for t in full}
        for t in rec:
            ref = keys[(int(t["template_id"]), int(t["window"]))]
            assert int(t["sample"]) == int(ref["sample"]) and float(t["snr"]) == float(ref["snr"])


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
    # windows shorter than the 256-sample chunk are refused too
    y = torch.zeros((2 * 4, 1024), dtype=torch.float32, device="cuda")
    rc = lloid.lib.sb_window_triggers_noalloc(y.data_ptr(), y.shape[1], 4, y.shape[1], 0, 128, 6.0, None,
                                              out.data_ptr(), cnt.data_ptr(), 1, None)
    assert rc == lloid.SB_EINVAL
    assert b"window_len" in lloid.lib.sb_last_error()
