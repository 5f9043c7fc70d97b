"""Host-side checks of the C-ABI library (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth

import paper_2410_16416_b300 as lloid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "lloid.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M))


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert {"svdbank_create", "filter_push", "triggers_pop", "svdbank_plan"} <= names
    lib = C.CDLL(lloid.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(lloid.SIGNATURES), "binding misses a declared entry point"


def test_context_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lloid.LloidError) as e:
        lloid.Context(0)
    assert e.value.code == lloid.SB_ECUDA


def _small_bank(n=8):
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(n, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 1, 0, 0)
    return lloid.decompose(h, spec.top_rate_hz, spec.slices), h


def independent_latency(levels_d, kmax, K=16):
    """Re-derive the streaming look-ahead: e_{k+1} = ceil((e_k+1+2K)/2)-1,
    Lam_k = max(2 Lam_{k+1} + 2K + 1, e_k - min D at k, 0)."""
    e = [0]
    for _ in range(kmax):
        x = e[-1] + 1 + 2 * K
        e.append(-(-x // 2) - 1)
    lam = [0] * (kmax + 1)
    for k in range(kmax, -1, -1):
        v = 0 if k == kmax else 2 * lam[k + 1] + 2 * K + 1
        if k in levels_d:
            v = max(v, e[k] - min(levels_d[k]))
        lam[k] = max(v, 0)
    return lam[0]


def test_plan_reports_latency_and_flops():
    bank, _ = _small_bank()
    info = lloid.plan(bank, max_push_samples=2048 * 4)
    assert info.k_max == 2
    assert info.latency_samples == independent_latency({0: [0], 2: [512]}, 2)
    flops = sum(2 * s.basis.shape[0] * (s.basis.shape[1] + 2 * bank.n_templates) * s.rate_hz for s in bank.slices)
    assert info.flops_per_second == round(flops)
    # a production-shaped slice layout (delays at each level)
    spec = synth.PRODUCTION_BIN
    lv = {}
    for sp in spec.slices:
        k = int(round(np.log2(spec.top_rate_hz / sp.rate_hz)))
        lv.setdefault(k, []).append(int(round(sp.t_start_s * sp.rate_hz)))
    assert independent_latency(lv, 5) == 1023


def test_plan_rejects_bad_banks():
    bank, _ = _small_bank()
    good = dict(max_push_samples=2048)
    lloid.plan(bank, **good)
    with pytest.raises(lloid.LloidError) as e:
        lloid.plan(bank, max_push_samples=2046)              # not a multiple of 2^k_max
    assert e.value.code == lloid.SB_EINVAL
    with pytest.raises(lloid.LloidError):
        lloid.plan(bank, max_push_samples=2048, window_s=1.0 / 3)
    with pytest.raises(lloid.LloidError):
        lloid.plan(bank, max_push_samples=0)
    import copy
    bad = copy.deepcopy(bank)
    bad.slices[1].rate_hz = 600.0                             # not top / 2^k
    with pytest.raises(lloid.LloidError):
        lloid.plan(bad, **good)
    bad = copy.deepcopy(bank)
    bad.slices[1].basis = bad.slices[1].basis[:, :-1]         # taps do not fill the span
    with pytest.raises(lloid.LloidError):
        lloid.plan(bad, **good)


def test_host_decomposition_matches_oracle_bank():
    """The product's host-side SVD setup and the oracle's agree (ranks, reconstructions)."""
    bank, h = _small_bank(12)
    ob = oracle.build_bank(h, synth.SMALL_BIN.top_rate_hz, synth.SMALL_BIN.slices)
    for s, o in zip(bank.slices, ob.slices):
        assert s.basis.shape == o.basis.shape
        assert np.abs(s.mixing @ s.basis - o.mixing @ o.basis).max() <= 1e-10
        assert np.abs(s.basis @ s.basis.T - np.eye(s.basis.shape[0])).max() <= 1e-12


def test_host_autocorrelation_matches_the_oracle():
    """The host setup's FFT autocorrelation (the xi^2 lag profile handed to svdbank_create) equals
    the oracle's direct sums."""
    from paper_2410_16416_b300 import svdbank
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(6, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 4, 0, 0)
    a = svdbank.template_autocorrelation(h, 16)
    b = oracle.autocorrelation(h, 16)
    assert a.shape == b.shape == (6, 33)
    assert np.abs(a - b).max() <= 1e-12
    bank = svdbank.decompose(h, spec.top_rate_hz, spec.slices)
    assert bank.autocorr is not None and np.abs(bank.autocorr - b).max() <= 1e-12


def _trig(tid, sample, snr):
    t = np.zeros(len(tid), dtype=lloid.TRIGGER_DTYPE)
    t["template_id"], t["sample"], t["snr"] = tid, sample, snr
    return t


def test_coincidences_match_the_oracle_and_the_fixture():
    """sb_coincidences (host only) against the oracle's brute force: the hand-worked fixture and
    random trigger sets with shuffled order, equal samples and duplicates; integer fields exact."""
    path = os.path.join(os.path.dirname(__file__), "golden", "coinc_hand_worked.txt")
    A, B = [], []
    for line in open(path):
        f = line.split()
        if f and f[0] in ("A", "B"):
            (A if f[0] == "A" else B).append((int(f[1]), int(f[2]), float(f[3])))
    cases = [(_trig(*zip(*A)), _trig(*zip(*B)), dt) for dt in (41, 42, 0, 100000)]
    g = np.random.default_rng(7)
    for n_a, n_b, dt in ((0, 5, 10), (7, 0, 10), (300, 250, 41), (200, 200, 0), (50, 60, 5000)):
        ta = _trig(g.integers(0, 12, n_a), g.integers(0, 4000, n_a), g.uniform(6, 30, n_a).astype(np.float32))
        tb = _trig(g.integers(0, 12, n_b), g.integers(0, 4000, n_b), g.uniform(6, 30, n_b).astype(np.float32))
        if n_a and n_b:
            tb["sample"][: min(n_a, n_b) // 3] = ta["sample"][: min(n_a, n_b) // 3]     # equal samples
        cases.append((ta, tb, dt))
    for ta, tb, dt in cases:
        got = lloid.coincidences(ta, tb, dt)
        ref = oracle.coincidences(ta["template_id"], ta["sample"], ta["snr"], tb["template_id"], tb["sample"],
                                  tb["snr"], dt)
        assert len(got) == len(ref)
        for r, w in zip(got, ref):
            assert (int(r["template_id"]), int(r["index_a"]), int(r["index_b"]), int(r["sample_a"]),
                    int(r["sample_b"])) == w[:5]
            assert abs(float(r["network_snr"]) - w[5]) <= 1e-6 * w[5]


def test_coincidences_arguments_and_overflow():
    ta = _trig([1, 1, 2], [100, 200, 300], [7.0, 8.0, 9.0])
    tb = _trig([1, 1, 2], [110, 190, 300], [7.5, 6.5, 8.5])
    n = C.c_int64()
    out = np.empty(2, dtype=lloid.COINC_DTYPE)
    rc = lloid.lib.sb_coincidences(ta.ctypes.data, 3, tb.ctypes.data, 3, 100, out.ctypes.data, 2, C.byref(n))
    assert rc == lloid.SB_EOVERFLOW and n.value == 5        # (100,110) (100,190) (200,110) (200,190) (300,300)
    assert list(out["sample_a"]) == [100, 100] and list(out["sample_b"]) == [110, 190]
    assert lloid.lib.sb_coincidences(ta.ctypes.data, 3, tb.ctypes.data, 3, -1, out.ctypes.data, 2,
                                     C.byref(n)) == lloid.SB_EINVAL
    assert lloid.lib.sb_coincidences(None, 3, tb.ctypes.data, 3, 5, out.ctypes.data, 2, C.byref(n)) == lloid.SB_EINVAL
    assert lloid.lib.sb_coincidences(None, 0, None, 0, 5, None, 0, C.byref(n)) == lloid.SB_OK and n.value == 0
    assert len(lloid.coincidences(ta, tb, 100)) == 5


def test_plan_checks_the_xi2_lag_profiles():
    """svdbank_plan (no device) accepts the oracle's autocorrelation and rejects one whose lag 0 is
    not 1 or that is not finite; a wrong shape is refused by the binding."""
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(4, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 5, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    R = oracle.autocorrelation(h, lloid.SB_XI2_HALF)
    lloid.plan(bank, max_push_samples=4096, autocorr=R)
    bad = R.copy()
    bad[2, lloid.SB_XI2_HALF] = 0.9
    with pytest.raises(lloid.LloidError):
        lloid.plan(bank, max_push_samples=4096, autocorr=bad)
    bad = R.copy()
    bad[1, 3] = np.nan
    with pytest.raises(lloid.LloidError):
        lloid.plan(bank, max_push_samples=4096, autocorr=bad)
    with pytest.raises(ValueError):
        lloid.plan(bank, max_push_samples=4096, autocorr=R[:, :5])


def test_plan_limits_banks_to_eight_rates():
    """A bank spans f0 down to f0 / 2^7: a slice at f0 / 2^8 is rejected, f0 / 2^7 is accepted."""
    import copy
    bank, _ = _small_bank()
    rng = np.random.default_rng(3)
    f0 = bank.top_rate_hz
    for k, ok in ((7, True), (8, False)):
        b = copy.deepcopy(bank)
        s = b.slices[1]
        s.rate_hz = f0 / 2 ** k
        q = int(round((s.t_end_s - s.t_start_s) * s.rate_hz))
        s.basis = np.linalg.qr(rng.standard_normal((q, s.basis.shape[0])))[0].T.copy()
        if ok:
            assert lloid.plan(b, max_push_samples=2 ** k * 4).k_max == k
        else:
            with pytest.raises(lloid.LloidError) as e:
                lloid.plan(b, max_push_samples=2 ** k * 4)
            assert e.value.code == lloid.SB_EINVAL
            assert "2^7" in str(e.value)
