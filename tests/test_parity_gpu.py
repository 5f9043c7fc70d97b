"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP32 mode bar: |rho_gpu - rho_oracle| <= 1e-4 max(1, |rho_oracle|) on every
template and every produced sample; triggers equal wherever the decision is
not within that tolerance of a tie.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_triggers, push_and_collect, rho_abs_error, rho_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_HALF = 0.05          # absolute |SNR| bound of the BF16 / FP16 modes, every sample
TOL_FP8 = 0.15           # absolute |SNR| bound of SB_FP8 before refinement, every window maximum


@pytest.fixture(scope="module")
def lloid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as m
    return m


@pytest.fixture(scope="module")
def small_case():
    """64-template bin, slices [0,1) s @ 2048 Hz and [1,8) s @ 512 Hz, 16 s of noise + one A = 12 injection."""
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 1, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 16 * 2048
    d = synth.white_noise(n, 1, 0, 0)
    synth.inject(d, h, 17, 12 * 2048 + 777, 12.0, 1.1)
    x = oracle.lloid_snr(bank, d)
    return spec, h, bank, d, x


def test_fp32_small_bin_matches_oracle(lloid, small_case):
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="fp32", threshold=6.0, window_s=1.0, max_push_samples=4096, keep_snr=True)
    lat = u.info().latency_samples
    (xg,) = push_and_collect(ctx, [u], [d], [2048] * 16)
    n_valid = d.shape[0] - lat
    assert xg.shape == (128, n_valid)
    err = rho_error(xg, x)
    print(f"fp32 small bin: max |rho| error / max(1, |rho|) {err:.2e}")
    assert err <= TOL_FP32, err
    ctx.sync()
    trig = ctx.pop_triggers()
    matched = check_triggers(trig, x, 2048, 6.0, n_valid, 2 * TOL_FP32)
    assert matched >= 1
    inj = trig[(trig["template_id"] == 17) & (trig["window"] == 12)]
    assert len(inj) == 1 and abs(inj["snr"][0] - 12.0) < 1.0
    ctx.close()


def test_fp32_every_window_max_matches_oracle(lloid, small_case):
    """Threshold 0: every (template, window) maximum is a trigger; all are compared."""
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, threshold=0.0, max_push_samples=8192)
    for t in range(0, d.shape[0], 8192):
        u.push(d[t:t + 8192], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    n_valid = d.shape[0] - u.info().latency_samples
    assert check_triggers(trig, x, 2048, 0.0, n_valid, 2 * TOL_FP32) == 64 * (n_valid // 2048)
    ctx.close()


def test_fp32_subsample_peaks_match_oracle(lloid, small_case):
    """Every trigger whose sub-sample peak was taken (both neighbours inside one push, a local
    maximum) matches the oracle's parabola vertex; most window maxima qualify."""
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, threshold=0.0, max_push_samples=8192)
    for t in range(0, d.shape[0], 8192):
        u.push(d[t:t + 8192], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    sub = trig[(trig["flags"] & lloid.SB_TRIG_SUBSAMPLE) != 0]
    assert len(sub) >= 0.8 * len(trig)
    worst_pk, worst_dt = 0.0, 0.0
    for t in sub:
        ref = oracle.subsample_peak(x, int(t["template_id"]), int(t["sample"]))
        assert ref is not None
        worst_pk = max(worst_pk, abs(t["snr_peak"] - ref[0]) / max(1.0, ref[0]))
        worst_dt = max(worst_dt, abs(t["dt_peak"] - ref[1]))
    print(f"fp32 sub-sample peaks: {len(sub)} of {len(trig)}; max |snr_peak| error {worst_pk:.2e}, "
          f"max |dt_peak| error {worst_dt:.2e} samples")
    assert worst_pk <= 2 * TOL_FP32 and worst_dt <= 2e-3
    plain = trig[(trig["flags"] & lloid.SB_TRIG_SUBSAMPLE) == 0]
    assert np.all(plain["snr_peak"] == plain["snr"]) and np.all(plain["dt_peak"] == 0.0)


def test_fp32_xi2_matches_oracle(lloid, small_case):
    """Threshold 0: every window maximum whose lags n* - 16 .. n* + 16 lie in one push carries xi^2,
    and it matches the oracle's xi^2 of the oracle's SNR at the same sample."""
    spec, h, bank, d, x = small_case
    R = oracle.autocorrelation(h, lloid.SB_XI2_HALF)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, threshold=0.0, max_push_samples=8192, autocorr=R)
    for t in range(0, d.shape[0], 8192):
        u.push(d[t:t + 8192], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    has = trig[(trig["flags"] & lloid.SB_TRIG_XI2) != 0]
    assert len(has) >= 0.9 * len(trig)
    worst, vals = 0.0, []
    for t in has:
        ref = oracle.xi2(x, R, int(t["template_id"]), int(t["sample"]), lloid.SB_XI2_HALF)
        assert ref is not None
        vals.append(ref)
        worst = max(worst, abs(t["xi2"] - ref) / max(1.0, ref))
    print(f"fp32 xi2: {len(has)} of {len(trig)}; max |xi2 error| / max(1, xi2) {worst:.2e}; "
          f"median xi2 {np.median(vals):.3f}")
    assert worst <= 2e-3
    assert np.all(trig[(trig["flags"] & lloid.SB_TRIG_XI2) == 0]["xi2"] == 0.0)


def test_two_detector_coincidence_of_an_injection(lloid, small_case):
    """Two detectors (one unit each, one grouped push per buffer) see the same template 13 samples
    apart: the coincidence generator pairs their triggers of that template, as the oracle pairs the
    oracle's triggers of the same strains."""
    spec, h, bank, d, x = small_case
    n = d.shape[0]
    n_c = 12 * 2048 + 777
    d1 = synth.white_noise(n, 1, 0, 1)
    synth.inject(d1, h, 17, n_c + 13, 11.0, 0.4)
    ctx = lloid.Context(0)
    u0 = ctx.create_unit(bank, detector=0, threshold=6.0, max_push_samples=8192)
    u1 = ctx.create_like(u0, detector=1)
    for t in range(0, n, 8192):
        ctx.push_group([u0, u1], [d[t:t + 8192], d1[t:t + 8192]], [t, t], False)
    ctx.sync()
    trig = ctx.pop_triggers()
    id0, id1, lat = u0.info().unit, u1.info().unit, u0.info().latency_samples
    ctx.close()
    ta, tb = trig[trig["unit"] == id0], trig[trig["unit"] == id1]
    max_dt = int(np.ceil(0.010 * spec.top_rate_hz)) + 2          # 10 ms of light travel + 2 samples
    co = lloid.coincidences(ta, tb, max_dt)
    hit = co[co["template_id"] == 17]
    assert len(hit) >= 1 and np.any(np.abs(hit["sample_a"] - n_c) <= 2) and np.any(np.abs(hit["sample_b"] - n_c - 13) <= 2)
    n_valid = n - lat
    x1 = oracle.lloid_snr(bank, d1)
    oa = oracle.triggers(x, int(spec.top_rate_hz), 6.0, n_valid)
    ob = oracle.triggers(x1, int(spec.top_rate_hz), 6.0, n_valid)
    ref = oracle.coincidences([t[0] for t in oa], [t[1] for t in oa], [t[3] for t in oa],
                              [t[0] for t in ob], [t[1] for t in ob], [t[3] for t in ob], max_dt)
    want = {(r[0], r[3], r[4]) for r in ref}
    got = {(int(r["template_id"]), int(r["sample_a"]), int(r["sample_b"])) for r in co}
    print(f"coincidences: {len(got)} on the device's triggers, {len(want)} on the oracle's")
    assert any(t == 17 and abs(sa - n_c) <= 2 and abs(sb - n_c - 13) <= 2 for t, sa, sb in want)
    assert want == got


def test_streaming_is_bitwise_independent_of_buffer_sizes(lloid, small_case):
    spec, h, bank, d, x = small_case
    runs = []
    for sizes in ([2048] * 16, [8192] * 4, [4, 2044, 4096, 12, 6132, 8192, 8192, 4096]):
        assert sum(sizes) == d.shape[0]
        ctx = lloid.Context(0)
        u = ctx.create_unit(bank, max_push_samples=8192, keep_snr=True)
        (xg,) = push_and_collect(ctx, [u], [d], sizes)
        ctx.sync()
        runs.append((xg, np.sort(ctx.pop_triggers(), order=["window", "template_id"])))
        ctx.close()
    for xg, tr in runs[1:]:
        assert np.array_equal(xg, runs[0][0])
        assert np.array_equal(tr, runs[0][1])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_pushes_equal_direct_pushes(lloid, small_case, precision):
    """Pushes captured into CUDA graphs (reused per group shape, updated in place) give bitwise
    the same SNR and triggers as kernels launched one by one, across changing push sizes."""
    spec, h, bank, d, x = small_case
    d2 = synth.white_noise(d.shape[0], 5, 0, 1)
    sizes = [2048] * 4 + [4096] * 2 + [2048] * 8
    runs = []
    for graphs in (False, True):
        ctx = lloid.Context(0)
        ctx.graphs(graphs)
        kw = dict(precision=precision, threshold=5.0, max_push_samples=4096, keep_snr=True)
        if precision != "fp32":
            kw["refine_threshold"] = 4.5
        units = [ctx.create_unit(bank, detector=det, **kw) for det in (0, 1)]
        xs = push_and_collect(ctx, units, [d, d2], sizes)
        ctx.sync()
        trig = np.sort(ctx.pop_triggers(), order=["unit", "window", "template_id"])
        st = ctx.stats()
        ctx.close()
        # pushes that time a new mixing launch shape run uncaptured
        tuned = st["autotune_shapes"] if precision != "fp32" else 0
        if graphs:
            assert len(sizes) - tuned <= st["graph_launches"] <= len(sizes) and st["graph_launches"] >= 1
        else:
            assert st["graph_launches"] == 0
        runs.append((xs, trig))
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    t0, t1 = runs[0][1], runs[1][1]
    for f in ("template_id", "sample", "window", "snr", "phase", "snr_peak", "dt_peak", "flags"):
        assert np.array_equal(t0[f], t1[f])
    assert len(t0) >= 1


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_autotuned_pipeline_equals_default(lloid, small_case, precision):
    """The mixing kernel's pipeline shape, timed and chosen per launch shape, leaves every output
    bitwise unchanged (tuning on vs off, with the tuning pushes themselves included)."""
    spec, h, bank, d, x = small_case
    sizes = [2048] * 3 + [4096] * 2 + [2048] * 5
    runs = []
    for tune in (False, True):
        ctx = lloid.Context(0)
        ctx.autotune(tune)
        u = ctx.create_unit(bank, precision=precision, threshold=5.0, max_push_samples=4096, keep_snr=True,
                            refine_threshold=4.5)
        xs = push_and_collect(ctx, [u], [d], sizes)
        ctx.sync()
        trig = np.sort(ctx.pop_triggers(), order=["unit", "window", "template_id"])
        st = ctx.stats()
        ctx.close()
        if tune:
            assert st["autotune_shapes"] >= 2 and st["autotune_launches"] >= 2 * st["autotune_shapes"]
        else:
            assert st["autotune_shapes"] == 0 and st["autotune_launches"] == 0
        runs.append((xs, trig))
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    t0, t1 = runs[0][1], runs[1][1]
    for f in ("template_id", "sample", "window", "snr", "phase", "snr_peak", "dt_peak", "flags"):
        assert np.array_equal(t0[f], t1[f])
    assert len(t0) >= 1


def _shape_banks(n, max_templates=40):
    banks = []
    for b in range(n):
        sb = synth.shape_only_bank(1000 + b, dur_range=(2.0, 6.0), l_range=(5, 40), max_templates=max_templates)
        banks.append(sb)
    return banks


def test_group_equals_alone_bitwise(lloid):
    """One unit's SNR and triggers are identical alone and inside a grouped push (uneven shapes)."""
    banks = _shape_banks(4)
    n = 6 * 4096
    strains = [synth.white_noise(n, 3, b, 0) for b in range(len(banks))]
    sizes = [4096] * 6
    ctx = lloid.Context(0)
    units = [ctx.create_unit(b, threshold=3.0, max_push_samples=4096, keep_snr=True) for b in banks]
    grouped = push_and_collect(ctx, units, strains, sizes)
    ctx.sync()
    tg = ctx.pop_triggers()
    ctx.close()
    for i, b in enumerate(banks):
        c2 = lloid.Context(0)
        u = c2.create_unit(b, threshold=3.0, max_push_samples=4096, keep_snr=True)
        (alone,) = push_and_collect(c2, [u], [strains[i]], sizes)
        c2.sync()
        ta = c2.pop_triggers()
        c2.close()
        assert np.array_equal(alone, grouped[i])
        mine = tg[tg["unit"] == i]
        assert np.array_equal(np.sort(ta[["template_id", "sample", "window", "snr", "phase"]], order=["window", "template_id"]),
                              np.sort(mine[["template_id", "sample", "window", "snr", "phase"]], order=["window", "template_id"]))


def test_grouped_uneven_banks_match_oracle(lloid):
    """Ragged shapes (M, L, Q, slice counts) in one grouped push, each unit against the oracle."""
    banks = _shape_banks(3, max_templates=37)
    n = 6 * 4096
    strains = [synth.white_noise(n, 4, b, 0) for b in range(len(banks))]
    ctx = lloid.Context(0)
    units = [ctx.create_unit(b, threshold=4.0, max_push_samples=8192, keep_snr=True) for b in banks]
    outs = push_and_collect(ctx, units, strains, [8192, 4096, 8192, 4096])
    for b, d, xg in zip(banks, strains, outs):
        ob = oracle.bank_from_arrays(b.n_templates, b.top_rate_hz, b.slices)
        xo = oracle.lloid_snr(ob, d)
        assert rho_error(xg, xo) <= TOL_FP32
    ctx.close()


def test_device_resident_strain_matches_host_strain(lloid, small_case):
    spec, h, bank, d, x = small_case
    res = []
    for on_dev in (False, True):
        ctx = lloid.Context(0)
        u = ctx.create_unit(bank, max_push_samples=4096, keep_snr=True)
        dd = torch.from_numpy(d).cuda() if on_dev else None
        (xg,) = push_and_collect(ctx, [u], [d], [4096] * 8, on_device=on_dev, device_strains=[dd] if on_dev else None)
        res.append(xg)
        ctx.close()
    assert np.array_equal(res[0], res[1])


def test_error_statuses(lloid, small_case):
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, max_push_samples=4096)
    u.push(d[:2048], 0)
    with pytest.raises(lloid.LloidError) as e:
        u.push(d[4096:6144], 4096)                          # gap
    assert e.value.code == lloid.SB_EGAP
    with pytest.raises(lloid.LloidError) as e:
        u.push(d[2048:2050], 2048)                          # not a multiple of 2^k_max
    assert e.value.code == lloid.SB_EINVAL
    with pytest.raises(lloid.LloidError) as e:
        u.push(np.zeros(8192, np.float32), 2048)            # over max_push_samples
    assert e.value.code == lloid.SB_EINVAL
    small = lloid.Context(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(lloid.LloidError) as e:
        small.create_unit(bank, max_push_samples=4096)
    assert e.value.code == lloid.SB_EBUSY
    small.close()
    ctx.close()


def test_production_bin_sampled_templates(lloid):
    """1000-template, 6-slice bin (4096 ... 128 Hz): 128 s through the GPU in 16-s pushes;
    the oracle recomputes 24 sampled templates (their SNR rows are independent)."""
    spec = synth.PRODUCTION_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 2, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 128 * 4096
    d = synth.white_noise(n, 2, 0, 0)
    synth.inject(d, h, 321, 100 * 4096 + 123, 15.0, 0.4)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, threshold=6.0, max_push_samples=16 * 4096, keep_snr=True)
    (xg,) = push_and_collect(ctx, [u], [d], [16 * 4096] * 8)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    pick = np.unique(np.concatenate([np.linspace(0, 999, 23).astype(int), [321]]))
    rows = np.stack([2 * pick, 2 * pick + 1], axis=1).ravel()
    sub = oracle.OracleBank(len(pick), bank.top_rate_hz,
                            [oracle.OracleSlice(s.rate_hz, s.t_start_s, s.t_end_s, s.level, s.delay, s.basis,
                                                s.mixing[rows], s.sigma) for s in bank.slices])
    xo = oracle.lloid_snr(sub, d)
    err = rho_error(xg[rows], xo)
    print(f"fp32 production bin (sampled templates): max |rho| error / max(1, |rho|) {err:.2e}")
    assert err <= TOL_FP32
    n_valid = xg.shape[1]
    tsub = trig[np.isin(trig["template_id"], pick)]
    tsub = tsub.copy()
    tsub["template_id"] = np.searchsorted(pick, tsub["template_id"])
    check_triggers(tsub, xo, 4096, 6.0, n_valid, 2 * TOL_FP32)
    hit = trig[(trig["template_id"] == 321) & (trig["window"] == 100)]
    assert len(hit) == 1 and abs(hit["snr"][0] - 15.0) < 1.0


# ---------------------------------------------------------------- 16-bit tensor-core modes
@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_half_small_bin_matches_oracle(lloid, small_case, precision):
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision=precision, threshold=6.0, max_push_samples=4096, keep_snr=True)
    (xg,) = push_and_collect(ctx, [u], [d], [2048] * 16)
    err = rho_abs_error(xg, x)
    print(f"{precision}: max |rho| error {err:.4f}")
    assert err <= TOL_HALF, err
    ctx.sync()
    trig = ctx.pop_triggers()
    n_valid = d.shape[0] - u.info().latency_samples
    assert check_triggers(trig, x, 2048, 6.0, n_valid, TOL_HALF, absolute=True) >= 1
    ctx.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_half_streaming_and_grouping_are_deterministic(lloid, precision):
    """Tensor-core modes: identical bits across push sizes and alone vs grouped."""
    banks = _shape_banks(3, max_templates=37)
    n = 6 * 4096
    strains = [synth.white_noise(n, 6, b, 0) for b in range(len(banks))]
    ctx = lloid.Context(0)
    units = [ctx.create_unit(b, precision=precision, threshold=4.0, max_push_samples=8192, keep_snr=True)
             for b in banks]
    grouped = push_and_collect(ctx, units, strains, [8192, 4096, 8192, 4096])
    for b, dd, xg in zip(banks, strains, grouped):
        ob = oracle.bank_from_arrays(b.n_templates, b.top_rate_hz, b.slices)
        assert rho_abs_error(xg, oracle.lloid_snr(ob, dd)) <= TOL_HALF
    ctx.close()
    c2 = lloid.Context(0)
    u = c2.create_unit(banks[1], precision=precision, threshold=4.0, max_push_samples=8192, keep_snr=True)
    (alone,) = push_and_collect(c2, [u], [strains[1]], [4096] * 6)
    c2.close()
    assert np.array_equal(alone, grouped[1])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_half_production_bin_sampled_templates(lloid, precision):
    spec = synth.PRODUCTION_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 2, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 96 * 4096
    d = synth.white_noise(n, 2, 0, 1)
    synth.inject(d, h, 500, 80 * 4096 + 99, 30.0, -0.8)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision=precision, threshold=6.0, max_push_samples=16 * 4096, keep_snr=True)
    (xg,) = push_and_collect(ctx, [u], [d], [16 * 4096] * 6)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    pick = np.unique(np.concatenate([np.linspace(0, 999, 15).astype(int), [500]]))
    rows = np.stack([2 * pick, 2 * pick + 1], axis=1).ravel()
    sub = oracle.OracleBank(len(pick), bank.top_rate_hz,
                            [oracle.OracleSlice(s.rate_hz, s.t_start_s, s.t_end_s, s.level, s.delay, s.basis,
                                                s.mixing[rows], s.sigma) for s in bank.slices])
    xo = oracle.lloid_snr(sub, d)
    err = rho_abs_error(xg[rows], xo)
    print(f"{precision} production bin (sampled templates): max |rho| error {err:.4f}")
    print(f"{precision} production: max |rho| error {err:.4f}")
    assert err <= TOL_HALF
    hit = trig[(trig["template_id"] == 500) & (trig["window"] == 80)]
    assert len(hit) == 1 and abs(hit["snr"][0] - 30.0) < 1.5


# ---------------------------------------------------------------- a6 FP32 refinement
@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_refined_window_maxima_match_oracle(lloid, small_case, precision):
    """Window maxima above the refine threshold are recomputed in FP32: every
    trigger (threshold 6 > refine 5.5) is flagged refined and equals the FP64
    oracle's window maximum to FP32 accuracy."""
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision=precision, threshold=6.0, refine_threshold=5.5, max_push_samples=4096)
    for t in range(0, d.shape[0], 4096):
        u.push(d[t:t + 4096], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    n_valid = d.shape[0] - u.info().latency_samples
    assert len(trig) >= 1 and np.all(trig["flags"] & lloid.SB_TRIG_REFINED)
    assert check_triggers(trig, x, 2048, 6.0, n_valid, 2 * TOL_FP32) >= 1
    ctx.close()


def test_refined_production_injection(lloid):
    """Production bin, BF16: the SNR-30 injection's trigger after refinement is within 1e-3 of the oracle."""
    spec = synth.PRODUCTION_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 2, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 96 * 4096
    d = synth.white_noise(n, 2, 0, 1)
    synth.inject(d, h, 500, 80 * 4096 + 99, 30.0, -0.8)
    ctx = lloid.Context(0)
    R = oracle.autocorrelation(h, lloid.SB_XI2_HALF)
    u = ctx.create_unit(bank, precision="bf16", threshold=6.0, refine_threshold=5.5, max_push_samples=16 * 4096,
                        autocorr=R)
    for t in range(0, n, 16 * 4096):
        u.push(d[t:t + 16 * 4096], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    hit = trig[(trig["template_id"] == 500) & (trig["window"] == 80)]
    assert len(hit) == 1 and hit["flags"][0] & lloid.SB_TRIG_REFINED
    rows = np.array([1000, 1001])
    sub = oracle.OracleBank(1, bank.top_rate_hz,
                            [oracle.OracleSlice(s.rate_hz, s.t_start_s, s.t_end_s, s.level, s.delay, s.basis,
                                                s.mixing[rows], s.sigma) for s in bank.slices])
    xo = oracle.lloid_snr(sub, d)
    wins, n_star, amax, ph = oracle.window_maxima(xo, 4096, 81 * 4096, 80 * 4096)
    print("refined", hit["snr"][0], "oracle", amax[0, 0], "samples", hit["sample"][0], n_star[0, 0])
    assert abs(hit["snr"][0] - amax[0, 0]) <= 1e-3
    assert hit["sample"][0] == n_star[0, 0]
    ref = oracle.subsample_peak(xo, 0, int(n_star[0, 0]))
    print("refined sub-sample peak", hit["snr_peak"][0], hit["dt_peak"][0], "oracle", ref)
    assert hit["flags"][0] & lloid.SB_TRIG_SUBSAMPLE and ref is not None
    assert abs(hit["snr_peak"][0] - ref[0]) <= 1e-3 and abs(hit["dt_peak"][0] - ref[1]) <= 5e-3
    xr = oracle.xi2(xo, R[500], 0, int(n_star[0, 0]), lloid.SB_XI2_HALF)
    print("refined xi2", hit["xi2"][0], "oracle", xr)
    assert hit["flags"][0] & lloid.SB_TRIG_XI2 and abs(hit["xi2"][0] - xr) <= 1e-3 * max(1.0, xr)
    # every trigger is refined, and every refined one whose lags are all in its push has xi^2
    assert np.all(trig["flags"] & lloid.SB_TRIG_REFINED)
    assert np.mean((trig["flags"] & lloid.SB_TRIG_XI2) != 0) >= 0.9


# ---------------------------------------------------------------- E4M3 mode (config 4)
def test_fp8_small_bin_error_distribution_and_refinement(lloid, small_case):
    """E4M3 basis FIR (per-basis-vector weight scales, two-term strain with a per-buffer scale,
    FP32 accumulate), BF16 mixing: before refinement every window maximum is within 0.15 of the
    oracle (the every-sample distribution is reported); after refinement every trigger (window
    maximum above 5.5) is recomputed in FP32 and matches the oracle within 1e-3."""
    spec, h, bank, d, x = small_case
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="fp8", threshold=0.0, refine_threshold=0.0, max_push_samples=4096,
                        keep_snr=True)
    (xg,) = push_and_collect(ctx, [u], [d], [4096] * 8)
    ctx.sync()
    raw = ctx.pop_triggers()
    ctx.close()
    n = xg.shape[1]
    rg = xg[0::2].astype(np.float64) + 1j * xg[1::2]
    ro = x[0::2, :n] + 1j * x[1::2, :n]
    q = np.percentile(np.abs(rg - ro), [50, 99, 100])
    nmax = check_triggers(raw, x, 2048, 0.0, n, TOL_FP8, absolute=True)
    print(f"fp8 unrefined: every-sample |rho| error p50 {q[0]:.4f} p99 {q[1]:.4f} max {q[2]:.4f}; "
          f"{nmax} window maxima within {TOL_FP8}")
    assert nmax == 64 * (n // 2048)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="fp8", threshold=6.0, refine_threshold=5.5, max_push_samples=4096)
    for t in range(0, d.shape[0], 4096):
        u.push(d[t:t + 4096], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    assert len(trig) >= 1 and np.all(trig["flags"] & lloid.SB_TRIG_REFINED)
    assert check_triggers(trig, x, 2048, 6.0, n, 1e-3, absolute=True) >= 1


def test_fp8_production_refined_injection(lloid):
    spec = synth.PRODUCTION_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 2, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 96 * 4096
    d = synth.white_noise(n, 2, 0, 1)
    synth.inject(d, h, 500, 80 * 4096 + 99, 30.0, -0.8)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="fp8", threshold=6.0, refine_threshold=5.5, max_push_samples=16 * 4096)
    for t in range(0, n, 16 * 4096):
        u.push(d[t:t + 16 * 4096], t)
    ctx.sync()
    trig = ctx.pop_triggers()
    ctx.close()
    hit = trig[(trig["template_id"] == 500) & (trig["window"] == 80)]
    assert len(hit) == 1 and hit["flags"][0] & lloid.SB_TRIG_REFINED
    rows = np.array([1000, 1001])
    sub = oracle.OracleBank(1, bank.top_rate_hz,
                            [oracle.OracleSlice(s.rate_hz, s.t_start_s, s.t_end_s, s.level, s.delay, s.basis,
                                                s.mixing[rows], s.sigma) for s in bank.slices])
    xo = oracle.lloid_snr(sub, d)
    wins, n_star, amax, ph = oracle.window_maxima(xo, 4096, 81 * 4096, 80 * 4096)
    print("fp8 refined", hit["snr"][0], "oracle", amax[0, 0])
    assert abs(hit["snr"][0] - amax[0, 0]) <= 1e-3 and hit["sample"][0] == n_star[0, 0]
