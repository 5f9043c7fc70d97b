"""GPU parity of the conditioning stage (PSD running average, whitening, gating; Sec. II.A)
against oracle.condition, through the C ABI (sb_cond_*).

Input: AR(1) coloured noise (a = 0.9, so the PSD spans about 25 dB) with a loud
sine-Gaussian glitch; the device output (FP32, FFT in shared memory) must equal
the oracle's FP64 conditioned series within 2e-5 on every sample where the
oracle's value is final (2e-3 in the start-up and glitch segments), be bitwise
independent of the push sizes, zero the gated span, and carry the same running
PSD.  The last test feeds the conditioned stream straight into the filter on
the device and compares the SNR with the oracle's filter of the oracle's
conditioned strain.
"""
import numpy as np
import pytest
import scipy.signal

import oracle
import synth
from helpers import check_triggers, rho_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5             # whitened (unit-variance) samples in steady state: FP32 FFT of 2048 points
TOL_LOOSE = 2e-3       # start-up segments and segments holding the glitch


@pytest.fixture(scope="module")
def lloid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as m
    return m


def coloured(n, seed, glitch_at=None, glitch_amp=0.0):
    e = synth.white_noise(n, 50, seed, 0).astype(np.float64)
    d = 3.0 * scipy.signal.lfilter([1.0], [1.0, -0.9], e)
    if glitch_at is not None:
        k = np.arange(n)
        d += glitch_amp * np.exp(-0.5 * ((k - glitch_at) / 8.0) ** 2) * np.sin(0.7 * (k - glitch_at))
    return d.astype(np.float32)


def run_cond(lloid, d, sizes, **kw):
    ctx = lloid.Context(0)
    c = lloid.Conditioner(ctx, max_push_samples=max(sizes), **kw)
    out = torch.zeros(d.shape[0], dtype=torch.float32, device="cuda")
    t = 0
    for sz in sizes:
        c.push(d[t:t + sz], out[t:t + sz])
        t += sz
    ctx.sync()
    y = out.cpu().numpy()
    P, seg = c.psd()
    lat = c.latency
    c.close()
    ctx.close()
    return y, P, seg, lat


def test_conditioner_matches_oracle(lloid):
    f0, N, n_avg, thr, half, taper = 2048, 4096, 8, 30.0, 512, 256
    n = 48 * f0
    d = coloured(n, 1, glitch_at=30 * f0 + 777, glitch_amp=2000.0)
    kw = dict(rate_hz=f0, fft_len=N, n_avg=n_avg, gate_threshold=thr, gate_half=half, gate_taper=taper)
    y, P, seg, lat = run_cond(lloid, d, [f0] * 48, **kw)
    assert lat == N // 2 + half + taper
    xg, Po = oracle.condition.condition(d, N, n_avg, thr, half, taper)
    xw, _ = oracle.condition.whiten(d, N, n_avg)
    # output sample i is the conditioned input sample i - lat; the oracle's is final where the
    # whitening is (m < len(xg)) and every glitch sample that can reach it is known (m + half + taper)
    m = np.arange(n) - lat
    ok = (m >= 0) & (m + half + taper < xg.shape[0])
    err = np.abs(y[ok] - xg[m[ok]])
    # FP32 rounding is a fraction of a segment's energy divided by the running PSD: samples that share
    # a segment with the glitch (energy ~100x the noise's) and the start-up segments (divided by the
    # average of only 1-3 periodograms, whose chi^2 bins come close to 0) get the looser bound
    centers = np.flatnonzero(np.abs(xw) > thr)
    assert centers.size > 0
    loose = np.zeros(xw.shape[0] + N, bool)
    loose[:4 * (N // 2)] = True
    for c in centers:
        loose[max(0, c - N):c + N] = True
    lo = loose[m[ok]]
    print(f"conditioner vs oracle: max |error| {err[~lo].max():.2e} over {(~lo).sum()} samples, "
          f"{err[lo].max():.2e} over the {lo.sum()} start-up or glitch-segment samples; psd after {seg} segments")
    assert err[~lo].max() <= TOL
    assert err[lo].max() <= TOL_LOOSE
    assert np.all(y[~ok & (m < 0)] == 0.0)
    # the glitch was found and removed on both sides
    gated = np.zeros(xw.shape[0], bool)
    for c in centers:
        gated[max(0, c - half):c + half + 1] = True
    out_gated = np.flatnonzero(gated[m[ok]])
    assert out_gated.size > 2 * half and np.all(y[ok][out_gated] == 0.0)
    # the running PSD after the last segment
    assert seg == Po.shape[0]
    rel = np.abs(P - Po[-1]) / Po[-1]
    assert rel.max() <= 1e-4, rel.max()


def test_conditioner_is_independent_of_push_sizes(lloid):
    f0, N = 2048, 2048
    d = coloured(24 * f0, 2, glitch_at=11 * f0 + 5, glitch_amp=1500.0)
    kw = dict(rate_hz=f0, fft_len=N, n_avg=4, gate_threshold=25.0, gate_half=300, gate_taper=200)
    a, Pa, _, _ = run_cond(lloid, d, [1024] * 48, **kw)
    b, Pb, _, _ = run_cond(lloid, d, [8192, 1024, 3072, 4096 * 3, 8192 * 2, 1024 * 6, 2048 * 3], **kw)
    assert np.array_equal(a, b) and np.array_equal(Pa, Pb)


def test_conditioner_rejects_bad_arguments(lloid):
    ctx = lloid.Context(0)
    with pytest.raises(lloid.LloidError) as e:
        lloid.Conditioner(ctx, 2048, 3000, 4, 0.0, 0, 1, 4096)          # not a power of two
    assert e.value.code == lloid.SB_EINVAL
    c = lloid.Conditioner(ctx, 2048, 1024, 4, 0.0, 0, 1, 4096)
    out = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(lloid.LloidError) as e:
        c.push(np.zeros(700, np.float32), out)                           # not a multiple of N/2
    assert e.value.code == lloid.SB_EINVAL
    c.close()
    ctx.close()


def test_conditioned_stream_feeds_the_filter(lloid):
    """Coloured noise plus an injection, conditioned on the device and pushed to an FP32 unit as a
    device buffer: the SNR equals the oracle's filter of the oracle's conditioned strain."""
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 4, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    f0, N = 2048, 4096
    n = 40 * f0
    d = coloured(n, 3)
    inj = np.zeros(n, np.float32)
    synth.inject(inj, h, 9, 26 * f0 + 321, 90.0, 0.7)             # loud in raw units: whitening rescales it
    d = (d + inj).astype(np.float32)
    kw = dict(rate_hz=f0, fft_len=N, n_avg=8, gate_threshold=40.0, gate_half=256, gate_taper=256)
    ctx = lloid.Context(0)
    c = lloid.Conditioner(ctx, max_push_samples=f0, **kw)
    u = ctx.create_unit(bank, threshold=6.0, max_push_samples=f0, keep_snr=True)
    out = torch.zeros(f0, dtype=torch.float32, device="cuda")
    xs = []
    for t in range(0, n, f0):
        c.push(d[t:t + f0], out)
        u.push(out, t)                                             # the same stream: ordered after the conditioner
        _, x = u.snr()
        if x.shape[1]:
            xs.append(x)
    ctx.sync()
    trig = ctx.pop_triggers()
    lat = c.latency
    c.close()
    ctx.close()
    xg = np.concatenate(xs, axis=1)
    xc, _ = oracle.condition.condition(d, N, 8, 40.0, 256, 256)
    cond = np.zeros(n, np.float64)
    cond[lat:lat + xc.shape[0]] = xc[:n - lat]                      # the conditioned stream, as pushed
    x_orc = oracle.lloid_snr(bank, cond.astype(np.float32))
    n_cmp = min(xg.shape[1], lat + xc.shape[0] - 2 * 512)           # where the oracle's stream is final
    err = rho_error(xg[:, :n_cmp], x_orc[:, :n_cmp])
    print(f"conditioned stream -> filter: max |rho| error / max(1, |rho|) {err:.2e}")
    assert err <= 5e-4
    hit = trig[(trig["template_id"] == 9) & (trig["window"] == (26 * f0 + 321 + lat) // f0)]
    assert len(hit) == 1 and float(hit["snr"][0]) > 7.0
    check_triggers(trig[trig["window"] < n_cmp // f0], x_orc, f0, 6.0, (n_cmp // f0) * f0, 1e-3)
