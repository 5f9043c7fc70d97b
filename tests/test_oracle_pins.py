"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the plausible oracle mistake it would catch.
"""
import math
import os

import numpy as np
import pytest
import scipy.signal
import scipy.special

import oracle
import synth
from oracle.resample import HALF_K


# ---------------------------------------------------------------- helpers
def brute_correlate(filters, d, delay):
    R, Q = filters.shape
    out = np.zeros((R, d.shape[0]))
    for r in range(R):
        for m in range(d.shape[0]):
            acc = 0.0
            for q in range(Q):
                i = m - delay - q
                if 0 <= i < d.shape[0]:
                    acc += filters[r, q] * d[i]
            out[r, m] = acc
    return out


def small_bin(n_templates=6, duration=2.0, f0=1024.0, slices=None):
    slices = slices or [synth.SliceSpec(f0, 0.0, 0.5), synth.SliceSpec(f0 / 4, 0.5, duration)]
    spec = synth.BinSpec(n_templates, 1.0, 3.0, f0, duration, slices)
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, f0, duration, 9, 0, 0)
    return spec, h


def dtft(g, w):
    j = np.arange(-(g.shape[0] // 2), g.shape[0] // 2 + 1)
    return np.real(np.exp(-1j * np.outer(w, j)) @ g)


# ---------------------------------------------------------------- P1 brute force
def test_p1_fft_correlation_matches_brute_force():
    """Catches: off-by-one delay, reversed filter, FFT wrap-around."""
    g = np.random.default_rng(1)
    f = g.standard_normal((3, 7))
    d = g.standard_normal(41)
    for delay in (0, 5, 40, 60):
        ref = brute_correlate(f, d, delay)
        got = oracle.causal_correlate(f, d, delay)
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_p1_direct_snr_brute_force_small():
    g = np.random.default_rng(2)
    h = g.standard_normal((4, 64))
    d = g.standard_normal(300).astype(np.float32)
    ref = brute_correlate(h, d.astype(np.float64), 0)
    got = oracle.direct_snr(h, d)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_p1_golden_hand_worked_fir():
    """Hand-worked example of step a2 stored under tests/golden (integers, exact)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fir_hand_worked.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, val = line.split("=")
        rows[key.strip()] = [float(v) for v in val.split()]
    v = np.array(rows["v"])[None, :]
    d = np.array(rows["d"])
    got = oracle.causal_correlate(v, d, int(rows["D"][0]))[0]
    assert np.allclose(got, rows["o"], atol=1e-12)


# ---------------------------------------------------------------- P2 SVD invariants
def test_p2_svd_invariants():
    """Catches: transposed basis/mixing, sigma^2 vs sigma truncation, wrong slice sampling."""
    spec, h = small_bin()
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    full = oracle.build_bank(h, spec.top_rate_hz, spec.slices, frac=1.0)
    for s, sf, sp in zip(bank.slices, full.slices, spec.slices):
        H = oracle.slice_filters(h, spec.top_rate_hz, sp.rate_hz, sp.t_start_s, sp.t_end_s)
        L = s.basis.shape[0]
        assert np.abs(s.basis @ s.basis.T - np.eye(L)).max() <= 1e-12
        err = np.linalg.norm(H - s.mixing @ s.basis) ** 2
        tail = float((s.sigma[L:] ** 2).sum())
        assert abs(err - tail) <= 1e-10 * float((s.sigma ** 2).sum())
        power = np.cumsum(s.sigma ** 2)
        assert power[L - 1] >= 0.9999 * power[-1]
        if L > 1:
            assert power[L - 2] < 0.9999 * power[-1]
        assert np.abs(sf.mixing @ sf.basis - H).max() <= 1e-12 * np.abs(H).max()


def test_p2_slice_filter_indexing():
    """H_s[a, q] = 2^k h[a, t_s f0 + q 2^k]: checked on a ramp template."""
    h = np.arange(2 * 1 * 64, dtype=np.float64).reshape(2, 64)
    H = oracle.slice_filters(h, 64.0, 16.0, 0.25, 1.0)         # k = 2, j0 = 16, Q = 12
    assert H.shape == (2, 12)
    assert H[0, 0] == 4 * h[0, 16] and H[1, 11] == 4 * h[1, 16 + 44]


# ---------------------------------------------------------------- P3 special case
def test_p3_full_rate_untruncated_equals_direct():
    """Two slices both at f0, no truncation: the SVD path is the direct sum exactly.

    Catches: wrong delay D_s, reversed taps, mixing/basis transposed, dropped slice.
    """
    f0 = 512.0
    spec, h = small_bin(n_templates=4, duration=1.0, f0=f0,
                        slices=[synth.SliceSpec(f0, 0.0, 0.25), synth.SliceSpec(f0, 0.25, 1.0)])
    bank = oracle.build_bank(h, f0, spec.slices, frac=1.0)
    d = synth.white_noise(2048, 7, 0, 0)
    x_svd = oracle.lloid_snr(bank, d)
    x_dir = oracle.direct_snr(h, d)
    assert np.abs(x_svd - x_dir).max() <= 1e-12 * np.abs(x_dir).max()


# ---------------------------------------------------------------- P4 resampler
def test_p3_row_subsets_are_independent(cfg_small):
    """mix_and_sum for a subset of the real filters returns exactly those rows of the full
    computation (each filter's SNR depends only on its own mixing row)."""
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    d = synth.white_noise(10 * 2048, 91, 0, 0).astype(np.float64)
    g = oracle.halfband()
    o = oracle.basis_outputs(bank, oracle.decimation_cascade(d, bank.k_max, g))
    full = oracle.mix_and_sum(bank, o, d.shape[0], g)
    rows = np.array([5, 6, 20, 21, 31])
    sub = oracle.mix_and_sum(bank, o, d.shape[0], g, rows)
    for k in full:
        assert np.array_equal(sub[k], full[k][rows])
    assert np.allclose(full[0], oracle.lloid_snr(bank, d), rtol=0, atol=1e-12)


def test_p4_halfband_structure():
    g = oracle.halfband()
    K2 = 2 * HALF_K
    assert g.shape == (4 * HALF_K + 1,)
    assert np.array_equal(g, g[::-1])
    assert abs(g.sum() - 1.0) <= 1e-15 * 4
    assert g[K2] == 0.5
    for j in range(-K2, K2 + 1):
        if j != 0 and j % 2 == 0:
            assert g[K2 + j] == 0.0


def test_p4_bessel_and_kaiser_match_library():
    """The I0 power series and the Kaiser window against scipy's independent routines."""
    for x in (0.0, 0.5, 1.0, 2.0, 5.0, 8.6):
        assert abs(oracle.bessel_i0(x) - scipy.special.i0(x)) <= 1e-13 * scipy.special.i0(x)
    w = oracle.kaiser(2 * HALF_K, 8.6)
    ref = scipy.signal.windows.kaiser(4 * HALF_K + 1, 8.6, sym=True)
    assert np.abs(w - ref).max() <= 1e-13


def test_p4_passband_and_stopband():
    """|H - 1| <= 1e-4 up to 0.8 of the decimated Nyquist; >= 80 dB rejection beyond 1.2 of it."""
    g = oracle.halfband()
    w_pass = np.linspace(0, 0.8 * np.pi / 2, 400)
    w_stop = np.linspace(1.2 * np.pi / 2, np.pi, 400)
    assert np.abs(dtft(g, w_pass) - 1.0).max() <= 1e-4
    assert np.abs(dtft(g, w_stop)).max() <= 1e-4
    # halfband symmetry H(w) + H(pi - w) = 1
    w = np.linspace(0, np.pi, 101)
    assert np.abs(dtft(g, w) + dtft(g, np.pi - w) - 1.0).max() <= 1e-13


def test_p4_tone_through_decimate_and_upsample():
    """A band-limited tone survives decimation and interpolation (amplitude, phase, alignment)."""
    g = oracle.halfband()
    n = 4096
    t = np.arange(n)
    f = 0.8 * 0.25                       # cycles per input sample: 0.8 of the output Nyquist
    x = np.cos(2 * np.pi * f * t + 0.3)
    y = oracle.decimate(x, g)
    m = np.arange(y.shape[0])
    ref = np.cos(2 * np.pi * f * 2 * m + 0.3)
    inner = slice(64, y.shape[0] - 64)
    assert np.abs(y[inner] - ref[inner]).max() <= 1e-4
    z = oracle.upsample(y, g)
    inner2 = slice(256, n - 256)
    assert np.abs(z[inner2] - x[inner2]).max() <= 2e-4
    assert np.array_equal(z[0::2][100:200], y[100:200])      # even outputs are copies


# ---------------------------------------------------------------- P5 / P8 injection
@pytest.fixture(scope="module")
def cfg_small():
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(16, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 3, 0, 0)
    return spec, h


def test_p5_p8_injection_recovered_untruncated(cfg_small):
    """Noise-free injection at A = 12: |rho(n_c)| = A within 1e-3 and arg rho = phi0 within 0.05.

    Catches: the 2^k slice gain, the x2 interpolation gain, level misalignment, phase sign.
    """
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices, frac=1.0)
    n = 12 * 2048
    for i, phi0 in ((3, 0.7), (11, -2.0)):
        d = np.zeros(n, np.float32)
        n_c = 10 * 2048 + 5
        synth.inject(d, h, i, n_c, 12.0, phi0)
        rho = oracle.complex_snr(oracle.lloid_snr(bank, d))[i, n_c]
        assert abs(abs(rho) - 12.0) <= 12e-3
        assert abs(math.remainder(np.angle(rho) - phi0, 2 * math.pi)) <= 0.05


def test_p6_truncation_bound(cfg_small):
    """|x_svd - x_dir| <= A |h - h_hat|_w + 1e-3 A on the injected filter pair (Cauchy-Schwarz)."""
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    n = 12 * 2048
    i, n_c, A = 5, 10 * 2048, 12.0
    d = np.zeros(n, np.float32)
    synth.inject(d, h, i, n_c, A, 0.4)
    xs = oracle.lloid_snr(bank, d)[:, n_c]
    xd = oracle.direct_snr(h, d)[:, n_c]
    for a in (2 * i, 2 * i + 1):
        werr = 0.0
        for s, sp in zip(bank.slices, spec.slices):
            H = oracle.slice_filters(h, spec.top_rate_hz, sp.rate_hz, sp.t_start_s, sp.t_end_s)
            werr += 2.0 ** (-s.level) * float(((H[a] - s.mixing[a] @ s.basis) ** 2).sum())
        assert abs(xs[a] - xd[a]) <= A * math.sqrt(werr) + 1e-3 * A


# ---------------------------------------------------------------- P7 gain chain
def test_p7_impulse_response_energy(cfg_small):
    """Unit-norm templates: the multirate path's impulse-response energy is 1 per real filter.

    White noise then gives E|rho|^2 = 2.  The path is periodically time varying
    (period 2^kmax), so the energy is averaged over the 4 impulse phases.
    """
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices, frac=1.0)
    n = 12 * 2048
    energies = []
    for phase in range(4):
        d = np.zeros(n, np.float32)
        d[2048 + phase] = 1.0
        x = oracle.lloid_snr(bank, d)
        energies.append((x ** 2).sum(axis=1))
    e = np.mean(energies, axis=0)
    assert np.abs(e - 1.0).max() <= 2e-3


def test_p7_rice_mean_over_seeds():
    """Unit-norm template at amplitude A in unit white noise: mean |rho(n_c)| = Rice mean.

    Rice(A, 1) mean = sqrt(pi/2) L_{1/2}(-A^2/2); checked over 240 seeds at 3 sigma.
    Uses a one-slice top-rate bank (untruncated) so that the run stays short.
    """
    f0 = 1024.0
    h, _ = synth.template_bank(2, 1.0, 1.5, f0, 1.0, 4, 0, 0)
    bank = oracle.build_bank(h, f0, [synth.SliceSpec(f0, 0.0, 0.5), synth.SliceSpec(f0 / 2, 0.5, 1.0)],
                             frac=1.0)
    A, n, n_c = 3.0, 2048, 1500
    vals = []
    for seed in range(240):
        d = synth.white_noise(n, 99, 0, seed)
        synth.inject(d, h, 0, n_c, A, 0.3)
        vals.append(abs(oracle.complex_snr(oracle.lloid_snr(bank, d))[0, n_c]))
    x = -A * A / 2
    lag = math.exp(x / 2) * ((1 - x) * scipy.special.i0(-x / 2) - x * scipy.special.i1(-x / 2))
    mean = math.sqrt(math.pi / 2) * lag
    var = 2 + A * A - mean ** 2
    assert abs(np.mean(vals) - mean) <= 3 * math.sqrt(var / len(vals))


# ---------------------------------------------------------------- P9 window max
def test_p9_window_max_brute_force_with_ties():
    """First-index tie-break, strict '>' threshold, windows on absolute multiples of W."""
    g = np.random.default_rng(5)
    x = g.standard_normal((6, 100))
    x[0, 13] = 5.0; x[1, 13] = 0.0
    x[0, 17] = 3.0; x[1, 17] = 4.0               # |rho| = 5 tie, later index
    x[2, 40:] = 0.0; x[3, 40:] = 0.0
    x[2, 44] = 2.0; x[2, 47] = -2.0              # tie with opposite signs
    W = 20
    wins, n_star, amax, ph = oracle.window_maxima(x, W, 100)
    for wi, w in enumerate(wins):
        for i in range(3):
            best, arg = -1.0, -1
            for n in range(w * W, (w + 1) * W):
                v = math.hypot(x[2 * i, n], x[2 * i + 1, n])
                if v > best:
                    best, arg = v, n
            assert n_star[wi, i] == arg and abs(amax[wi, i] - best) <= 1e-15
    assert n_star[0, 0] == 13 and n_star[2, 1] == 44
    trig = oracle.triggers(x, W, 5.0, 100)
    assert all(t[3] > 5.0 for t in trig)
    assert not any(t[0] == 0 and t[2] == 0 for t in trig)     # |rho| = 5 is not > 5


# ---------------------------------------------------------------- P10 shift invariance
def test_p10_shift_by_rate_period_is_exact(cfg_small):
    """Prepending 2^kmax zeros shifts the output by exactly 2^kmax samples.

    Every rate's signal starts at its own index 0, so the first template length
    plus the resampler spans is a start-up transient and is excluded, and so is
    the end, where the shifted input lost its last samples.
    """
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    d = synth.white_noise(12 * 2048, 8, 0, 0)
    sh = 2 ** bank.k_max
    d2 = np.concatenate([np.zeros(sh, np.float32), d[:-sh]])
    x1 = oracle.lloid_snr(bank, d)
    x2 = oracle.lloid_snr(bank, d2)
    skip = int(spec.duration_s * spec.top_rate_hz) + 8 * 2 * HALF_K * sh
    end = d.shape[0] - sh - 8 * 2 * HALF_K * sh          # the dropped tail reaches back this far
    assert np.abs(x2[:, skip + sh:end + sh] - x1[:, skip:end]).max() <= 1e-12 * np.abs(x1).max()


# ---------------------------------------------------------------- P11 sub-sample peak
def test_p11_subsample_vertex_is_the_exact_parabola():
    """The vertex equals that of numpy.polyfit's degree-2 fit through the three samples of |rho|^2
    (an exact interpolation), and non-maxima are refused."""
    g = np.random.default_rng(11)
    for _ in range(200):
        x = g.standard_normal((2, 7))
        n = 3
        rho2 = x[0] ** 2 + x[1] ** 2
        res = oracle.subsample_peak(x, 0, n)
        is_max = rho2[n] >= rho2[n - 1] and rho2[n] >= rho2[n + 1] and rho2[n - 1] - 2 * rho2[n] + rho2[n + 1] < 0
        if not is_max:
            assert res is None
            continue
        a, b, c = np.polyfit([-1.0, 0.0, 1.0], rho2[n - 1:n + 2], 2)
        t_v = -b / (2 * a)
        assert abs(res[1] - t_v) <= 1e-12 and abs(t_v) <= 0.5
        assert abs(res[0] ** 2 - (c - b * b / (4 * a))) <= 1e-12 * rho2[n]
    edge = np.ones((2, 4))
    assert oracle.subsample_peak(edge, 0, 0) is None and oracle.subsample_peak(edge, 0, 3) is None


def test_p11_subsample_peak_recovers_a_fractional_delay(cfg_small):
    """A noise-free injection delayed by a fraction tau of a sample (band-limited shift): the
    on-grid maximum loses SNR, the sub-sample peak is closer to A and sits near n_c + tau."""
    spec, h = cfg_small
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices, frac=1.0)
    n = 12 * 2048
    n_c, i, A = 10 * 2048 + 5, 7, 12.0
    base = np.zeros(n)
    synth.inject(base, h, i, n_c, A, 0.4)
    spec_f = np.fft.rfft(base)
    k = np.arange(spec_f.shape[0])
    for tau in (-0.4, -0.15, 0.2, 0.35):
        d = np.fft.irfft(spec_f * np.exp(-2j * np.pi * k * tau / n), n).astype(np.float32)
        x = oracle.lloid_snr(bank, d)
        mag = np.abs(oracle.complex_snr(x)[i, n_c - 4:n_c + 5])
        n_star = n_c - 4 + int(np.argmax(mag))
        grid = float(mag.max())
        pk, dt = oracle.subsample_peak(x, i, n_star)
        assert abs(pk - A) < abs(grid - A)
        assert abs(n_star + dt - (n_c + tau)) <= 0.1


# ---------------------------------------------------------------- P12 xi^2 signal consistency
XI_J = 16


def test_p12_autocorrelation_matches_fft_and_symmetries(cfg_small):
    """R_i[j] equals the FFT cross-correlation of the complex template with itself (zero padded),
    R_i[0] = 1 and R_i[-j] = conj(R_i[j])."""
    spec, h = cfg_small
    R = oracle.autocorrelation(h[:8], XI_J)
    for i in range(4):
        c = h[2 * i].astype(np.float64) + 1j * h[2 * i + 1]
        n = 2 * c.shape[0]
        F = np.fft.fft(c, n)
        corr = np.fft.ifft(F * np.conj(F))
        ref = np.array([corr[j % n] for j in range(-XI_J, XI_J + 1)]) / np.sum(np.abs(c) ** 2)
        assert np.abs(R[i] - ref).max() <= 1e-12
        assert abs(R[i, XI_J] - 1.0) <= 1e-14
        assert np.abs(R[i, :XI_J][::-1] - np.conj(R[i, XI_J + 1:])).max() <= 1e-14


def test_p12_xi2_is_one_on_average_in_white_noise(cfg_small):
    """In unit-variance white noise the numerator's expectation is the denominator, so the mean of
    xi^2 at fixed samples is 1 (a missing factor 2, a conjugate or a reversed lag fails)."""
    spec, h = cfg_small
    hs = h[:8]
    R = oracle.autocorrelation(hs, XI_J)
    N = hs.shape[1]
    d = synth.white_noise(N + 60 * 2048, 12, 0, 0)
    x = oracle.direct_snr(hs, d)
    vals = [oracle.xi2(x, R, i, n, XI_J) for i in range(4) for n in range(N + 64, x.shape[1] - 64, 97)]
    m = float(np.mean(vals))
    assert abs(m - 1.0) <= 0.04, m
    assert np.all(np.array(vals) > 0.0)
    # without the factor 2 of the complex series' variance the mean would be 2
    half = [v * float(np.sum(2.0 - 2.0 * np.abs(R[i]) ** 2)) / float(np.sum(1.0 - np.abs(R[i]) ** 2))
            for v, i in zip(vals, [i for i in range(4) for _ in range(N + 64, x.shape[1] - 64, 97)])]
    assert abs(float(np.mean(half)) - 2.0) <= 0.08


def test_p12_xi2_separates_a_matched_signal_from_a_mismatched_one(cfg_small):
    """Noise-free: a template's own injection gives xi^2 ~ 0 at its peak; the same data filtered by
    another template of the bank (its own SNR peak) gives xi^2 far above that; the lag-reversed
    autocorrelation (R[-j] for R[j]) is not consistent with the matched peak either."""
    spec, h = cfg_small
    R = oracle.autocorrelation(h, XI_J)
    N = h.shape[1]
    n_c, A = N + 3 * 2048 + 11, 12.0
    d = np.zeros(n_c + 2 * 2048)
    synth.inject(d, h, 3, n_c, A, 0.7)
    x = oracle.direct_snr(h, d)
    rho = np.abs(oracle.complex_snr(x))
    n3 = int(np.argmax(rho[3]))
    assert n3 == n_c
    matched = oracle.xi2(x, R, 3, n3, XI_J)
    reversed_lag = oracle.xi2(x, R[3, ::-1], 3, n3, XI_J)
    others = []
    for i in (0, 9, 14):
        n_i = n_c - 1024 + int(np.argmax(rho[i, n_c - 1024:n_c + 1024]))
        others.append(oracle.xi2(x, R, i, n_i, XI_J) / (rho[i, n_i] ** 2))
    per_snr2 = matched / A ** 2
    assert per_snr2 <= 1e-4, per_snr2
    assert reversed_lag / A ** 2 > 100 * per_snr2
    assert min(others) > 100 * per_snr2, (others, per_snr2)


# ---------------------------------------------------------------- P13 coincidence generator
def _coinc_fixture():
    path = os.path.join(os.path.dirname(__file__), "golden", "coinc_hand_worked.txt")
    A, B, P = [], [], {}
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "A":
            A.append((int(f[1]), int(f[2]), float(f[3])))
        elif f[0] == "B":
            B.append((int(f[1]), int(f[2]), float(f[3])))
        else:
            P.setdefault(int(f[1]), []).append((int(f[2]), int(f[3]), int(f[4]), int(f[5]), int(f[6]), float(f[7])))
    return A, B, P


def test_p13_coincidences_match_the_hand_worked_fixture():
    A, B, P = _coinc_fixture()
    for max_dt, want in P.items():
        got = oracle.coincidences([a[0] for a in A], [a[1] for a in A], [a[2] for a in A],
                                  [b[0] for b in B], [b[1] for b in B], [b[2] for b in B], max_dt)
        assert [g[:5] for g in got] == [w[:5] for w in want]
        assert all(abs(g[5] ** 2 - w[5]) <= 1e-9 for g, w in zip(got, want))


def test_p13_coincidences_symmetry_and_window_monotonicity():
    """Swapping the detectors swaps the roles of every pair; a wider window keeps every pair of a
    narrower one; max_dt = 0 pairs equal samples only."""
    g = np.random.default_rng(13)
    ta, sa, ra = g.integers(0, 6, 60), g.integers(0, 3000, 60), g.uniform(6, 20, 60)
    tb, sb, rb = g.integers(0, 6, 50), g.integers(0, 3000, 50), g.uniform(6, 20, 50)
    ab = oracle.coincidences(ta, sa, ra, tb, sb, rb, 40)
    ba = oracle.coincidences(tb, sb, rb, ta, sa, ra, 40)
    assert sorted((t, i, j) for t, i, j, *_ in ab) == sorted((t, j, i) for t, i, j, *_ in ba)
    narrow = {(t, i, j) for t, i, j, *_ in oracle.coincidences(ta, sa, ra, tb, sb, rb, 10)}
    assert narrow <= {(t, i, j) for t, i, j, *_ in ab} and len(narrow) < len(ab)
    sb2 = sb.copy()
    sb2[:10] = sa[:10]
    tb2 = tb.copy()
    tb2[:10] = ta[:10]
    zero = oracle.coincidences(ta, sa, ra, tb2, sb2, rb, 0)
    assert all(r[3] == r[4] for r in zero) and {(i, j) for _, i, j, *_ in zero} >= {(k, k) for k in range(10)}


# ---------------------------------------------------------------- P14 whitening (R28)
def test_p14_fixed_psd_returns_the_scaled_input():
    """With a known flat PSD s^2 the whitener must return d / s exactly past the first hop (the
    window's shifted copies sum to one and rfft / irfft are inverses) and w[n] d[n] / s in the
    first hop.  A wrong window, hop, overlap-add offset or FFT normalisation fails this."""
    N, s = 64, 2.5
    d = np.random.default_rng(1).standard_normal(N * 10)
    x, _ = oracle.condition.whiten(d, N, 4, psd=np.full(N // 2 + 1, s * s))
    H = N // 2
    assert x.shape[0] == (d.shape[0] - N) // H * H + H
    assert np.allclose(x[H:], d[H:x.shape[0]] / s, rtol=0, atol=1e-12)
    w = np.sin(np.pi * np.arange(H) / N) ** 2
    assert np.allclose(x[:H], w * d[:H] / s, rtol=0, atol=1e-12)


def test_p14_running_average_is_the_mean_then_exponential():
    """For the first n_avg segments the running PSD equals numpy's mean of the periodograms so far;
    a constant periodogram stays constant; later segments weigh 1 / n_avg."""
    rng = np.random.default_rng(2)
    S = rng.exponential(1.0, size=(12, 9))
    P = oracle.condition.running_psd(S, 5)
    for j in range(5):
        assert np.allclose(P[j], S[:j + 1].mean(axis=0), rtol=1e-13, atol=0)
    assert np.allclose(P[5], 0.8 * P[4] + 0.2 * S[5], rtol=1e-13, atol=0)
    assert np.allclose(oracle.condition.running_psd(np.full((7, 3), 4.0), 3), 4.0, rtol=0, atol=1e-14)


def test_p14_periodogram_normalisation_against_a_tone():
    """A unit-amplitude cosine on bin k (not 0, not N/2) has |X[k]| = sum(w) / 2 = N / 4 under the
    periodic Hann window (Parseval-free closed form), so S[k] = (N/4)^2 / (3N/8)."""
    N, k = 128, 9
    n = np.arange(N * 3)
    d = np.cos(2 * np.pi * k * n / N)
    X = oracle.condition.segment_spectra(d, N)
    assert np.allclose(np.abs(X[:, k]), N / 4, rtol=1e-12)
    w = oracle.condition.hann_periodic(N)
    assert math.isclose(float(np.sum(w ** 2)), 3 * N / 8, rel_tol=1e-12)


def test_p14_scale_invariance():
    """Whitening divides by the data's own amplitude: c d whitens to the same series."""
    d = np.random.default_rng(3).standard_normal(4096)
    x1, _ = oracle.condition.whiten(d, 256, 8)
    x2, _ = oracle.condition.whiten(7.5 * d, 256, 8)
    assert np.allclose(x1, x2, rtol=1e-10, atol=1e-12)


def test_p14_white_noise_stays_white_with_unit_variance():
    """sigma = 3 white noise whitens to unit variance, uncorrelated samples (statistics over 2^18)."""
    N = 512
    d = 3.0 * np.random.default_rng(4).standard_normal(1 << 18)
    x, P = oracle.condition.whiten(d, N, 32)
    xs = x[32 * N:]                                    # past the running average's start-up
    assert abs(xs.var() - 1.0) < 0.02
    assert abs(np.corrcoef(xs[:-1], xs[1:])[0, 1]) < 0.01
    assert abs(np.median(P[-1][1:-1]) / 9.0 - 1.0) < 0.2      # per-bin variance ~ sigma^2 (chi^2 spread)


def test_p14_coloured_noise_whitens_to_a_flat_spectrum():
    """AR(1) noise d[n] = a d[n-1] + e[n] has the per-bin variance 1 / |1 - a e^{-i w}|^2: the
    running PSD follows it (band averages within 5 %) and the whitened output's averaged
    periodogram is flat within 6 % with unit variance, although the input spans 25 dB."""
    a, N = 0.9, 512
    e = np.random.default_rng(5).standard_normal(1 << 19)
    d = scipy.signal.lfilter([1.0], [1.0, -a], e)
    x, P = oracle.condition.whiten(d, N, 64)
    f = np.arange(N // 2 + 1)
    theory = 1.0 / np.abs(1.0 - a * np.exp(-2j * np.pi * f / N)) ** 2
    Pm = P[-64:].mean(axis=0)
    for lo in range(8, N // 2 - 16, 16):                # band averages away from DC
        r = Pm[lo:lo + 16].mean() / theory[lo:lo + 16].mean()
        assert abs(r - 1.0) < 0.05, (lo, r)
    xs = x[64 * N:]
    assert abs(xs.var() - 1.0) < 0.03
    _, pxx = scipy.signal.welch(xs, nperseg=256)
    band = pxx[1:121].reshape(-1, 8).mean(axis=1)        # 15 bands of 8 bins (of 129), DC excluded
    assert band.max() / band.min() < 1.12, band


# ---------------------------------------------------------------- P15 gating (R29)
def test_p15_gate_matches_the_hand_worked_fixture():
    path = os.path.join(os.path.dirname(__file__), "golden", "gate_hand_worked.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    x = np.ones(40)
    x[10], x[30] = 10.0, -12.0
    y = oracle.condition.gate(x, 5.0, 2, 4)
    for n, v in rows:
        assert abs(y[int(n)] - float(v)) < 1e-12, (n, y[int(n)], v)
    assert np.array_equal(oracle.condition.gate(x, 50.0, 2, 4), x)          # nothing above threshold


def test_p15_a_loud_glitch_is_removed_and_the_rest_untouched():
    """A sine-Gaussian glitch of peak 500 sigma in white noise: after conditioning every sample
    within `half` of a sample above the threshold is zero, and samples farther than
    half + taper from all of them equal the ungated whitened series exactly."""
    N, half, taper, thr = 512, 200, 100, 25.0
    rng = np.random.default_rng(6)
    d = rng.standard_normal(1 << 16)
    c = 40000
    n = np.arange(d.shape[0])
    d += 500.0 * np.exp(-0.5 * ((n - c) / 6.0) ** 2) * np.sin(0.9 * (n - c))
    xw, _ = oracle.condition.whiten(d, N, 16)
    xg, _ = oracle.condition.condition(d, N, 16, thr, half, taper)
    centers = np.flatnonzero(np.abs(xw) > thr)
    assert centers.size > 0 and np.all(np.abs(centers - c) < 64)
    r = np.min(np.abs(np.arange(xw.shape[0])[:, None] - centers[None, :]), axis=1)
    assert np.all(xg[r <= half] == 0.0)
    assert np.array_equal(xg[r >= half + taper], xw[r >= half + taper])
    mid = r == half + taper // 2
    assert np.allclose(xg[mid], 0.5 * xw[mid], rtol=1e-12)

