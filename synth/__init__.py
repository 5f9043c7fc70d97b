"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This module only *draws* inputs: white Gaussian strain, Newtonian-order chirp
templates that stand in for the paper's LAL template bank (Sec. II.A, Sec. III.B),
injections, and the random "shape-only" SVD banks of the batching workload.
It holds none of the matched filter's arithmetic (no resampling, no
correlation, no SVD, no reconstruction, no peak finding); both the oracle and
the CUDA library consume what it returns.

Every random draw comes from ``numpy.random.SeedSequence(20241016)`` keyed by
a tuple (workload, bin, detector, purpose, ...), so any excerpt of any stream
can be regenerated independently.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

ROOT_SEED = 20241016
T_SUN_S = 4.925491e-6          # G * Msun / c^3 in seconds
KIND_NOISE, KIND_BANK, KIND_INJ, KIND_SHAPE = 1, 2, 3, 4


def rng(*key: int) -> np.random.Generator:
    """Generator for a keyed child of the root seed (key = non-negative ints)."""
    ss = np.random.SeedSequence(ROOT_SEED, spawn_key=tuple(int(k) for k in key))
    return np.random.Generator(np.random.PCG64(ss))


# --------------------------------------------------------------------------
# strain
# --------------------------------------------------------------------------
def white_noise(n: int, *key: int) -> np.ndarray:
    """Unit-variance white Gaussian strain, drawn in FP64 and rounded to FP32.

    Both the oracle and the device path read the same FP32 values, so input
    rounding is not part of any parity error.
    """
    return rng(KIND_NOISE, *key).standard_normal(n).astype(np.float32)


def white_noise_block(block: int, block_len: int, *key: int) -> np.ndarray:
    """Block ``block`` (length ``block_len``) of an endless keyed noise stream.

    Streams are generated block-wise so that any excerpt (serving loop, long
    runs) can be regenerated without generating what precedes it.
    """
    return rng(KIND_NOISE, *key, 1_000_000 + block).standard_normal(block_len).astype(np.float32)


# --------------------------------------------------------------------------
# templates: Newtonian-order chirps (stand-in for the paper's bank, Sec. III.B)
# --------------------------------------------------------------------------
def _tau_of_f(f: float, mchirp: float) -> float:
    """Newtonian time to coalescence (s) at gravitational-wave frequency f."""
    return (5.0 / 256.0) * (math.pi * f) ** (-8.0 / 3.0) * (T_SUN_S * mchirp) ** (-5.0 / 3.0)


def newtonian_chirp(mchirp: float, f0: float, duration_s: float,
                    taper_frac: float = 0.05) -> Tuple[np.ndarray, np.ndarray]:
    """Cosine and sine phase of one equal-mass Newtonian chirp, FP64.

    Index j counts samples *before* coalescence at rate f0 (j = 0 is the last
    sample).  f(tau) = pi^-1 (5/(256 tau))^(3/8) (T_sun Mc)^(-5/8),
    Phi(tau) = -2 (tau/(5 T_sun Mc))^(5/8), amplitude ~ tau^(-1/4); the
    waveform ends where f reaches min(f_ISCO, 0.45 f0) and only the last
    ``duration_s`` seconds are kept.  A Tukey taper (Hann ramps over
    ``taper_frac`` of the span at each end) is applied and each phase is
    normalised to unit sum of squares at rate f0.
    """
    n = int(round(duration_s * f0))
    m_total = mchirp / 0.25 ** 0.6                     # equal masses, eta = 1/4
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * m_total * T_SUN_S)
    tau_end = _tau_of_f(min(f_isco, 0.45 * f0), mchirp)
    tau = np.arange(n, dtype=np.float64) / f0 + tau_end
    phase = -2.0 * (tau / (5.0 * T_SUN_S * mchirp)) ** 0.625
    amp = tau ** -0.25
    win = np.ones(n)
    r = max(1, int(taper_frac * n))
    ramp = 0.5 * (1.0 - np.cos(np.pi * np.arange(r) / r))
    win[:r] = ramp                                     # coalescence end
    win[n - r:] = ramp[::-1]                           # early (low-frequency) end
    hc = amp * np.cos(phase) * win
    hs = amp * np.sin(phase) * win
    hc /= math.sqrt(float(np.dot(hc, hc)))
    hs /= math.sqrt(float(np.dot(hs, hs)))
    return hc, hs


def template_bank(n_templates: int, mc_lo: float, mc_hi: float, f0: float,
                  duration_s: float, *key: int) -> Tuple[np.ndarray, np.ndarray]:
    """(h, mchirp): h has 2M rows, row a = 2i + p (p = 0 cosine, p = 1 sine)."""
    mc = np.sort(rng(KIND_BANK, *key).uniform(mc_lo, mc_hi, n_templates))
    n = int(round(duration_s * f0))
    h = np.empty((2 * n_templates, n), dtype=np.float64)
    for i, m in enumerate(mc):
        h[2 * i], h[2 * i + 1] = newtonian_chirp(float(m), f0, duration_s)
    return h, mc


def inject(strain: np.ndarray, h: np.ndarray, template: int, n_c: int,
           amplitude: float, phi0: float) -> None:
    """Add A (cos phi0 h_c + sin phi0 h_s) with coalescence at sample n_c, in place.

    strain[n_c - j] += A (cos phi0 h_{2i}[j] + sin phi0 h_{2i+1}[j]); the
    result is rounded to the strain's dtype.
    """
    wave = amplitude * (math.cos(phi0) * h[2 * template] + math.sin(phi0) * h[2 * template + 1])
    j = np.arange(h.shape[1])
    n = n_c - j
    ok = (n >= 0) & (n < strain.shape[0])
    acc = strain.astype(np.float64)
    acc[n[ok]] += wave[ok]
    strain[:] = acc.astype(strain.dtype)


@dataclasses.dataclass
class Injection:
    template: int
    n_c: int
    amplitude: float
    phi0: float


def injection_plan(n_inj: int, n_templates: int, n_samples: int, f0: float,
                   spacing_s: float, amp_lo: float, amp_hi: float, *key: int) -> List[Injection]:
    """Coalescence times on a jittered grid with at least ``spacing_s`` between them."""
    g = rng(KIND_INJ, *key)
    out = []
    span = int(spacing_s * f0)
    for k in range(n_inj):
        base = (k + 1) * span
        n_c = base + int(g.integers(0, max(1, span // 4)))
        if n_c >= n_samples:
            break
        out.append(Injection(int(g.integers(0, n_templates)), n_c,
                             float(g.uniform(amp_lo, amp_hi)), float(g.uniform(0.0, 2 * math.pi))))
    return out


# --------------------------------------------------------------------------
# workload shapes
# --------------------------------------------------------------------------
@dataclasses.dataclass
class SliceSpec:
    rate_hz: float
    t_start_s: float
    t_end_s: float


@dataclasses.dataclass
class BinSpec:
    """One SVD bin: its templates and its time slices (rate per slice)."""
    n_templates: int
    mc_lo: float
    mc_hi: float
    top_rate_hz: float
    duration_s: float
    slices: List[SliceSpec]


# Small bin: 64 templates, 8 s, slices [0,1) s at 2048 Hz and [1,8) s at 512 Hz.
SMALL_BIN = BinSpec(64, 1.0, 3.0, 2048.0, 8.0,
                    [SliceSpec(2048.0, 0.0, 1.0), SliceSpec(512.0, 1.0, 8.0)])

# Production-shaped bin: 1000 templates, 60 s, six slices 4096 ... 128 Hz.  The
# boundaries keep each slice's starting frequency below 0.8 of its Nyquist rate
# for chirp mass >= 1.0.
PRODUCTION_BIN = BinSpec(1000, 1.0, 1.5, 4096.0, 60.0,
                         [SliceSpec(4096.0, 0.0, 1 / 32), SliceSpec(2048.0, 1 / 32, 1 / 8),
                          SliceSpec(1024.0, 1 / 8, 1 / 2), SliceSpec(512.0, 1 / 2, 4.0),
                          SliceSpec(256.0, 4.0, 20.0), SliceSpec(128.0, 20.0, 60.0)])


# The paper's own benchmark bank (Sec. IV): 1,004 templates of 73 s, one bank per detector of a
# three-detector search.  Same mass range and slicing as the production bin, the last slice
# extended to the template span.
PAPER_BIN = BinSpec(1004, 1.0, 1.5, 4096.0, 73.0,
                    [SliceSpec(4096.0, 0.0, 1 / 32), SliceSpec(2048.0, 1 / 32, 1 / 8),
                     SliceSpec(1024.0, 1 / 8, 1 / 2), SliceSpec(512.0, 1 / 2, 4.0),
                     SliceSpec(256.0, 4.0, 20.0), SliceSpec(128.0, 20.0, 73.0)])


def scaled_bin(spec: BinSpec, n_templates: int) -> BinSpec:
    return dataclasses.replace(spec, n_templates=n_templates)


# --------------------------------------------------------------------------
# shape-only banks for the batching workload (random weights, no templates)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class ShapeSlice:
    rate_hz: float
    t_start_s: float
    t_end_s: float
    basis: np.ndarray      # [L, Q] orthonormal rows, FP64
    mixing: np.ndarray     # [2M, L], FP64


@dataclasses.dataclass
class ShapeBank:
    n_templates: int
    top_rate_hz: float
    slices: List[ShapeSlice]


def shape_only_bank(bin_index: int, top_rate_hz: float = 4096.0,
                    m_range=(200, 2000), s_range=(3, 8), dur_range=(2.0, 120.0),
                    l_range=(50, 600), max_templates: int = 0) -> ShapeBank:
    """Random bank with the shape statistics of a production bin.

    M ~ logU[200, 2000], S ~ U{3..8} slices at rates top/2^s, durations
    ~ logU[2, 120] s, slice boundaries t_s = T (s/S)^2 rounded to 1/f_s,
    L_s ~ logU[50, 600] capped at min(2M, Q_s).  Basis rows are orthonormal
    (randomly chosen, randomly signed DCT-II basis vectors); mixing rows are
    Gaussian, rescaled so that the summed
    white-noise variance of every real filter, sum_s 2^-k_s |M_s[a,:]|^2, is 1.
    """
    g = rng(KIND_SHAPE, bin_index)
    M = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
    if max_templates:
        M = min(M, max_templates)
    S = int(g.integers(s_range[0], s_range[1] + 1))
    T = float(math.exp(g.uniform(math.log(dur_range[0]), math.log(dur_range[1]))))
    slices: List[ShapeSlice] = []
    bounds = [0.0]
    for s in range(1, S + 1):
        f_s = top_rate_hz / 2 ** (s - 1)
        t = T * (s / S) ** 2
        t = round(t * f_s) / f_s
        # at least one low-rate sample per slice; boundary must be on the grid of
        # both adjacent rates (the coarser one is f_s/2)
        f_next = top_rate_hz / 2 ** s
        t = max(t, bounds[-1] + 16.0 / f_s)
        t = math.ceil(t * f_next - 1e-9) / f_next if s < S else math.ceil(t * f_s - 1e-9) / f_s
        bounds.append(t)
    weight = np.zeros(2 * M)
    raw = []
    for s in range(S):
        f_s = top_rate_hz / 2 ** s
        Q = int(round((bounds[s + 1] - bounds[s]) * f_s))
        L = int(round(math.exp(g.uniform(math.log(l_range[0]), math.log(l_range[1])))))
        L = max(1, min(L, 2 * M, Q))
        # L distinct DCT-II basis vectors of length Q with random signs: orthonormal rows
        freq = np.sort(g.choice(Q, size=L, replace=False))
        sign = np.where(g.random(L) < 0.5, -1.0, 1.0)
        qq = np.arange(Q) + 0.5
        V = np.cos(np.pi * freq[:, None] * qq[None, :] / Q) * np.sqrt(2.0 / Q)
        V[freq == 0] *= np.sqrt(0.5)
        V *= sign[:, None]
        Mx = g.standard_normal((2 * M, L))
        weight += (Mx ** 2).sum(axis=1) * 2.0 ** (-s)
        raw.append((f_s, bounds[s], bounds[s + 1], V, Mx))
    scale = 1.0 / np.sqrt(weight)
    for f_s, t0, t1, V, Mx in raw:
        slices.append(ShapeSlice(f_s, t0, t1, V, Mx * scale[:, None]))
    return ShapeBank(M, top_rate_hz, slices)


def production_shape_bank(index: int, top_rate_hz: float = 4096.0) -> ShapeBank:
    """Random bank shaped like the production bin: about 1000 templates (U[800, 1200]),
    its six slices (4096 ... 128 Hz over 60 s) and basis counts near its SVD ranks
    (14, 23, 46, 191, 451, 679, each scaled by U[0.8, 1.2]), orthonormal DCT bases."""
    g = rng(KIND_SHAPE, 100000 + index)
    M = int(g.integers(800, 1201))
    ranks = (14, 23, 46, 191, 451, 679)
    weight = np.zeros(2 * M)
    raw = []
    for s, (sp, r) in enumerate(zip(PRODUCTION_BIN.slices, ranks)):
        Q = int(round((sp.t_end_s - sp.t_start_s) * sp.rate_hz))
        L = max(1, min(int(round(r * g.uniform(0.8, 1.2))), Q, 2 * M))
        freq = np.sort(g.choice(Q, size=L, replace=False))
        qq = np.arange(Q) + 0.5
        V = np.cos(np.pi * freq[:, None] * qq[None, :] / Q) * np.sqrt(2.0 / Q)
        V[freq == 0] *= np.sqrt(0.5)
        Mx = g.standard_normal((2 * M, L))
        k = int(round(math.log2(top_rate_hz / sp.rate_hz)))
        weight += (Mx ** 2).sum(axis=1) * 2.0 ** (-k)
        raw.append((sp, V, Mx))
    scale = 1.0 / np.sqrt(weight)
    return ShapeBank(M, top_rate_hz, [ShapeSlice(sp.rate_hz, sp.t_start_s, sp.t_end_s, V, Mx * scale[:, None])
                                      for sp, V, Mx in raw])
