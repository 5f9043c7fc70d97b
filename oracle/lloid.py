"""Oracle: direct matched filter and the LLOID multirate SVD filter, FP64 on the CPU.

Follows the filtering stage of Sec. II.A: the conditioned (here: already
white) strain is down-sampled to each slice rate, cross-correlated with the
orthonormal basis filters, the "orthogonal SNR" series are multiplied by the
SVD coefficients, and the per-slice SNR segments are up-sampled and summed;
SNR peaks above a threshold become triggers, with their phase (Sec. II.A,
Fig. 1 caption).

Notation: f0 top rate, n top-rate sample, a = 2i + p real filter (p = 0
cosine, p = 1 sine), slice s at level k_s (rate f0/2^k_s), delay
D_s = t_s f_s, Q_s taps, L_s basis vectors.

    direct:   x_a[n] = sum_{j<N} h_a[j] d[n - j]                    (d = 0 for n < 0)
    a1:       d^(k+1)[m] = sum_j g[j] d^(k)[2m - j]
    a2:       o_{s,l}[m] = sum_{q<Q_s} v_{s,l}[q] d^(k_s)[m - D_s - q]
    a3:       c_{s,a}[m] = sum_l M_s[a,l] o_{s,l}[m]
    a4:       y^(kmax) = sum_{s: k_s = kmax} c_s;
              y^(k-1)[n] = sum_m 2 g[n - 2m] y^(k)[m] + sum_{s: k_s = k-1} c_s[n];  x = y^(0)
    a5:       rho_i = x_{2i} + i x_{2i+1}; per window [wW f0, (w+1)W f0): n* = first argmax |rho_i|,
              a trigger if |rho_i[n*]| > threshold, phase = atan2(x_{2i+1}, x_{2i}).

Convolutions are evaluated with numpy's FFT (a library primitive; the FFT
against brute-force sums is one of this oracle's pins).

Test infrastructure only: nothing in the product imports this package.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

from .resample import decimate, halfband, upsample
from .svdbank import OracleBank


def _nfft(n: int) -> int:
    return 1 << max(1, (n - 1).bit_length())


def causal_correlate(filters: np.ndarray, d: np.ndarray, delay: int = 0,
                     rows_per_chunk: int = 64) -> np.ndarray:
    """out[r, m] = sum_q filters[r, q] d[m - delay - q] for m in [0, len(d)); d = 0 outside."""
    filters = np.atleast_2d(filters)
    R, Q = filters.shape
    n = d.shape[0]
    out = np.zeros((R, n))
    if delay >= n:
        return out
    nf = _nfft(n + Q)
    D = np.fft.rfft(d, nf)
    for r0 in range(0, R, rows_per_chunk):
        F = np.fft.rfft(filters[r0:r0 + rows_per_chunk], nf, axis=1)
        full = np.fft.irfft(F * D[None, :], nf, axis=1)
        out[r0:r0 + rows_per_chunk, delay:] = full[:, : n - delay]
    return out


def direct_snr(h: np.ndarray, strain: np.ndarray) -> np.ndarray:
    """x_a[n] = sum_j h_a[j] d[n - j]: the full-template correlation (no SVD, no resampling)."""
    return causal_correlate(h, strain.astype(np.float64))


def decimation_cascade(strain: np.ndarray, k_max: int, g: np.ndarray) -> List[np.ndarray]:
    """[d^(0), d^(1), ..., d^(k_max)] with d^(0) = strain (FP64)."""
    out = [strain.astype(np.float64)]
    for _ in range(k_max):
        out.append(decimate(out[-1], g))
    return out


def basis_outputs(bank: OracleBank, levels: List[np.ndarray]) -> List[np.ndarray]:
    """o_s [L_s, n_k] for every slice (step a2)."""
    return [causal_correlate(s.basis, levels[s.level], s.delay) for s in bank.slices]


def lloid_levels(bank: OracleBank, strain: np.ndarray, g: np.ndarray = None) -> Dict[int, np.ndarray]:
    """y^(k) [2M, n/2^k] for every level k (steps a1-a4); y^(0) is the top-rate SNR x."""
    if g is None:
        g = halfband()
    n = strain.shape[0]
    if n % (2 ** bank.k_max):
        raise ValueError("strain length must be a multiple of 2^k_max")
    levels = decimation_cascade(strain, bank.k_max, g)
    return mix_and_sum(bank, basis_outputs(bank, levels), n, g)


def mix_and_sum(bank: OracleBank, o: List[np.ndarray], n: int, g: np.ndarray = None,
                rows: np.ndarray = None) -> Dict[int, np.ndarray]:
    """Steps a3-a4 from the basis outputs o (one [L_s, n/2^k_s] array per slice): y^(k) for
    every level, for the real filters `rows` (default: all 2M, in order)."""
    if g is None:
        g = halfband()
    k_max = bank.k_max
    c_by_level: Dict[int, np.ndarray] = {}
    for s, os_ in zip(bank.slices, o):
        mix = s.mixing if rows is None else s.mixing[rows]
        c = mix @ os_
        c_by_level[s.level] = c_by_level.get(s.level, 0.0) + c
    n_rows = 2 * bank.n_templates if rows is None else len(rows)
    y: Dict[int, np.ndarray] = {}
    y[k_max] = c_by_level.get(k_max, np.zeros((n_rows, n >> k_max)))
    for k in range(k_max, 0, -1):
        y[k - 1] = upsample(y[k], g) + c_by_level.get(k - 1, 0.0)
    return y


def lloid_snr(bank: OracleBank, strain: np.ndarray, g: np.ndarray = None) -> np.ndarray:
    """x [2M, n]: the multirate SVD reconstruction of every real filter's SNR series."""
    return lloid_levels(bank, strain, g)[0]


def complex_snr(x: np.ndarray) -> np.ndarray:
    """rho_i = x_{2i} + i x_{2i+1}."""
    return x[0::2] + 1j * x[1::2]


def window_maxima(x: np.ndarray, window_len: int, n_valid: int, n_start: int = 0):
    """Per (window, template): first argmax of |rho| over [w W, (w+1) W).

    Only windows lying entirely inside [n_start, n_valid) are returned.
    Returns (windows [nw], n_star [nw, M], abs_rho [nw, M], phase [nw, M]).
    """
    rho = complex_snr(x)
    w0 = -(-n_start // window_len)
    w1 = n_valid // window_len
    wins = np.arange(w0, w1)
    M = rho.shape[0]
    n_star = np.zeros((len(wins), M), dtype=np.int64)
    amax = np.zeros((len(wins), M))
    ph = np.zeros((len(wins), M))
    for wi, w in enumerate(wins):
        seg = rho[:, w * window_len:(w + 1) * window_len]
        mag = np.abs(seg)
        j = np.argmax(mag, axis=1)             # first index of the maximum
        n_star[wi] = w * window_len + j
        pick = seg[np.arange(M), j]
        amax[wi] = np.abs(pick)
        ph[wi] = np.arctan2(pick.imag, pick.real)
    return wins, n_star, amax, ph


def triggers(x: np.ndarray, window_len: int, threshold: float, n_valid: int,
             n_start: int = 0) -> List[Tuple[int, int, int, float, float]]:
    """(template, sample, window, |rho|, phase) for each window maximum with |rho| > threshold."""
    wins, n_star, amax, ph = window_maxima(x, window_len, n_valid, n_start)
    out = []
    for wi, w in enumerate(wins):
        for i in np.nonzero(amax[wi] > threshold)[0]:
            out.append((int(i), int(n_star[wi, i]), int(w), float(amax[wi, i]), float(ph[wi, i])))
    return out


def subsample_peak(x: np.ndarray, i: int, n: int):
    """Sub-sample peak of template i around sample n.

    Sec. III attributes the small SNR gap to GstLAL to its sub-sample
    interpolation at peak finding (left as future work there); the method is
    not given.  Reading: the vertex of the parabola through |rho|^2 at
    n - 1, n, n + 1, taken only when n is a local maximum with both neighbours
    inside the series.  Returns (|rho| at the vertex, vertex offset from n in
    samples) or None.
    """
    if n < 1 or n + 1 >= x.shape[1]:
        return None
    rho2 = x[2 * i, n - 1:n + 2] ** 2 + x[2 * i + 1, n - 1:n + 2] ** 2
    ym, y0, yp = (float(v) for v in rho2)
    den = ym - 2.0 * y0 + yp
    if not (y0 >= ym and y0 >= yp and den < 0.0):
        return None
    dt = 0.5 * (ym - yp) / den
    return float(np.sqrt(y0 - 0.25 * (ym - yp) * dt)), dt



def autocorrelation(h: np.ndarray, J: int) -> np.ndarray:
    """R_i[j], j = -J..J: the normalised complex autocorrelation of template i.

    Sec. II.A computes the signal-consistency value xi^2 for every trigger,
    following the GstLAL method it cites.  Reading: with h_i = h_{2i} + i h_{2i+1}
    (the cosine and sine phases at f0),
        R_i[j] = sum_q h_i[q] conj(h_i[q - j]) / sum_q |h_i[q]|^2,
    so R_i[0] = 1, R_i[-j] = conj(R_i[j]), and in white unit-variance noise
    E[rho_i[n + j] conj(rho_i[n])] = 2 R_i[j].  A matched signal of phase phi
    gives rho_i[n_c + j] ~ A e^{i phi} R_i[j].  Returns [M, 2J + 1] complex.
    """
    M, N = h.shape[0] // 2, h.shape[1]
    out = np.empty((M, 2 * J + 1), dtype=np.complex128)
    for i in range(M):
        c = h[2 * i].astype(np.float64) + 1j * h[2 * i + 1].astype(np.float64)
        norm = float(np.sum(np.abs(c) ** 2))
        for j in range(-J, J + 1):
            if j >= 0:
                s = np.sum(c[j:] * np.conj(c[:N - j]))
            else:
                s = np.sum(c[:N + j] * np.conj(c[-j:]))
            out[i, j + J] = s / norm
    return out


def xi2(x: np.ndarray, R: np.ndarray, i: int, n: int, J: int):
    """xi^2 of template i at sample n (Sec. II.A; reading of the cited method).

        xi^2 = sum_{|j|<=J} |rho[n + j] - rho[n] R[j]|^2 / sum_{|j|<=J} (2 - 2 |R[j]|^2)

    The denominator is the numerator's expectation in white noise, so xi^2 is
    about 1 for noise and near 0 for a signal that matches the template.
    Returns None unless all of n - J .. n + J lie inside the series.
    """
    if n - J < 0 or n + J >= x.shape[1]:
        return None
    z = x[2 * i, n - J:n + J + 1] + 1j * x[2 * i + 1, n - J:n + J + 1]
    r = R[i] if R.ndim == 2 else R
    num = float(np.sum(np.abs(z - z[J] * r) ** 2))
    den = float(np.sum(2.0 - 2.0 * np.abs(r) ** 2))
    return num / den
