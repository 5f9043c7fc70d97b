"""Host-side setup: time-slice a template group and decompose each slice by SVD.

This is the setup stage of Sec. II.A (templates grouped, split into time
slices sampled at their own rates, each slice decomposed by SVD into
orthonormal basis filters and coefficients).  It runs once per bank, in FP64
on the host; its output is what ``svdbank_create`` consumes.

Slice s covers [t_s, t_{s+1}) seconds before coalescence at rate
f_s = f0 / 2^k.  Its filter matrix takes every 2^k-th template sample starting
t_s f0 samples before coalescence, scaled by 2^k (the decimated data carry
1/2^k of the band's samples).  The SVD keeps the fewest basis vectors whose
squared singular values reach ``keep_power`` of the total.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class BankSlice:
    rate_hz: float
    t_start_s: float
    t_end_s: float
    basis: np.ndarray      # [L, Q]: orthonormal rows
    mixing: np.ndarray     # [2M, L]


@dataclasses.dataclass
class SVDBank:
    n_templates: int
    top_rate_hz: float
    slices: List[BankSlice]
    autocorr: Optional[np.ndarray] = None      # [M, 2 J + 1] complex, for the xi^2 of each trigger

    def basis_counts(self) -> List[int]:
        return [s.basis.shape[0] for s in self.slices]


def decompose(templates: np.ndarray, top_rate_hz: float, slice_specs: Sequence,
              keep_power: float = 0.9999) -> SVDBank:
    """templates: [2M, N] real filters (row 2i cosine, 2i+1 sine), sample j = j/f0 s before coalescence."""
    twoM, N = templates.shape
    out = []
    for sp in slice_specs:
        level = int(round(math.log2(top_rate_hz / sp.rate_hz)))
        stride = 1 << level
        first = int(round(sp.t_start_s * top_rate_hz))
        taps = int(round((sp.t_end_s - sp.t_start_s) * sp.rate_hz))
        cols = first + stride * np.arange(taps)
        if cols[-1] >= N:
            raise ValueError("slice extends past the template length")
        H = float(stride) * templates[:, cols]
        u, sig, vt = np.linalg.svd(H, full_matrices=False)
        energy = np.cumsum(sig * sig)
        rank = min(int(np.searchsorted(energy, keep_power * energy[-1])) + 1, sig.size)
        out.append(BankSlice(sp.rate_hz, sp.t_start_s, sp.t_end_s,
                             np.ascontiguousarray(vt[:rank]), np.ascontiguousarray(u[:, :rank] * sig[:rank])))
    return SVDBank(twoM // 2, top_rate_hz, out, template_autocorrelation(templates, XI2_HALF))


XI2_HALF = 16        # lags -16 .. 16 (SB_XI2_HALF)


def template_autocorrelation(templates: np.ndarray, half: int) -> np.ndarray:
    """R_i[j] = sum_q h_i[q] conj(h_i[q - j]) / sum_q |h_i[q]|^2 for j = -half .. half, with
    h_i = templates[2i] + i templates[2i + 1]: the lag profile of a matched peak (rho[n_c + j] ~
    rho[n_c] R_i[j]) that the signal-consistency value compares against.  By FFT, zero padded."""
    twoM, N = templates.shape
    c = templates[0::2].astype(np.float64) + 1j * templates[1::2].astype(np.float64)
    nfft = 1 << int(math.ceil(math.log2(2 * N)))
    F = np.fft.fft(c, nfft, axis=1)
    corr = np.fft.ifft(F * np.conj(F), axis=1)
    lags = np.arange(-half, half + 1) % nfft
    return corr[:, lags] / np.sum(np.abs(c) ** 2, axis=1, keepdims=True)
