"""Oracle: the halfband resampler used by the LLOID cascade (FP64, CPU).

The paper states only that LLOID "down-samples" the conditioned data and
"up-samples and sums" the per-slice SNR segments (Sec. II.A); it gives no
filter design.  Reading used here (one halfband kernel, cascaded one octave
at a time):

* g[j], |j| <= 2K, K = 16 (65 taps), is a Kaiser-windowed halfband low-pass:
  g[0] = 1/2, g[j] = 0 for even j != 0, and the odd taps are proportional to
  sinc(j/2) * w_Kaiser,beta(j) (beta = 8.6), scaled so that they sum to 1/2.
  Then sum_j g[j] = 1 (unit DC gain) and H(w) + H(pi - w) = 1 exactly.
* decimation by two: d'[m] = sum_j g[j] d[2m - j];
* interpolation by two: y'[n] = sum_m 2 g[n - 2m] y[m];
  even outputs are copies: y'[2m] = y[m].
* Every signal starts at index 0: samples at negative indices are zero at
  every rate, and samples past the end of the array are zero (the oracle is
  zero-phase and non-causal).

Test infrastructure only: nothing in the product imports this package.
"""
from __future__ import annotations

import numpy as np

HALF_K = 16          # K: the kernel spans |j| <= 2K
KAISER_BETA = 8.6


def bessel_i0(x: float, terms: int = 60) -> float:
    """Modified Bessel function I0 from its power series sum_k ((x/2)^k / k!)^2."""
    acc, term = 1.0, 1.0
    half = 0.5 * x
    for k in range(1, terms):
        term *= (half / k) ** 2
        acc += term
    return acc


def kaiser(n_half: int, beta: float) -> np.ndarray:
    """Kaiser window on j = -n_half..n_half: I0(beta sqrt(1-(j/n_half)^2)) / I0(beta)."""
    j = np.arange(-n_half, n_half + 1, dtype=np.float64)
    r = np.sqrt(np.maximum(0.0, 1.0 - (j / n_half) ** 2))
    den = bessel_i0(beta)
    return np.array([bessel_i0(beta * v) / den for v in r])


def halfband(K: int = HALF_K, beta: float = KAISER_BETA) -> np.ndarray:
    """The 4K+1 taps g[-2K..2K] (array index j + 2K)."""
    j = np.arange(-2 * K, 2 * K + 1, dtype=np.float64)
    w = kaiser(2 * K, beta)
    g = np.zeros_like(j)
    odd = (np.abs(j).astype(np.int64) % 2) == 1
    x = j[odd] / 2.0
    g[odd] = np.sin(np.pi * x) / (np.pi * x) * w[odd]
    g[odd] *= 0.5 / g[odd].sum()
    g[2 * K] = 0.5
    return g


def decimate(d: np.ndarray, g: np.ndarray) -> np.ndarray:
    """d'[m] = sum_j g[j] d[2m - j] for m in [0, ceil(n/2)); d is zero outside [0, n)."""
    K2 = (g.shape[0] - 1) // 2
    full = np.convolve(d, g)                 # full[i] = sum_j' g[j'] d[i - j']
    n_out = (d.shape[0] + 1) // 2
    return full[K2: K2 + 2 * n_out: 2].copy()


def upsample(y: np.ndarray, g: np.ndarray) -> np.ndarray:
    """y'[n] = sum_m 2 g[n - 2m] y[m] for n in [0, 2 len(y)); rows are independent.

    Accepts one signal (1-D) or a stack of signals (2-D, time on the last axis).
    """
    K2 = (g.shape[0] - 1) // 2
    y2 = np.atleast_2d(y)
    z = np.zeros((y2.shape[0], 2 * y2.shape[1]))
    z[:, 0::2] = y2
    out = np.empty_like(z)
    for r in range(z.shape[0]):
        full = np.convolve(z[r], 2.0 * g)
        out[r] = full[K2: K2 + z.shape[1]]
    return out if y.ndim == 2 else out[0]
