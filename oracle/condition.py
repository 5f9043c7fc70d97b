"""Oracle: data conditioning ahead of the filter -- PSD estimate, whitening, gating (Sec. II.A).

Sec. II.A conditions the strain before LLOID: the noise power spectral density
is estimated, a running average of it whitens the data, and large deviations
of the whitened data are gated out (Fig. 1 caption: "whitening and gating").
The paper cites GstLAL for the method and gives no formulas, so the steps
below are readings (recorded in the design notes as R28 and R29), written out
in the order the paper names them.  FP64 numpy; numpy's real FFT is the only
library primitive.

Whitening (R28).  N-sample segments (N even) start every H = N/2 samples:
segment j covers input samples [jH, jH + N), j = 0, 1, ...  (the strain is 0
before sample 0).
    w[n]    = sin^2(pi n / N), n < N            (periodic Hann: sum_j w[n - jH] = 1)
    X_j[f]  = sum_n w[n] d[jH + n] e^{-2 pi i f n / N},  f = 0 .. N/2
    S_j[f]  = |X_j[f]|^2 / sum_n w[n]^2        (the variance of white noise, per bin)
    P_j     = P_{j-1} + (S_j - P_{j-1}) / min(j + 1, n_avg),  P_{-1} = 0
              (the running average: the mean of all periodograms so far for
              the first n_avg segments, then an exponential average of weight
              1 / n_avg)
    Y_j[f]  = X_j[f] / sqrt(P_{j-1}[f])        (P_0 for j = 0; 0 where it is 0)
    z_j     = inverse real DFT of Y_j (N samples)
    x[n]    = sum_j z_j[n - jH]                 (overlap-add)
Each segment is whitened by the average of the segments before it (the
first by its own periodogram), so a loud glitch is not divided by its own
power and stays above the gate's threshold.  White noise of variance s^2 gives P ~ s^2, Y ~ X / s and x ~ d / s: the
window sums to one, so the output keeps the input's time series, divided by
the noise amplitude, bin by bin.  x[n] is final once the segments covering n
are, i.e. for n < J H after J segments; samples [0, H) carry only segment 0
(a start-up taper).

Gating (R29).  Every whitened sample with |x[c]| > threshold is a glitch
sample c.  With r(n) = min_c |n - c| (the distance to the nearest glitch
sample), the gated series is x[n] g(r(n)):
    g(r) = 0                                    r <= half
           sin^2(pi (r - half) / (2 taper))      half < r < half + taper
           1                                    r >= half + taper
so every sample within `half` of a glitch sample is removed and the data
return to full weight over a Hann ramp of `taper` samples.

Test infrastructure only: nothing in the product imports this module.
"""
from __future__ import annotations

import numpy as np


def hann_periodic(N: int) -> np.ndarray:
    """w[n] = sin^2(pi n / N): shifted copies H = N/2 apart sum to one."""
    return np.sin(np.pi * np.arange(N) / N) ** 2


def segment_spectra(d: np.ndarray, N: int) -> np.ndarray:
    """X_j[f] for every complete segment j (rows), f = 0 .. N/2."""
    H = N // 2
    w = hann_periodic(N)
    J = (d.shape[0] - N) // H + 1 if d.shape[0] >= N else 0
    return np.stack([np.fft.rfft(w * d[j * H:j * H + N]) for j in range(J)]) if J else \
        np.zeros((0, H + 1), complex)


def running_psd(S: np.ndarray, n_avg: int) -> np.ndarray:
    """P_j for the periodograms S_j (rows), the running average of R28."""
    P = np.zeros_like(S)
    prev = np.zeros(S.shape[1])
    for j in range(S.shape[0]):
        prev = prev + (S[j] - prev) / min(j + 1, n_avg)
        P[j] = prev
    return P


def whiten(d: np.ndarray, N: int, n_avg: int, psd: np.ndarray = None):
    """Whitened series x[0 .. J H) and the running PSD P_j after each segment j (rows).

    psd: a fixed per-bin variance to divide by instead of the running average
    (a special case used by the pins)."""
    d = np.asarray(d, dtype=np.float64)
    H = N // 2
    X = segment_spectra(d, N)
    w = hann_periodic(N)
    S = np.abs(X) ** 2 / np.sum(w ** 2)
    P = running_psd(S, n_avg) if psd is None else np.broadcast_to(psd, S.shape)
    J = X.shape[0]
    x = np.zeros(J * H + H)
    for j in range(J):
        Pw = P[j - 1] if (j >= 1 and psd is None) else P[j]          # the average of earlier segments
        with np.errstate(divide="ignore", invalid="ignore"):
            Y = np.where(Pw > 0, X[j] / np.sqrt(Pw), 0.0)
        x[j * H:j * H + N] += np.fft.irfft(Y, N)
    return x[:J * H], np.array(P)


def gate(x: np.ndarray, threshold: float, half: int, taper: int) -> np.ndarray:
    """x[n] g(r(n)) with r(n) the distance to the nearest sample where |x| > threshold."""
    x = np.asarray(x, dtype=np.float64)
    centers = np.flatnonzero(np.abs(x) > threshold)
    if threshold <= 0 or centers.size == 0:
        return x.copy()
    n = np.arange(x.shape[0])
    # distance to the nearest glitch sample: the closest center at or after n, and at or before n
    right = np.searchsorted(centers, n, side="left")
    r = np.full(n.shape, np.inf)
    has_r = right < centers.size
    r[has_r] = centers[right[has_r]] - n[has_r]
    has_l = right > 0
    r[has_l] = np.minimum(r[has_l], n[has_l] - centers[right[has_l] - 1])
    g = np.ones_like(x)
    g[r <= half] = 0.0
    ramp = (r > half) & (r < half + taper)
    g[ramp] = np.sin(np.pi * (r[ramp] - half) / (2.0 * taper)) ** 2
    return x * g


def condition(d: np.ndarray, N: int, n_avg: int, threshold: float, half: int, taper: int):
    """Whitening then gating: the conditioned series (final for n < J H) and the PSD estimates."""
    x, P = whiten(d, N, n_avg)
    return gate(x, threshold, half, taper), P
