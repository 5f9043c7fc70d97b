"""Oracle: time slicing and per-slice SVD of a template group (setup stage, Sec. II.A).

The paper splits each group of ~1000 templates into time slices, samples each
slice at its own rate and decomposes it by SVD into orthonormal basis filters
and a coefficient ("mixing") matrix (Sec. II.A).  Readings used here:

* slice s covers tau in [t_s, t_{s+1}) seconds before coalescence at rate
  f_s = f0 / 2^k_s; its filter for real template a is
  h_{a,s}[q] = 2^k_s h_a[t_s f0 + q 2^k_s], q < Q_s = (t_{s+1} - t_s) f_s
  (the 2^k_s factor keeps the amplitude when the data are decimated k_s times);
* H_s = U S V^T; the rank L_s is the smallest L with
  sum_{l<L} sigma_l^2 >= frac * sum_l sigma_l^2 (frac = 0.9999, on the power);
* basis v_{s,l} = row l of V^T (orthonormal), mixing M_s = U[:, :L] diag(sigma[:L]).

Test infrastructure only: nothing in the product imports this package.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np


@dataclasses.dataclass
class OracleSlice:
    rate_hz: float
    t_start_s: float
    t_end_s: float
    level: int            # k_s: f_s = f0 / 2^k_s
    delay: int            # D_s = t_s f_s
    basis: np.ndarray     # [L_s, Q_s]
    mixing: np.ndarray    # [2M, L_s]
    sigma: np.ndarray     # all singular values of H_s (for the truncation pins)


@dataclasses.dataclass
class OracleBank:
    n_templates: int
    top_rate_hz: float
    slices: List[OracleSlice]

    @property
    def k_max(self) -> int:
        return max(s.level for s in self.slices)


def level_of(rate_hz: float, top_rate_hz: float) -> int:
    k = int(round(math.log2(top_rate_hz / rate_hz)))
    if abs(top_rate_hz / 2 ** k - rate_hz) > 1e-9 * rate_hz:
        raise ValueError("slice rate must be the top rate divided by a power of two")
    return k


def slice_filters(h: np.ndarray, top_rate_hz: float, rate_hz: float,
                  t_start_s: float, t_end_s: float) -> np.ndarray:
    """H_s[a, q] = 2^k h[a, t_s f0 + q 2^k]  (templates indexed back from coalescence)."""
    k = level_of(rate_hz, top_rate_hz)
    step = 2 ** k
    j0 = int(round(t_start_s * top_rate_hz))
    Q = int(round((t_end_s - t_start_s) * rate_hz))
    idx = j0 + step * np.arange(Q)
    return step * h[:, idx]


def truncated_svd(H: np.ndarray, frac: float = 0.9999):
    """(basis [L, Q], mixing [2M, L], sigma): keep the smallest L reaching frac of sum sigma^2."""
    U, s, Vt = np.linalg.svd(H, full_matrices=False)
    power = np.cumsum(s ** 2)
    L = int(np.searchsorted(power, frac * power[-1]) + 1)
    L = min(L, s.shape[0])
    return Vt[:L].copy(), U[:, :L] * s[:L], s


def build_bank(h: np.ndarray, top_rate_hz: float, slices: Sequence, frac: float = 0.9999) -> OracleBank:
    """SVD bank from templates h [2M, N] and slice specs (rate_hz, t_start_s, t_end_s)."""
    out = []
    for sp in slices:
        H = slice_filters(h, top_rate_hz, sp.rate_hz, sp.t_start_s, sp.t_end_s)
        if frac >= 1.0:
            U, s, Vt = np.linalg.svd(H, full_matrices=False)
            basis, mixing = Vt, U * s
        else:
            basis, mixing, s = truncated_svd(H, frac)
        k = level_of(sp.rate_hz, top_rate_hz)
        out.append(OracleSlice(sp.rate_hz, sp.t_start_s, sp.t_end_s, k,
                               int(round(sp.t_start_s * sp.rate_hz)), basis, mixing, s))
    return OracleBank(h.shape[0] // 2, top_rate_hz, out)


def bank_from_arrays(n_templates: int, top_rate_hz: float, slices: Sequence) -> OracleBank:
    """Wrap given (rate, t_start, t_end, basis, mixing) slices as an OracleBank."""
    out = []
    for sp in slices:
        k = level_of(sp.rate_hz, top_rate_hz)
        out.append(OracleSlice(sp.rate_hz, sp.t_start_s, sp.t_end_s, k,
                               int(round(sp.t_start_s * sp.rate_hz)),
                               np.asarray(sp.basis, dtype=np.float64),
                               np.asarray(sp.mixing, dtype=np.float64), np.zeros(0)))
    return OracleBank(n_templates, top_rate_hz, out)
