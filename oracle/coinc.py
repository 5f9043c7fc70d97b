"""Oracle: the coincidence generator that follows the filter (Sec. II.A).

Sec. II.A passes the triggers of every detector to a coincidence generator that
pairs triggers found with the same template within the light-travel time
between the detectors.  Reading: a trigger a of detector A and a trigger b of
detector B coincide when a.template_id == b.template_id and
|a.sample - b.sample| <= max_dt (top-rate samples; the caller converts the
light-travel time plus any timing margin).  Every such pair is reported, with
the network SNR sqrt(snr_a^2 + snr_b^2), in the order (template_id, sample_a,
sample_b, index_a, index_b).

Test infrastructure only: nothing in the product imports this package.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def coincidences(tid_a: Sequence[int], sample_a: Sequence[int], snr_a: Sequence[float],
                 tid_b: Sequence[int], sample_b: Sequence[int], snr_b: Sequence[float],
                 max_dt: int) -> List[Tuple[int, int, int, int, int, float]]:
    """All pairs (template_id, index_a, index_b, sample_a, sample_b, network_snr), by brute force."""
    out = []
    for i in range(len(tid_a)):
        for j in range(len(tid_b)):
            if int(tid_a[i]) != int(tid_b[j]):
                continue
            if abs(int(sample_a[i]) - int(sample_b[j])) > max_dt:
                continue
            out.append((int(tid_a[i]), i, j, int(sample_a[i]), int(sample_b[j]),
                        math.sqrt(float(snr_a[i]) ** 2 + float(snr_b[j]) ** 2)))
    out.sort(key=lambda r: (r[0], r[3], r[4], r[1], r[2]))
    return out
