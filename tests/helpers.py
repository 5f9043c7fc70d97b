"""Shared helpers of the GPU parity tests (device path vs the FP64 oracle)."""
import numpy as np

import oracle


def push_and_collect(ctx, units, strains, sizes, on_device=False, device_strains=None):
    """Push `strains` (list per unit) in chunks of `sizes`; return per unit the
    concatenated top-rate SNR x [2M, n] for n in [0, T - latency)."""
    outs = [[] for _ in units]
    firsts = [None for _ in units]
    t = 0
    for sz in sizes:
        chunk = [s[t:t + sz] for s in (device_strains if on_device else strains)]
        ctx.push_group(units, chunk, [t] * len(units), on_device)
        for i, u in enumerate(units):
            f, x = u.snr()
            if x.shape[1] == 0:
                continue
            if firsts[i] is None:
                firsts[i] = f
                assert f == 0
            outs[i].append(x)
        t += sz
    return [np.concatenate(o, axis=1) if o else None for o in outs]


def rho_error(x_gpu, x_orc):
    """max |rho_gpu - rho_orc| / max(1, |rho_orc|) over every template and sample."""
    n = x_gpu.shape[1]
    rg = x_gpu[0::2].astype(np.float64) + 1j * x_gpu[1::2].astype(np.float64)
    ro = x_orc[0::2, :n] + 1j * x_orc[1::2, :n]
    return float((np.abs(rg - ro) / np.maximum(1.0, np.abs(ro))).max())


def rho_abs_error(x_gpu, x_orc):
    """max |rho_gpu - rho_orc| over every template and sample."""
    n = x_gpu.shape[1]
    rg = x_gpu[0::2].astype(np.float64) + 1j * x_gpu[1::2].astype(np.float64)
    ro = x_orc[0::2, :n] + 1j * x_orc[1::2, :n]
    return float(np.abs(rg - ro).max())


def check_triggers(trig, x_orc, win_len, threshold, n_valid, tol, unit=None, template_ids=None, absolute=False):
    """GPU triggers vs the oracle's window maxima on windows inside [0, n_valid).

    Unique facts are compared exactly; where floating point may legitimately
    decide differently (a window maximum within tol of the threshold, or two
    samples within tol of each other), the GPU's choice is checked for validity.
    Returns the number of matched triggers.
    """
    maxima = oracle.window_maxima(x_orc, win_len, n_valid)
    rho = oracle.complex_snr(x_orc)
    return check_triggers_maxima(trig, maxima, lambda i, n: abs(rho[i, n]), rho.shape[0], threshold, tol,
                                 unit=unit, template_ids=template_ids, absolute=absolute)


def check_triggers_maxima(trig, maxima, rho_abs, n_templates, threshold, tol, unit=None, template_ids=None,
                          absolute=False, errors=None):
    """check_triggers against precomputed oracle window maxima (wins, n_star, amax, phase), with
    rho_abs(i, n) = |rho_i[n]| of the oracle.  When `errors` is a list, every matched trigger's
    |snr - oracle maximum| is appended to it."""
    if unit is not None:
        trig = trig[trig["unit"] == unit]
    wins, n_star, amax, ph = maxima
    scale = (lambda m: 1.0) if absolute else (lambda m: max(1.0, m))
    got = {}
    for t in trig:
        key = (int(t["template_id"]), int(t["window"]))
        assert key not in got, f"duplicate trigger {key}"
        got[key] = t
    ids = template_ids if template_ids is not None else np.arange(n_templates)
    matched = 0
    for wi, w in enumerate(wins):
        for i in range(n_templates):
            key = (int(ids[i]), int(w))
            m = amax[wi, i]
            if key in got:
                t = got.pop(key)
                assert m > threshold - tol * scale(m), f"spurious trigger {key}: oracle max {m}"
                assert abs(t["snr"] - m) <= tol * scale(m), (key, t["snr"], m)
                if errors is not None:
                    errors.append(abs(float(t["snr"]) - m))
                n = int(t["sample"])
                if n != n_star[wi, i]:
                    assert abs(rho_abs(i, n) - m) <= 2 * tol * scale(m), (key, n, n_star[wi, i])
                else:
                    dphi = np.angle(np.exp(1j * (t["phase"] - ph[wi, i])))
                    assert abs(dphi) <= 10 * tol * scale(m) / max(m, 1e-3) + 1e-5, (key, dphi)
                matched += 1
            else:
                assert m <= threshold + tol * scale(m), f"missing trigger {key}: oracle max {m}"
    assert not got, f"triggers in windows the oracle has none: {list(got)[:5]}"
    return matched
