"""Serving: continuous batching under an HBM budget, each stream's result equal alone and in the mix,
and equal to the oracle's filter of the stream's buffers."""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["template_id", "sample", "window", "snr", "phase", "flags"]


@pytest.fixture(scope="module")
def lloid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as m
    return m


def _streams(lloid, n_banks=3, n_buf=6):
    from paper_2410_16416_b300 import serve
    banks = [synth.shape_only_bank(2000 + b, dur_range=(2.0, 6.0), l_range=(5, 40), max_templates=37)
             for b in range(n_banks)]
    g = np.random.default_rng(7)
    reqs = []
    for b, bank in enumerate(banks):
        for det in (0, 1):
            r = len(reqs)
            reqs.append(serve.StreamRequest(
                name=f"bin{b}-det{det}", bank=bank, detector=det,
                arrivals=serve.poisson_arrivals(g, n_buf, 0.6 * r),
                strain=(lambda j, r=r: synth.white_noise_block(j, 4096, 8, r)),
                unit_kwargs=dict(precision="bf16", threshold=3.0, refine_threshold=5.5)))
    return banks, reqs


def _alone(lloid, req, n_buf):
    ctx = lloid.Context(0)
    u = ctx.create_unit(req.bank, detector=req.detector, max_push_samples=4096, **req.unit_kwargs)
    for j in range(n_buf):
        u.push(req.strain(j), j * 4096)
    ctx.sync()
    tr = ctx.pop_triggers()
    ctx.close()
    return np.sort(tr[FIELDS], order=["window", "template_id"])


def test_continuous_batching_matches_alone(lloid):
    from paper_2410_16416_b300 import serve
    banks, reqs = _streams(lloid)
    per_unit = max(lloid.plan(b, precision="bf16", refine_threshold=5.5, max_push_samples=4096).device_bytes
                   for b in banks)
    ctx = lloid.Context(0, hbm_budget_bytes=int(3.5 * per_unit))     # at most ~3 streams resident at once
    rep = serve.run(ctx, reqs, 4096, time_scale=10.0)
    ctx.close()
    s = rep.summary()
    assert s["buffers"] == 6 * len(reqs)
    assert rep.admitted_late >= 1 and rep.max_concurrent < len(reqs)
    assert np.isfinite(s["p99_latency_s"])
    for r, req in enumerate(reqs):
        mine = np.sort(rep.triggers[rep.trigger_stream == r][FIELDS], order=["window", "template_id"])
        alone = _alone(lloid, req, 6)
        assert len(alone) > 0
        assert np.array_equal(mine, alone), req.name
    # and the served triggers are the oracle's: every stream's buffers, filtered in FP64, give the
    # same window maxima (BF16 below the refine threshold: within 0.05; refined above it)
    for r, req in enumerate(reqs):
        d = np.concatenate([req.strain(j) for j in range(6)])
        ob = oracle.bank_from_arrays(req.bank.n_templates, req.bank.top_rate_hz, req.bank.slices)
        x = oracle.lloid_snr(ob, d)
        lat = lloid.plan(req.bank, max_push_samples=4096, **req.unit_kwargs).latency_samples
        mine = rep.triggers[rep.trigger_stream == r]
        assert check_triggers(mine, x, 4096, 3.0, d.shape[0] - lat, 0.05, absolute=True) == len(mine) > 0


def test_create_like_shares_the_bank(lloid):
    """A unit made with svdbank_create_like filters exactly like one made from the bank."""
    banks, reqs = _streams(lloid, n_banks=1, n_buf=4)
    ctx = lloid.Context(0)
    a = ctx.create_unit(banks[0], detector=0, max_push_samples=4096, **reqs[0].unit_kwargs)
    b = ctx.create_like(a, detector=1)
    assert b.info().device_bytes == a.info().device_bytes
    for j in range(4):
        ctx.push_group([a, b], [reqs[0].strain(j), reqs[1].strain(j)], [j * 4096] * 2, False)
    ctx.sync()
    tr = ctx.pop_triggers()
    a.destroy()                                   # b keeps the shared bank alive
    b.push(reqs[1].strain(4), 4 * 4096)
    ctx.sync()
    ctx.close()
    got = np.sort(tr[tr["unit"] == 1][FIELDS], order=["window", "template_id"])
    ref = _alone(lloid, reqs[1], 4)
    assert np.array_equal(got, ref)
