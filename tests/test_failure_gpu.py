"""Failure detection on the device without a fault: a bounded wait that runs out.

sb_ctx_test_wait bounds the basis-FIR kernel's waits by 1 ms and makes the
first tile's producer skip one K chunk's load: nothing is ever issued for it,
so the consumer's wait expires.  The kernel must then let its issued copies
land, let its issued MMAs finish, free its TMEM and return; the host reports
SB_ETIMEOUT from triggers_pop, and a fresh context completes a normal push that
matches the oracle.  Nothing faults, traps or hangs.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from helpers import push_and_collect, rho_abs_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lloid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as m
    return m


def test_bounded_wait_expires_and_the_next_context_works(lloid):
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(spec.n_templates, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 21, 0, 0)
    bank = oracle.build_bank(h, spec.top_rate_hz, spec.slices)
    d = synth.white_noise(12 * 2048, 21, 0, 0)
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="bf16", threshold=6.0, max_push_samples=4096)
    u.push(d[:4096], 0)
    ctx.sync()
    ctx.pop_triggers()                                           # a normal push first
    ctx.test_wait(1_000_000, 1)                                  # 1 ms bound; chunk 1 of tile 0 never loaded
    t = time.perf_counter()
    u.push(d[4096:8192], 4096)
    ctx.sync()
    elapsed = time.perf_counter() - t
    with pytest.raises(lloid.LloidError) as e:
        ctx.pop_triggers()
    assert e.value.code == lloid.SB_ETIMEOUT
    assert b"site 3" in lloid.lib.sb_last_error()                # the MMA issuer's wait on the skipped chunk
    assert elapsed < 1.0, elapsed                                # the 1 ms bound, not the 2 s default
    ctx.test_wait(0, -1)
    ctx.close()
    # the device stays usable: a fresh context filters normally
    ctx = lloid.Context(0)
    u = ctx.create_unit(bank, precision="bf16", threshold=6.0, max_push_samples=4096, keep_snr=True)
    (xg,) = push_and_collect(ctx, [u], [d], [4096] * 3)
    ctx.sync()
    ctx.pop_triggers()
    ctx.close()
    x = oracle.lloid_snr(bank, d)
    assert rho_abs_error(xg, x) <= 0.05
