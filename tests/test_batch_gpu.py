"""Grouped batch parity at full size: three uneven bins of the batch workload in one grouped push.

The bins come from the batch workload's generator (shape-only banks:
M logU[200, 2000], 3-8 slices at 4096/2^s Hz, spans 2-120 s, L logU[50, 600]):
bin 48 (1984 templates, 4 slices, L up to 544, 44 s), bin 149 (1483 templates,
8 slices, 46 s) and bin 192 (1674 templates, 6 slices, 119 s).  They are pushed
together (every stage one launch over the three units) for 16 s of their own
noise, in BF16; every real filter's SNR on every sample and every window
maximum are compared with the oracle (FP64, basis outputs shared, mixing and
up-sampling in row chunks).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_triggers_maxima

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BINS = (48, 149, 192)
F0 = 4096
SECONDS = 16
PUSH = 8 * F0
SIZES = [PUSH, PUSH, 4 * F0]             # 20 s pushed: final for n < 20 s - latency (about 1 s here)
TOL_HALF = 0.05
ROWS = 200


@pytest.fixture(scope="module")
def lloid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_16416_b300 as m
    return m


def test_grouped_batch_bins_full_size(lloid):
    banks = [synth.shape_only_bank(b) for b in BINS]
    n = sum(SIZES)
    strains = [synth.white_noise(n, 60, b, 0) for b in BINS]
    ctx = lloid.Context(0)
    units = [ctx.create_unit(bk, precision="bf16", threshold=0.0, max_push_samples=PUSH, keep_snr=True)
             for bk in banks]
    xs = [[] for _ in units]
    t = 0
    for sz in SIZES:
        ctx.push_group(units, [s[t:t + sz] for s in strains], [t] * len(units), False)
        for i, u in enumerate(units):
            _, x = u.snr()
            if x.shape[1]:
                xs[i].append(x)
        t += sz
    ctx.sync()
    trig = ctx.pop_triggers()
    ids = [u.info().unit for u in units]
    ctx.close()
    nv = SECONDS * F0
    for i, (bk, d) in enumerate(zip(banks, strains)):
        xg = np.concatenate(xs[i], axis=1)[:, :nv]
        assert xg.shape[1] == nv
        ob = oracle.bank_from_arrays(bk.n_templates, bk.top_rate_hz, bk.slices)
        g = oracle.halfband()
        o = oracle.basis_outputs(ob, oracle.decimation_cascade(d, ob.k_max, g))
        M = bk.n_templates
        n_star = np.empty((SECONDS, M), np.int64)
        amax = np.empty((SECONDS, M))
        ph = np.empty((SECONDS, M))
        x32 = np.empty((2 * M, nv), np.float32)
        worst = 0.0
        for r0 in range(0, 2 * M, ROWS):
            rows = np.arange(r0, min(2 * M, r0 + ROWS))
            x = oracle.mix_and_sum(ob, o, d.shape[0], g, rows)[0][:, :nv]
            _, ns, am, pp = oracle.window_maxima(x, F0, nv)
            c0 = r0 // 2
            n_star[:, c0:c0 + ns.shape[1]], amax[:, c0:c0 + ns.shape[1]], ph[:, c0:c0 + ns.shape[1]] = ns, am, pp
            gg = xg[rows].astype(np.float64)
            worst = max(worst, float(np.abs((gg[0::2] + 1j * gg[1::2]) - (x[0::2] + 1j * x[1::2])).max()))
            x32[rows] = x
        errs = []
        rho_abs = lambda ii, nn: float(np.hypot(np.float64(x32[2 * ii, nn]), np.float64(x32[2 * ii + 1, nn])))
        mine = trig[(trig["unit"] == ids[i]) & (trig["window"] < SECONDS)]
        m = check_triggers_maxima(mine, (np.arange(SECONDS), n_star, amax, ph), rho_abs, M, 0.0, TOL_HALF,
                                  absolute=True, errors=errs)
        print(f"batch bin {BINS[i]} ({M} templates, L={[s.basis.shape[0] for s in bk.slices]}): max |rho| error "
              f"{worst:.4f} on every sample, {max(errs):.4f} over {m} window maxima")
        assert worst <= TOL_HALF
        assert m == M * SECONDS
