"""The benchmark's work model and warm-up rule (host logic of bench.py, no GPU)."""
import math

import bench
import synth
import paper_2410_16416_b300 as lloid


def _bank():
    spec = synth.SMALL_BIN
    h, _ = synth.template_bank(8, spec.mc_lo, spec.mc_hi, spec.top_rate_hz, spec.duration_s, 1, 0, 0)
    return lloid.decompose(h, spec.top_rate_hz, spec.slices)


def test_work_model_counts_the_methods_flops():
    bank = _bank()
    units, secs = 2, 4.0
    M2 = 2 * bank.n_templates
    f0 = bank.top_rate_hz
    k_of = lambda s: int(round(math.log2(f0 / s.rate_hz)))
    kmax = max(k_of(s) for s in bank.slices)
    fir = sum(2.0 * s.basis.shape[0] * s.basis.shape[1] * secs * s.rate_hz for s in bank.slices)
    mix = sum(2.0 * M2 * s.basis.shape[0] * secs * s.rate_hz for s in bank.slices)
    interp = sum(32.0 * M2 * secs * f0 / 2 ** k for k in range(kmax))
    for precision in ("bf16", "fp8"):
        flops, bytes_, inter = bench.algorithmic_model(bank, units, secs, precision)
        assert math.isclose(flops["fir"], units * fir, rel_tol=1e-12)
        assert math.isclose(flops["mix"], units * (mix + interp), rel_tol=1e-12)
        # the stored levels' SNR, written once and read once in FP16, is the design's intermediate
        y = sum(2 * 2.0 * M2 * secs * f0 / 2 ** k for k in range(1, kmax + 1))
        assert math.isclose(inter, units * y, rel_tol=1e-12)
        assert bytes_["mix"] > 0 and flops["upsample"] == 0
    flops, _, inter = bench.algorithmic_model(bank, units, secs, "fp32")
    assert math.isclose(flops["mix"], units * mix, rel_tol=1e-12)
    assert math.isclose(flops["upsample"], units * interp, rel_tol=1e-12)
    assert inter == 0


def test_warm_up_covers_the_graph_ring():
    assert bench.warm_pushes(3, True) == bench.GRAPH_RING
    assert bench.warm_pushes(3, False) == 3
    assert bench.warm_pushes(bench.GRAPH_RING + 4, True) == bench.GRAPH_RING + 4
