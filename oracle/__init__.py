"""FP64 CPU oracle for the LLOID multirate SVD matched filter and its trigger generator.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the filtering stage of Sec. II.A (with the readings listed in
each module's docstring).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the CUDA library never does, and
the two share no code.  Inputs come from the separate ``synth`` module.

Pins (tests/test_oracle_pins.py) tie it to things other than itself: brute
force sums, SVD invariants (orthonormality, Eckart-Young), the reduction of
the multirate path to the direct correlation for one untruncated full-rate
slice, resampler closed forms, the noise-free injection recovering its
amplitude and phase, white-noise statistics (E|rho|^2 = 2), tabulated values
of I0, window-max brute force, shift invariance, and for the sub-sample peak
the exact parabola of numpy.polyfit and a fractional-delay injection; for the
conditioning (whitening and gating, ``oracle.condition``) the flat-PSD special
case, the running average against numpy's mean, a tone's closed-form
periodogram, scale invariance, white and AR(1) noise statistics, and a
hand-worked gate.
"""
from .resample import bessel_i0, decimate, halfband, kaiser, upsample
from .coinc import coincidences
from . import condition
from .svdbank import OracleBank, OracleSlice, bank_from_arrays, build_bank, slice_filters, truncated_svd
from .lloid import (autocorrelation, basis_outputs, causal_correlate, complex_snr, decimation_cascade, direct_snr,
                    lloid_levels, lloid_snr, mix_and_sum, subsample_peak, triggers, window_maxima, xi2)
