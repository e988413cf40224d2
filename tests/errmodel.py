"""Per-bin bounds for spot checks of a transform against exact FP64 values.

The transform tolerances are relative L2 norms over the whole field:
tau = 5e-6 (FP32), 1e-5 (split-BF16 tensor-core form), 3e-3 (FP16 form).  A
spot check compares single bins (or single real points), so it needs a bound
per bin.  Error model (rounding errors independent and zero-mean, unit
roundoff u of the arithmetic the transform runs in):

* Spread part.  A rounding made before the last stages is carried through
  the rest of the transform, whose stages are unitary up to a scale, so its
  energy is shared out over all outputs.  If the whole field meets its
  tolerance, ||dX|| <= tau ||X||, the bins' errors have an rms of at most
  tau * rms(X), rms(X) = sqrt(mean |X|^2).  Taking each sampled bin's error
  as a complex Gaussian of that size, the largest of n sampled bins exceeds
  z tau rms(X) with probability n exp(-z^2): z = 4.5 gives under 2e-7 for
  n <= 100 bins.  With tau = 5e-6 this is the 2e-5 * rms(X) scaling of a
  spot bin in FP32 with z = 4 (the first form of these tests), widened to
  z = 4.5.
* Local part.  The roundings of the last stages that form bin k land on bin
  k alone: a relative error of a few u, |dX[k]| ~ c u |X[k]|.  In the spread
  part it is invisible, but on a dominant bin (a spectrum-shaped field has
  bins 100 to 700 times its rms) it is the larger part: at 1024^3 a few u
  times |X[k]| = 700 rms(X) is ~1e-4 rms(X), well above 2e-5 rms(X).  The
  bound takes c = 8: the complex multiply-add chains of the last two radix
  stages (each output of a radix-R stage is R products summed, rounding at
  each step; the twiddle tables add one more rounding per product).

bound_k = 4.5 tau rms(X) + 8 u |X[k]|.
"""
from __future__ import annotations

import numpy as np

# unit roundoff of the arithmetic: FP32; split-BF16 (hi + lo keep 16
# significant bits, and the dropped lo*lo product is 2^-18 relative); FP16
U = {0: 2.0 ** -24, 1: 2.0 ** -17, 2: 2.0 ** -11}
# rel-L2 tolerance per direction
TAU = {0: 5e-6, 1: 1e-5, 2: 3e-3}
Z_SPREAD = 4.5
C_LOCAL = 8.0


def spot_bound(ref, rms, dtype=0):
    """Allowed |got - ref| per spot value: Z_SPREAD tau rms + C_LOCAL u |ref|."""
    return Z_SPREAD * TAU[dtype] * rms + C_LOCAL * U[dtype] * np.abs(np.asarray(ref))


def spot_report(got, ref, rms, dtype=0):
    """The two parts of the error in units of the model: the largest error
    over the bound, and the largest error in units of tau * rms (the spread
    scale) -- the numbers a failing assertion prints."""
    err = np.abs(np.asarray(got) - np.asarray(ref))
    b = spot_bound(ref, rms, dtype)
    return {"max_err_over_bound": float(np.max(err / b)),
            "max_err_over_tau_rms": float(np.max(err) / (TAU[dtype] * rms))}
