"""Per-bin bounds for spot checks of a transform against exact FP64 values.

The transform tolerances are relative L2 norms over the whole field:
tau = 5e-6 (FP32), 1e-5 (split-BF16 tensor-core form), 3e-3 (FP16 form).  A
spot check compares single bins (or single real points), so it needs a bound
per bin.  Error model (rounding errors independent and zero-mean, unit
roundoff u of the arithmetic the transform runs in):

* Spread part.  A rounding made in an early stage is carried through the
  rest of the transform, whose stages are unitary up to a scale, so its
  energy is shared out over many outputs.  If the whole field meets its
  tolerance, ||dX|| <= tau ||X||, the bins' errors have an rms of at most
  tau * rms(X), rms(X) = sqrt(mean |X|^2).  Taking each sampled bin's error
  as a complex Gaussian of that size, the largest of n sampled bins exceeds
  z tau rms(X) with probability n exp(-z^2): z = 4.5 gives under 2e-7 for
  n <= 100 bins.  With tau = 5e-6 this is the 2e-5 * rms(X) scaling of a
  spot bin in FP32 with z = 4 (the first form of these tests), widened to
  z = 4.5.
* Line part.  A 3D transform is three passes of 1D transforms along the
  axes; the roundings of a pass stay on the line they were made on (the
  line's own transform spreads them over that line only).  A bin on a line
  that carries much more energy than the field's average (a spectrum-shaped
  field has its energy in a few low-k lines) therefore sees errors of a few
  u times the line's rms, sqrt(log2 n) of them added up over a line's
  stages: C_LINE u sqrt(log2 n) (l0 + l1 + l2), l_a the rms of |X| over the
  axis-a line through the bin.
* Local part.  The roundings of the last stages that form bin k land on bin
  k alone: a relative error of a few u, |dX[k]| ~ c u |X[k]|.  On a dominant
  bin (100 to 2000 times rms(X) on the spectrum-shaped fields) this is the
  largest part; C_LOCAL = 8 covers the complex multiply-add chains of the last
  two radix stages.

bound_k = 4.5 tau rms(X) + C_LINE u sqrt(log2 n) (l0 + l1 + l2) + C_LOCAL u |X[k]|,
C_LINE = C_LOCAL = 8.

Measured on every bin of the spectrum-shaped fields at 512^3 and 1024^3
against the exact spectrum: the FP32 and FP16 forms stay within it (largest
error 0.46 / 0.75 of the bound in FP32, 0.63 / 0.98 in FP16).  Without the
line part 45 of 67 million bins (512^3) and 1544 of 538 million (1024^3)
exceeded it in FP32; with the spread part alone (the first form, 2e-5 rms),
581 and 3373.  The split-BF16 form does not fit this shape: 0.03-0.05 % of
the bins of those fields exceed the bound (largest 4.2 times), because the
error of one split-BF16 radix-16 contraction scales with the sum of its
inputs' magnitudes, not with a line's rms; its checks rest on the whole-field
rel-L2 (1024^3, against the oracle), and its spot bins are taken only on the
white uniform field, where no bin or line dominates.
"""
from __future__ import annotations

import math

import numpy as np

# unit roundoff of the arithmetic: FP32; split-BF16 (hi + lo keep 16
# significant bits, and the dropped lo*lo product is 2^-18 relative); FP16
U = {0: 2.0 ** -24, 1: 2.0 ** -17, 2: 2.0 ** -11}
# rel-L2 tolerance per direction
TAU = {0: 5e-6, 1: 1e-5, 2: 3e-3}
Z_SPREAD = 4.5
C_LINE = 8.0
C_LOCAL = 8.0


def spot_bound(ref, rms, dtype=0, lines=0.0, n=2):
    """Allowed |got - ref| per spot value.  lines: l0 + l1 + l2 per value
    (0 where the line part is not used, e.g. a white field); n: the longest
    axis (the line part's sqrt(log2 n))."""
    return (Z_SPREAD * TAU[dtype] * rms + C_LINE * U[dtype] * math.sqrt(math.log2(max(n, 2))) * np.asarray(lines)
            + C_LOCAL * U[dtype] * np.abs(np.asarray(ref)))


def spot_report(got, ref, rms, dtype=0, lines=0.0, n=2):
    """The largest error over the bound, and the largest error in units of
    tau * rms (the spread scale): the numbers a failing assertion prints."""
    err = np.abs(np.asarray(got) - np.asarray(ref))
    b = spot_bound(ref, rms, dtype, lines, n)
    return {"max_err_over_bound": float(np.max(err / b)),
            "max_err_over_tau_rms": float(np.max(err) / (TAU[dtype] * rms))}


def line_rms(X, ks):
    """l0 + l1 + l2 of each index k = (k0, k1, k2) of a 3D array (numpy, or a
    torch tensor on any device): the rms of |X| over the three axis lines
    through it."""
    def rms(v):
        v = v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)
        return math.sqrt(float(np.mean(np.abs(v.astype(np.complex128)) ** 2)))
    return np.array([rms(X[:, k1, k2]) + rms(X[k0, :, k2]) + rms(X[k0, k1, :]) for k0, k1, k2 in ks])
