"""Uniform applied field h_e(t) for the oracle (TEST INFRASTRUCTURE ONLY).

The paper's thin-film examples use h_e = t (Section 2.3) and the bulk examples
h_e = (0, 0, t) or (0, 0, A sin(w t)) (Section 3.2).  Two forms are supported:
  * piecewise linear through knots (t_k, v_k), held constant outside [t_0, t_K];
  * a sinusoid amp * sin(2 pi t / period).

The time derivative of the piecewise-linear form is the slope of a segment.  A stage of an
integrator step that ends exactly on a knot must use the slope of the segment the step lies
in, so `hedot` takes an optional segment index; without it the segment is the one with
t_k <= t < t_{k+1} (right-continuous).
Pinned by tests/test_oracle_waveform.py (values and slopes of hand-made knot sets).
"""
from __future__ import annotations

import bisect
import math


class Waveform:
    def __init__(self, knots_t=None, knots_v=None, sin_amp=0.0, sin_period=1.0):
        if knots_t is not None and len(knots_t) > 0:
            assert len(knots_t) == len(knots_v)
            assert all(b > a for a, b in zip(knots_t, knots_t[1:])), "knots must increase"
            self.kt = [float(t) for t in knots_t]
            self.kv = [float(v) for v in knots_v]
            self.sin = None
        else:
            self.kt = []
            self.kv = []
            self.sin = (float(sin_amp), float(sin_period))

    # segment k covers [kt[k], kt[k+1]); -1 is before the first knot, K-1 after the last
    def segment(self, t: float) -> int:
        if self.sin is not None:
            return 0
        return bisect.bisect_right(self.kt, t) - 1

    def he(self, t: float) -> float:
        if self.sin is not None:
            a, p = self.sin
            return a * math.sin(2.0 * math.pi * t / p)
        k = self.segment(t)
        if k < 0:
            return self.kv[0]
        if k >= len(self.kt) - 1:
            return self.kv[-1]
        s = (t - self.kt[k]) / (self.kt[k + 1] - self.kt[k])
        return self.kv[k] + s * (self.kv[k + 1] - self.kv[k])

    def hedot(self, t: float, seg: int | None = None) -> float:
        if self.sin is not None:
            a, p = self.sin
            w = 2.0 * math.pi / p
            return a * w * math.cos(w * t)
        k = self.segment(t) if seg is None else seg
        if k < 0 or k >= len(self.kt) - 1:
            return 0.0
        return (self.kv[k + 1] - self.kv[k]) / (self.kt[k + 1] - self.kt[k])

    def next_knot(self, t: float) -> float:
        """Smallest knot strictly greater than t (inf if none)."""
        if self.sin is not None:
            return math.inf
        i = bisect.bisect_right(self.kt, t)
        return self.kt[i] if i < len(self.kt) else math.inf
