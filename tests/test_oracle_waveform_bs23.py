"""Pins of the oracle's waveform and BS23 integrator against closed forms (no GPU)."""
import math

import numpy as np
import pytest

from oracle.bs23 import ACCEPT, BS23, LogEntry
from oracle.waveform import Waveform


def test_piecewise_linear_values_and_slopes():
    w = Waveform((0.0, 0.5, 1.0), (0.0, 0.25, 0.25))
    assert w.he(0.25) == pytest.approx(0.125, abs=0)
    assert w.hedot(0.25) == 0.5
    assert w.hedot(0.75) == 0.0
    assert w.he(2.0) == 0.25 and w.hedot(2.0) == 0.0          # held after the last knot
    assert w.he(-1.0) == 0.0 and w.hedot(-1.0) == 0.0         # held before the first knot
    assert w.segment(0.5) == 1                                # right-continuous
    assert w.hedot(0.5, seg=0) == 0.5                         # left slope on request
    assert w.next_knot(0.2) == 0.5 and w.next_knot(0.5) == 1.0 and w.next_knot(1.0) == math.inf


def test_sinusoid():
    w = Waveform(sin_amp=0.8, sin_period=1.0)
    assert w.he(0.25) == pytest.approx(0.8, rel=1e-15)
    assert w.hedot(0.0) == pytest.approx(0.8 * 2 * math.pi, rel=1e-15)
    assert w.next_knot(0.3) == math.inf


def _fixed_steps(rhs, y0, h, n):
    """Drive the oracle integrator with forced, always-accepted steps of size h."""
    s = BS23(rhs, Waveform((0.0,), (0.0,)), rtol=1.0, atol=1.0)
    s.start(0.0, np.atleast_1d(np.asarray(y0, dtype=float)), 1.0)
    t = 0.0
    for i in range(n):
        s.replay([LogEntry(t, h, t + h, ACCEPT, (0 if i == 0 else -1, 0, 0, 0), 0.0)])
        t = s.t
    return s


def _plain(f):
    return lambda t, y, seg, force: (f(t, y), 1, 0)


def test_stability_polynomial_one_step():
    # any 3-stage explicit RK method of order 3 has R(z) = 1 + z + z^2/2 + z^3/6
    for lam, h in [(-1.0, 0.1), (-3.0, 0.7), (2.0, 0.25)]:
        s = _fixed_steps(_plain(lambda t, y: lam * y), 1.0, h, 1)
        z = lam * h
        assert s.y[0] == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6, rel=1e-14)


def test_polynomial_exactness_and_error_estimate():
    h = 0.3
    # third-order solution exact for y = t^3
    s = _fixed_steps(_plain(lambda t, y: np.array([3 * t * t])), 0.0, h, 1)
    assert s.y[0] == pytest.approx(h ** 3, rel=1e-14)
    # E = y_3rd - y_2nd: zero on y = t^2, equal to -h^3/8 on y = t^3 (hand-derived from b, b_hat)
    s2 = BS23(_plain(lambda t, y: np.array([2 * t])), Waveform((0.0,), (0.0,)), rtol=0, atol=1.0)
    s2.start(0.0, np.array([0.0]), 1.0)
    s2.h = h
    s2.attempt(10.0)
    assert abs(s2.log[-1].err) < 1e-15
    s3 = BS23(_plain(lambda t, y: np.array([3 * t * t])), Waveform((0.0,), (0.0,)), rtol=0, atol=1.0)
    s3.start(0.0, np.array([0.0]), 1.0)
    s3.h = h
    s3.attempt(10.0)
    assert s3.log[-1].err == pytest.approx(h ** 3 / 8, rel=1e-12)


def test_third_order_global_convergence():
    errs = []
    for n in (20, 40, 80):
        s = _fixed_steps(_plain(lambda t, y: np.array([math.cos(t)])), 0.0, 2.0 / n, n)
        errs.append(abs(s.y[0] - math.sin(2.0)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 < r < 3.2 for r in rates), rates


def test_adaptive_controller_and_knot_clipping():
    w = Waveform((0.0, 0.5, 2.0), (0.0, 1.0, 1.0))

    def rhs(t, y, seg, force):
        return -y + w.hedot(t, seg), 1, 0          # y' = -y + h_e'(t)

    s = BS23(rhs, w, rtol=1e-6, atol=1e-6)
    s.start(0.0, np.array([0.0]), 2.0)
    s.advance(1.0)
    s.advance(2.0)
    # exact: y = 2(1 - e^-t) on [0, .5], then decays with y' = -y
    y_half = 2 * (1 - math.exp(-0.5))
    assert s.y[0] == pytest.approx(y_half * math.exp(-1.5), abs=2e-5)
    ends = [e.t_new for e in s.log if e.outcome == ACCEPT]
    assert 0.5 in ends and 1.0 in ends and ends[-1] == 2.0
    i = ends.index(0.5)
    nxt = [e for e in s.log if e.outcome == ACCEPT][i + 1]
    assert nxt.iters[0] >= 0                        # k1 recomputed after the slope jump
    assert all(e.err <= 1.0 for e in s.log if e.outcome == ACCEPT)


def test_failed_first_stage_is_retried_with_half_step():
    # a right-hand side whose outside iteration fails on its first two calls: the attempts are
    # rejected (h halved) and k1 is evaluated again each time, as for any failed stage
    calls = {"n": 0}

    def rhs(t, y, seg, force):
        calls["n"] += 1
        return -y, 1, (3 if calls["n"] <= 2 else 0)

    s = BS23(rhs, Waveform((0.0,), (0.0,)), rtol=1e-6, atol=1e-6, h0=0.1)
    s.start(0.0, np.array([1.0]), 1.0)
    s.advance(0.3)
    assert [e.outcome for e in s.log[:2]] == [2, 2]
    assert s.log[0].iters[0] >= 0 and s.log[1].iters[0] >= 0 and s.log[2].iters[0] >= 0
    assert s.log[1].h == pytest.approx(0.05) and s.log[2].h == pytest.approx(0.025)
    assert s.y[0] == pytest.approx(math.exp(-0.3), rel=1e-5)


def test_sliver_step_before_a_knot_does_not_collapse_the_step_size():
    # an output time one ulp before a knot (numpy's linspace gives 0.49999999999999994 for 0.5)
    # leaves a step of 5.6e-17 to the knot; the step after it starts again from the proposal
    # the sliver replaced instead of from 5 x 5.6e-17 (which is below h_min)
    w = Waveform((0.0, 0.5, 1.0), (0.0, 0.25, 0.25))

    def rhs(t, y, seg, force):
        return -y + w.hedot(t, seg), 1, 0

    s = BS23(rhs, w, rtol=1e-6, atol=1e-6)
    s.start(0.0, np.array([0.0]), 1.0)
    t_out = np.linspace(0.05, 1.0, 20)
    assert t_out[9] < 0.5 and 0.5 - t_out[9] < 1e-15
    for t in t_out:
        assert s.advance(float(t)) == 0
    assert s.t == 1.0
    sliver = [e for e in s.log if e.outcome == ACCEPT and e.h < 1e-12]
    assert len(sliver) == 1 and sliver[0].t_new == 0.5
    after = s.log[s.log.index(sliver[0]) + 1]
    assert after.h > 1e-4
