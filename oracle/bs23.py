"""Bogacki-Shampine 3(2) integrator for the method of lines (TEST INFRASTRUCTURE ONLY).

The paper integrates g_dot = f(g, t) (and h_dot = f(t, h)) with Matlab's ode23 (Section 2.2),
i.e. the Bogacki-Shampine 3(2) pair (Bogacki and Shampine, Appl. Math. Lett. 2 (1989) 321),
and handles a failed outside iteration by letting the step control shrink the step
(Section 2.2).  The oracle implements the published pair, not Matlab's internals:

  c = (0, 1/2, 3/4, 1);  a21 = 1/2;  a32 = 3/4 (a31 = 0);
  y_{n+1} = y_n + h (2/9 k1 + 1/3 k2 + 4/9 k3)            (third order, also the 4th stage)
  k4 = f(t_n + h, y_{n+1})                                 (first same as last)
  E = h (-5/72 k1 + 1/12 k2 + 1/9 k3 - 1/8 k4)             (3rd minus embedded 2nd order:
                                                            b_hat = (7/24, 1/4, 1/3, 1/8))
  err = max_i |E_i| / (atol + rtol max(|y_n,i|, |y_{n+1},i|)),  accept if err <= 1.

Step control (a standard choice; the paper states none):
  accept: h <- h min(5, max(0.2, 0.9 err^(-1/3))), capped at 1x right after a rejection; after
          a step that was shortened to end on a knot or output time, h <- h_prop min(1, fac)
          with h_prop the proposal before the shortening (a step shortened to a sliver, e.g. an
          output time one ulp before a knot, must not collapse the next step)
  reject: h <- h max(0.2, 0.9 err^(-1/3));  non-converged stage (k1 included): h <- h/2, and
  a non-converged k1 is evaluated again on the next attempt (its warm start has advanced)
  h < h_min stops with STEP_UNDERFLOW.
Steps are clipped so that they end exactly on the next output time or h_e knot (a step within
10% of reaching it is stretched to it).  A step that ends on a knot discards k4 as the next k1,
because h_e_dot jumps there; stage derivatives of h_e use the segment the step lies in.

Before every attempt `on_attempt()` and after an accepted step `on_accept()` are called (the
film problem starts an attempt from the accepted step's free-space h_dot).  Every attempted step is logged; `replay`
re-executes a logged sequence with the same step sizes, decisions and per-stage iteration
counts (lock-step comparison with another solver).
Pinned by tests/test_oracle_bs23.py: the stability polynomial 1+z+z^2/2+z^3/6 of one step on
y' = lambda y, exactness on polynomial solutions (degree 3 for y_{n+1}, 2 for the embedded
solution), third-order global convergence on y' = cos t, and the controller on a decaying ODE.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

OK, NOCONV, STEP_UNDERFLOW = 0, 3, 5
REJECT_ERR, ACCEPT, REJECT_NOCONV = 0, 1, 2


@dataclasses.dataclass
class LogEntry:
    t: float
    h: float
    t_new: float
    outcome: int          # REJECT_ERR / ACCEPT / REJECT_NOCONV
    iters: tuple          # iterations of stages k1..k4, -1 when not evaluated
    err: float


class BS23:
    """Adaptive BS23 integrator around a right-hand side rhs(t, y, seg, force_iters)."""

    def __init__(self, rhs, waveform, *, rtol=1e-6, atol=1e-6, h0=0.0, h_min=1e-12, on_accept=None,
                 on_attempt=None):
        self.rhs = rhs
        self.on_accept = on_accept            # called after every accepted step
        self.on_attempt = on_attempt          # called before the first evaluation of every attempt
        self.wf = waveform
        self.rtol, self.atol, self.h0, self.h_min = rtol, atol, h0, h_min
        self.log: list[LogEntry] = []
        self.n_rhs = 0
        self.t = None
        self.y = None
        self.h = None
        self.k1 = None
        self.failed = False

    def start(self, t0: float, y0: np.ndarray, t_end: float):
        self.t = float(t0)
        self.y = np.array(y0, dtype=np.float64)
        self.h = self.h0 if self.h0 > 0 else min(1e-3, 0.01 * (t_end - t0))
        self.k1 = None
        self.failed = False

    def _f(self, t, y, seg, force=None):
        self.n_rhs += 1
        return self.rhs(t, y, seg, force)

    def attempt(self, t_target: float, forced: LogEntry | None = None) -> int:
        """One step attempt towards t_target.  Returns its outcome."""
        if self.on_attempt is not None:
            self.on_attempt()
        t, y = self.t, self.y
        t_lim = min(t_target, self.wf.next_knot(t))
        h_prop = self.h
        if forced is None:
            h = self.h
            clipped = t + 1.1 * h >= t_lim
            if clipped:
                h = t_lim - t
        else:
            h = forced.h
            clipped = forced.outcome == ACCEPT and forced.t_new == t_lim
        seg = self.wf.segment(t)
        it = [-1, -1, -1, -1]
        fi = (lambda s: None) if forced is None else (lambda s: forced.iters[s])

        st = OK
        if self.k1 is None or (forced is not None and forced.iters[0] >= 0):
            # a non-converged k1 rejects the attempt like any stage (Section 2.2: the step
            # control reacts, and the warm-started iteration continues on the next attempt)
            k1v, it[0], st = self._f(t, y, seg, fi(0))
            self.k1 = k1v if st == OK else None
        k1 = self.k1
        outcome = ACCEPT
        if st == OK:
            k2, it[1], st = self._f(t + 0.5 * h, y + 0.5 * h * k1, seg, fi(1))
        if st == OK:
            k3, it[2], st = self._f(t + 0.75 * h, y + 0.75 * h * k2, seg, fi(2))
        if st == OK:
            ynew = y + h * (2.0 / 9.0 * k1 + 1.0 / 3.0 * k2 + 4.0 / 9.0 * k3)
            t_new = t_lim if clipped else t + h
            k4, it[3], st = self._f(t_new, ynew, seg, fi(3))
        err = math.inf
        if st != OK:
            outcome = REJECT_NOCONV
        else:
            E = h * (-5.0 / 72.0 * k1 + 1.0 / 12.0 * k2 + 1.0 / 9.0 * k3 - 1.0 / 8.0 * k4)
            scale = self.atol + self.rtol * np.maximum(np.abs(y), np.abs(ynew))
            err = float(np.max(np.abs(E) / scale))
            outcome = ACCEPT if err <= 1.0 else REJECT_ERR
        if forced is not None:
            outcome = forced.outcome

        if outcome == ACCEPT:
            if self.on_accept is not None:
                self.on_accept()
            self.t, self.y = t_new, ynew
            knot_hit = clipped and t_lim == self.wf.next_knot(t)
            self.k1 = None if knot_hit else k4
            fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** (-1.0 / 3.0)))
            if self.failed:
                fac = min(fac, 1.0)
            # a step shortened to end on a knot or output time says nothing about longer steps:
            # the next one starts from the proposal it replaced (never above it)
            self.h = h_prop * min(fac, 1.0) if (clipped and h < h_prop) else h * fac
            self.failed = False
        elif outcome == REJECT_ERR:
            self.h = h * max(0.2, 0.9 * err ** (-1.0 / 3.0))
            self.failed = True
        else:
            self.h = 0.5 * h
            self.failed = True
        self.log.append(LogEntry(t, h, self.t if outcome == ACCEPT else t, outcome, tuple(it), err))
        return outcome

    def advance(self, t_target: float, max_attempts: int = 10 ** 7) -> int:
        n = 0
        while self.t < t_target:
            self.attempt(t_target)
            n += 1
            if self.h < self.h_min:
                return STEP_UNDERFLOW
            if n >= max_attempts:
                raise RuntimeError("too many step attempts")
        return OK

    def replay(self, entries) -> None:
        """Re-execute logged attempts with their step sizes, decisions and iteration counts."""
        for e in entries:
            assert abs(e.t - self.t) <= 1e-12 * max(1.0, abs(self.t)), (e.t, self.t)
            self.attempt(e.t_new if e.outcome == ACCEPT else math.inf, forced=e)
