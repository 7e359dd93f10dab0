"""Discrete adjoint of a thin-film solve (TEST INFRASTRUCTURE ONLY).

The paper has no adjoint.  This oracle differentiates, exactly, the discrete map that the
integrator of Section 2.2 evaluates once its decisions are frozen, so that the map is a smooth
function of its inputs:

  * the time steps (t_n, h_n) of the Bogacki-Shampine 3(2) integrator are given, all accepted,
    each inside one waveform segment;
  * every right-hand side runs a given number of outside iterations (Eqs. 10-12): the counts
    the stop test of Section 2.3 chose in a forward run, or any counts the caller fixes;
  * the outside iteration is warm-started as the integrator runs it: every call starts from the
    free-space h_dot of the previous call (the first call from a given field, or cold from
    h_e_dot), so the iterate is carried from call to call and is differentiated as state.

Map.  y_{n+1} = y_n + h_n (2/9 k1 + 1/3 k2 + 4/9 k3),  k1 = f(y_n),  k2 = f(y_n + h_n/2 k1),
k3 = f(y_n + 3 h_n/4 k2) (k1 of step n + 1 is the integrator's k4 of step n: the same call),
with h_e_dot the slope of the step's waveform segment; loss L = 1/2 dx dy sum (h_z(T) -
target)^2,  h_z = h_e(T) + F^-1[(|k|/2) F g(T)] (end of Section 2.1); parameters: the per-cell
critical current density jc (Eq. 3, in the film) and the values v_k of the piecewise-linear
h_e(t).

Derivative pieces (reverse order of the forward):
  * every spectral operator T f = Re F^-1[M F f] has the transpose Re F^-1[conj(M) F v];
  * the shift of Eq. 10 and the centring of Eq. 11 are rank-one corrections, transposed as such;
  * the warm start enters the first shift on free space, and the last iterate leaves the call:
    their cotangents are carried backwards from call to call;
  * Eq. 3: de/dj = rho (I + (n-1) j^ j^T) in the film, rho_out I elsewhere;
    de/djc = -(n/jc) e in the film; for the elliptic law e = rho(s) A j, s^2 = j^T A j,
    A = diag(1, 1/gamma^2) (FilmProblem's gamma): de/dj = rho (A + (n-1) (A j)(A j)^T / s^2);
  * the Runge-Kutta stages in reverse, each through the right-hand side's vector-Jacobian
    product; h_e_dot -> knot values through the segment slope, h_e(T) through the interpolation
    weights.

The cold-start, fixed-count right-hand side (FilmAdjoint(problem, iters).rhs / rhs_vjp, P, P_T)
is the special case of one call that starts from h_e_dot.

Pinned by tests/test_oracle_adjoint2d.py: the forward right-hand side equals
oracle.film2d.FilmProblem.rhs with the same start and iteration count, call after call; the
transposed outside iteration passes the dot-product test <P x, v> = <x, P^T v> in all its
inputs (h_dot_in, h_e_dot, warm start) and outputs (g_dot, last iterate); the vector-Jacobian
product of f and the gradient of L agree with central finite differences of the map; mistakes
planted in copies (the warm-start coupling dropped, a transposed operator flipped) fail them.
"""
from __future__ import annotations

import numpy as np

from .film2d import FilmProblem

B = (2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0)      # Bogacki-Shampine weights of the third-order solution


class FilmAdjoint:
    """f(g; jc, h_e_dot, warm start) of a film with a fixed outside-iteration count, its
    vector-Jacobian product, and the frozen-step, frozen-count solve with its gradient.
    `iters` is the count of the cold-start single calls (rhs, rhs_vjp, P, P_T)."""

    def __init__(self, problem: FilmProblem, iters: int = 1):
        assert iters >= 1 and problem.out.any(), "the adjoint needs free space and I >= 1"
        self.p = problem
        self.I = int(iters)
        self.out = problem.out.astype(np.float64)
        self.cond = problem.conductor
        self.nout = float(problem.out.sum())
        self.N = float(problem.nx * problem.ny)

    # ---- spectral operators and their transposes ------------------------------------------
    def T(self, M, f):
        return self.p.apply(M, f)

    def Tt(self, M, v):
        return self.p.apply(np.conj(M), v)

    # ---- the outside iteration as a linear map of (h_dot_in, h_e_dot) -----------------------
    def _shift(self, hd, s):
        A = (hd.sum() - self.N * s) / self.nout                  # Eq. 10
        return hd - A * self.out

    def P_warm(self, hin, s, warm, iters):
        """The outside iteration from the warm start `warm` (free space) with exactly `iters`
        iterations: (g_dot on the conductor, last iterate h_dot)."""
        p = self.p
        hd = self._shift(np.where(p.out, warm, hin), s)          # Eq. 10
        for i in range(iters):
            u = self.T(p.K1, hd)                                 # Eq. 11
            gd = u - (u * self.out).sum() / self.nout
            if i == iters - 1:
                break
            w = self.T(p.K2, gd * self.out)                      # Eq. 12
            hd = self._shift(hd - self.out * w, s)
        return np.where(self.cond, gd, 0.0), hd

    def P_T_warm(self, v, wbar, iters):
        """Transpose of P_warm: for the cotangents v of g_dot and wbar of the last iterate (None:
        0), the cotangents (of h_dot_in on the conductor, of h_e_dot, of the warm start on free
        space)."""
        p = self.p
        gbar = np.where(self.cond, v, 0.0)
        hbar = np.zeros_like(gbar) if wbar is None else self.out * wbar
        sbar = 0.0
        for i in reversed(range(iters)):
            if i < iters - 1:
                # h_dot_{i+1} = shift(z), z = h_dot_i - out * K2 (out * g_dot_i)
                tot = (hbar * self.out).sum()
                sbar += self.N / self.nout * tot
                zbar = hbar - tot / self.nout
                hbar = zbar
                gbar = self.out * self.Tt(p.K2, -self.out * zbar)
            # g_dot_i = u_i - C(u_i), u_i = K1 h_dot_i
            ubar = gbar - self.out * gbar.sum() / self.nout
            hbar = hbar + self.Tt(p.K1, ubar)
        # h_dot_0 = shift(where(out, warm, h_dot_in))
        tot = (hbar * self.out).sum()
        sbar += self.N / self.nout * tot
        pre = hbar - tot / self.nout
        return np.where(self.p.out, 0.0, pre), sbar, self.out * pre

    def P(self, hin, s):
        """Cold start (free-space h_dot = h_e_dot) and self.I iterations."""
        return self.P_warm(hin, s, np.full_like(hin, s), self.I)[0]

    def P_T(self, v):
        """Transpose of P: (adjoint of h_dot_in, adjoint of h_e_dot)."""
        hb, sb, wb = self.P_T_warm(v, None, self.I)
        return hb, sb + wb.sum()

    # ---- the right-hand side and its vector-Jacobian product ------------------------------
    def call(self, g, jc, s, warm, iters):
        """One right-hand side as the integrator runs it: f(g; jc, h_e_dot) from the warm start
        `warm` with `iters` outside iterations.  Returns (g_dot, last iterate, tape)."""
        p = self.p
        jx, jy = self.T(p.Dy, g), -self.T(p.Dx, g)               # Eq. 2
        a = np.where(p.sc, 1.0 / (p.gamma * p.gamma), 1.0)       # A = diag(1, a)
        jabs = np.sqrt(jx * jx + a * jy * jy)                    # s = |j|_A
        rho_sc = (p.e0 / jc) * (jabs / jc) ** (p.n - 1.0)        # Eq. 3
        rho = np.where(p.sc, rho_sc, p.rho_out)
        ex, ey = rho * jx, rho * a * jy
        hin = np.where(self.cond, -(self.T(p.Dx, ey) - self.T(p.Dy, ex)), 0.0)   # Eq. 4 / 9
        gd, last = self.P_warm(hin, s, warm, iters)
        return gd, last, (jx, jy, jabs, rho, ex, ey, a)

    def call_vjp(self, tape, jc, iters, v, wbar):
        """(adjoint of g, of the jc map, of h_e_dot, of the warm start) of one call for the
        cotangents v of its g_dot and wbar of its last iterate (None: 0)."""
        p = self.p
        jx, jy, jabs, rho, ex, ey, a = tape
        hbar_in, sbar, warm_bar = self.P_T_warm(v, wbar, iters)
        rbar = np.where(self.cond, -hbar_in, 0.0)                # h_in = -raw on the conductor
        eybar = self.Tt(p.Dx, rbar)                              # raw = Dx e_y - Dy e_x
        exbar = -self.Tt(p.Dy, rbar)
        safe = np.where(jabs > 0, jabs, 1.0)
        # unit vector A j / s
        ux, uy = np.where(jabs > 0, jx / safe, 0.0), np.where(jabs > 0, a * jy / safe, 0.0)
        proj = ux * exbar + uy * eybar
        nn = np.where(p.sc, p.n - 1.0, 0.0)                      # Ohm's law elsewhere
        jxbar = rho * (exbar + nn * ux * proj)
        jybar = rho * (a * eybar + nn * uy * proj)
        jcbar = np.where(p.sc, -(p.n / jc) * (exbar * ex + eybar * ey), 0.0)
        gbar = self.Tt(p.Dy, jxbar) - self.Tt(p.Dx, jybar)       # j_x = Dy g, j_y = -Dx g
        return gbar, jcbar, sbar, warm_bar

    def rhs(self, g, jc, s):
        """Cold-start, self.I-iteration right-hand side: (g_dot, tape)."""
        gd, _, tape = self.call(g, jc, s, np.full_like(np.asarray(g, dtype=np.float64), s), self.I)
        return gd, tape

    def rhs_vjp(self, tape, jc, v):
        """(adjoint of g, of the jc map, of h_e_dot) of the cold-start right-hand side."""
        gb, cb, sb, wb = self.call_vjp(tape, jc, self.I, v, None)
        return gb, cb, sb + wb.sum()

    # ---- the frozen-step solve, the loss and its gradient ----------------------------------
    @staticmethod
    def _segment(kt, t0, t1):
        k = int(np.searchsorted(kt, t0, side="right")) - 1
        assert 0 <= k < len(kt) - 1 and t1 <= kt[k + 1] + 1e-15, "a step must lie in one segment"
        return k

    @staticmethod
    def _he(kt, kv, t):
        k = int(np.searchsorted(kt, t, side="right")) - 1
        k = min(max(k, 0), len(kt) - 2)
        w = (t - kt[k]) / (kt[k + 1] - kt[k])
        return kv[k] + w * (kv[k + 1] - kv[k]), k, w

    def _steps(self, y, warm, jc, kt, kv, steps, iters, n0, n1, keep):
        """Steps n0 .. n1-1 from (y, warm); returns (y, warm, tapes)."""
        tapes = []
        for n in range(n0, n1):
            t, h = steps[n]
            k = self._segment(kt, t, t + h)
            s = (kv[k + 1] - kv[k]) / (kt[k + 1] - kt[k])
            if warm is None:
                warm = np.full_like(y, s)                        # cold start: h_e_dot
            ks, st = [], []
            for j, (a, kprev) in enumerate(((0.0, None), (0.5, 0), (0.75, 1))):
                gs = y if kprev is None else y + a * h * ks[kprev]
                kj, warm, tp = self.call(gs, jc, s, warm, iters[3 * n + j])
                ks.append(kj)
                st.append(tp)
            if keep:
                tapes.append((h, k, tuple(st), tuple(iters[3 * n:3 * n + 3])))
            y = y + h * (B[0] * ks[0] + B[1] * ks[1] + B[2] * ks[2])
        return y, warm, tapes

    def solve(self, g0, jc, kt, kv, steps, iters, warm0=None, keep=False):
        """Advance g0 over the given (t, h) steps with the given outside-iteration counts (3 per
        step: k1, k2, k3), the warm start carried from call to call (warm0: the first call's,
        None: cold from h_e_dot); with keep, also the calls' tapes."""
        iters = list(iters)
        assert len(iters) == 3 * len(steps)
        y = np.array(g0, dtype=np.float64)
        warm = None if warm0 is None else np.array(warm0, dtype=np.float64)
        y, _, tapes = self._steps(y, warm, jc, kt, kv, steps, iters, 0, len(steps), keep)
        return (y, tapes) if keep else y

    def loss(self, g0, jc, kt, kv, steps, target, iters, warm0=None):
        T = steps[-1][0] + steps[-1][1]
        y = self.solve(g0, jc, kt, kv, steps, iters, warm0)
        hz = self._he(kt, kv, T)[0] + self.T(self.p.Kh, y)
        return 0.5 * self.p.dx * self.p.dy * float(((hz - target) ** 2).sum())

    def gradient(self, g0, jc, kt, kv, steps, target, iters, warm0=None, ckpt_every=None):
        """(L, dL/djc, dL/dv, dL/dwarm0) by the discrete adjoint of the frozen-step,
        frozen-count solve (dL/dwarm0 is None for a cold first call, whose start is h_e_dot).
        With ckpt_every = C the forward keeps the state and warm start every C steps and the
        reverse sweep recomputes each segment's tapes from them (same result, less memory)."""
        p = self.p
        kt = np.asarray(kt, dtype=np.float64)
        kv = np.asarray(kv, dtype=np.float64)
        iters = list(iters)
        N = len(steps)
        assert len(iters) == 3 * N
        C = N if not ckpt_every else min(int(ckpt_every), N)
        T = steps[-1][0] + steps[-1][1]
        y = np.array(g0, dtype=np.float64)
        warm = None if warm0 is None else np.array(warm0, dtype=np.float64)
        ckpts = []
        for n0 in range(0, N, C):
            ckpts.append((y, warm))
            y, warm, _ = self._steps(y, warm, jc, kt, kv, steps, iters, n0, min(N, n0 + C), False)
        he, kT, wT = self._he(kt, kv, T)
        res = he + self.T(p.Kh, y) - target
        dA = p.dx * p.dy
        L = 0.5 * dA * float((res * res).sum())
        jcbar = np.zeros_like(np.asarray(jc, dtype=np.float64) * np.ones_like(y))
        vbar = np.zeros_like(kv)
        vbar[kT] += (1.0 - wT) * dA * res.sum()
        vbar[kT + 1] += wT * dA * res.sum()
        lam = dA * self.Tt(p.Kh, res)
        wbar = None                                              # cotangent of the last iterate
        for si in reversed(range(len(ckpts))):
            n0 = si * C
            ys, ws = ckpts[si]
            _, _, tapes = self._steps(ys, ws, jc, kt, kv, steps, iters, n0, min(N, n0 + C), True)
            for m in reversed(range(len(tapes))):
                n = n0 + m
                h, k, (t1, t2, t3), (i1, i2, i3) = tapes[m]
                lk3 = h * B[2] * lam
                lk2 = h * B[1] * lam
                lk1 = h * B[0] * lam
                ly = lam.copy()
                sbar = 0.0
                gb, cb, sb, wbar = self.call_vjp(t3, jc, i3, lk3, wbar)   # k3 = f(y + 3h/4 k2)
                ly += gb
                lk2 += 0.75 * h * gb
                jcbar += cb
                sbar += sb
                gb, cb, sb, wbar = self.call_vjp(t2, jc, i2, lk2, wbar)   # k2 = f(y + h/2 k1)
                ly += gb
                lk1 += 0.5 * h * gb
                jcbar += cb
                sbar += sb
                gb, cb, sb, wbar = self.call_vjp(t1, jc, i1, lk1, wbar)   # k1 = f(y)
                ly += gb
                jcbar += cb
                sbar += sb
                if n == 0 and warm0 is None:
                    sbar += wbar.sum()                           # the cold start is h_e_dot
                    wbar = None
                dt = kt[k + 1] - kt[k]                           # slope of segment k
                vbar[k + 1] += sbar / dt
                vbar[k] -= sbar / dt
                lam = ly
        return L, jcbar, vbar, wbar
