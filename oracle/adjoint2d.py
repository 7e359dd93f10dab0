"""Discrete adjoint of a thin-film solve (TEST INFRASTRUCTURE ONLY).

The paper has no adjoint; this oracle differentiates, exactly, the discrete map that Section 2
defines once two choices are frozen, so that the map is a plain function of its inputs:

  * the outside iteration (Eqs. 10-12) starts cold (free-space h_dot = h_e_dot) and runs a
    fixed number I of iterations: f(g; jc, h_e_dot) has no memory of earlier calls;
  * the time steps (t_n, h_n) of the Bogacki-Shampine 3(2) integrator are given (taken from a
    forward run), and every step is accepted; a step lies inside one waveform segment.

Map.  y_{n+1} = y_n + h_n (2/9 k1 + 1/3 k2 + 4/9 k3),  k1 = f(y_n),  k2 = f(y_n + h_n/2 k1),
k3 = f(y_n + 3 h_n/4 k2), with h_e_dot the slope of the step's waveform segment;
loss L = 1/2 dx dy sum (h_z(T) - target)^2,  h_z = h_e(T) + F^-1[(|k|/2) F g(T)] (end of
Section 2.1); parameters: the per-cell critical current density jc (Eq. 3, in the film) and
the values v_k of the piecewise-linear h_e(t).

Derivative pieces (reverse order of the forward):
  * every spectral operator T f = Re F^-1[M F f] has the transpose Re F^-1[conj(M) F v];
  * the shift of Eq. 10 and the centring of Eq. 11 are rank-one corrections, transposed as such;
  * Eq. 3: de/dj = rho (I + (n-1) j^ j^T) in the film, rho_out I elsewhere;
    de/djc = -(n/jc) e in the film;
  * the Runge-Kutta stages in reverse, each through the right-hand side's vector-Jacobian
    product; h_e_dot -> knot values through the segment slope, h_e(T) through the interpolation
    weights.

Pinned by tests/test_oracle_adjoint2d.py: the forward right-hand side equals
oracle.film2d.FilmProblem.rhs with the same cold start and iteration count; the transposed
outside iteration passes the dot-product test <P x, v> = <x, P^T v>; the vector-Jacobian
product of f and the gradient of L agree with central finite differences of the map.
"""
from __future__ import annotations

import numpy as np

from .film2d import FilmProblem

B = (2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0)      # Bogacki-Shampine weights of the third-order solution


class FilmAdjoint:
    """f(g; jc, h_e_dot) of a film with a cold, fixed-count outside iteration, its
    vector-Jacobian product, and the frozen-step solve with its gradient."""

    def __init__(self, problem: FilmProblem, iters: int):
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

    def P(self, hin, s):
        p = self.p
        hd = self._shift(np.where(p.out, s, hin), s)
        for i in range(self.I):
            u = self.T(p.K1, hd)                                 # Eq. 11
            gd = u - (u * self.out).sum() / self.nout
            if i == self.I - 1:
                break
            w = self.T(p.K2, gd * self.out)                      # Eq. 12
            hd = self._shift(hd - self.out * w, s)
        return np.where(self.cond, gd, 0.0)

    def P_T(self, v):
        """Transpose of P: (adjoint of h_dot_in, adjoint of h_e_dot)."""
        p = self.p
        gbar = np.where(self.cond, v, 0.0)
        hbar = np.zeros_like(gbar)
        sbar = 0.0
        for i in reversed(range(self.I)):
            if i < self.I - 1:
                # h_dot_{i+1} = shift(z), z = h_dot_i - out * K2 (out * g_dot_i)
                tot = (hbar * self.out).sum()
                sbar += self.N / self.nout * tot
                zbar = hbar - tot / self.nout
                hbar = zbar
                gbar = self.out * self.Tt(p.K2, -self.out * zbar)
            # g_dot_i = u_i - C(u_i), u_i = K1 h_dot_i
            ubar = gbar - self.out * gbar.sum() / self.nout
            hbar = hbar + self.Tt(p.K1, ubar)
        # h_dot_0 = shift(where(out, s, h_dot_in))
        tot = (hbar * self.out).sum()
        sbar += self.N / self.nout * tot
        pre = hbar - tot / self.nout
        return np.where(self.p.out, 0.0, pre), sbar + (pre * self.out).sum()

    # ---- the right-hand side and its vector-Jacobian product ------------------------------
    def rhs(self, g, jc, s):
        """f(g; jc, h_e_dot) and the values its vector-Jacobian product needs."""
        p = self.p
        jx, jy = self.T(p.Dy, g), -self.T(p.Dx, g)               # Eq. 2
        jabs = np.sqrt(jx * jx + jy * jy)
        rho_sc = (p.e0 / jc) * (jabs / jc) ** (p.n - 1.0)        # Eq. 3
        rho = np.where(p.sc, rho_sc, p.rho_out)
        ex, ey = rho * jx, rho * jy
        hin = np.where(self.cond, -(self.T(p.Dx, ey) - self.T(p.Dy, ex)), 0.0)   # Eq. 4 / 9
        return self.P(hin, s), (jx, jy, jabs, rho, ex, ey)

    def rhs_vjp(self, tape, jc, v):
        """(adjoint of g, of the jc map, of h_e_dot) for the cotangent v of f."""
        p = self.p
        jx, jy, jabs, rho, ex, ey = tape
        hbar_in, sbar = self.P_T(v)
        rbar = np.where(self.cond, -hbar_in, 0.0)                # h_in = -raw on the conductor
        eybar = self.Tt(p.Dx, rbar)                              # raw = Dx e_y - Dy e_x
        exbar = -self.Tt(p.Dy, rbar)
        safe = np.where(jabs > 0, jabs, 1.0)
        ux, uy = np.where(jabs > 0, jx / safe, 0.0), np.where(jabs > 0, jy / safe, 0.0)
        proj = ux * exbar + uy * eybar
        nn = np.where(p.sc, p.n - 1.0, 0.0)                      # Ohm's law elsewhere
        jxbar = rho * (exbar + nn * ux * proj)
        jybar = rho * (eybar + nn * uy * proj)
        jcbar = np.where(p.sc, -(p.n / jc) * (exbar * ex + eybar * ey), 0.0)
        gbar = self.Tt(p.Dy, jxbar) - self.Tt(p.Dx, jybar)       # j_x = Dy g, j_y = -Dx g
        return gbar, jcbar, sbar

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

    def solve(self, g0, jc, kt, kv, steps, keep=False):
        """Advance g0 over the given (t, h) steps; with keep, also the stage tapes."""
        y = np.array(g0, dtype=np.float64)
        tapes = []
        for t, h in steps:
            k = self._segment(kt, t, t + h)
            s = (kv[k + 1] - kv[k]) / (kt[k + 1] - kt[k])
            k1, t1 = self.rhs(y, jc, s)
            k2, t2 = self.rhs(y + 0.5 * h * k1, jc, s)
            k3, t3 = self.rhs(y + 0.75 * h * k2, jc, s)
            if keep:
                tapes.append((h, k, (t1, t2, t3)))
            y = y + h * (B[0] * k1 + B[1] * k2 + B[2] * k3)
        return (y, tapes) if keep else y

    def loss(self, g0, jc, kt, kv, steps, target):
        T = steps[-1][0] + steps[-1][1]
        y = self.solve(g0, jc, kt, kv, steps)
        hz = self._he(kt, kv, T)[0] + self.T(self.p.Kh, y)
        return 0.5 * self.p.dx * self.p.dy * float(((hz - target) ** 2).sum())

    def gradient(self, g0, jc, kt, kv, steps, target):
        """(L, dL/djc, dL/dv) by the discrete adjoint of the frozen-step solve."""
        p = self.p
        kt = np.asarray(kt, dtype=np.float64)
        kv = np.asarray(kv, dtype=np.float64)
        T = steps[-1][0] + steps[-1][1]
        y, tapes = self.solve(g0, jc, kt, kv, steps, keep=True)
        he, kT, wT = self._he(kt, kv, T)
        res = he + self.T(p.Kh, y) - target
        dA = p.dx * p.dy
        L = 0.5 * dA * float((res * res).sum())
        jcbar = np.zeros_like(np.asarray(jc, dtype=np.float64) * np.ones_like(y))
        vbar = np.zeros_like(kv)
        vbar[kT] += (1.0 - wT) * dA * res.sum()
        vbar[kT + 1] += wT * dA * res.sum()
        lam = dA * self.Tt(p.Kh, res)
        for h, k, (t1, t2, t3) in reversed(tapes):
            lk3 = h * B[2] * lam
            lk2 = h * B[1] * lam
            lk1 = h * B[0] * lam
            ly = lam.copy()
            sbar = 0.0
            gb, cb, sb = self.rhs_vjp(t3, jc, lk3)               # k3 = f(y + 3h/4 k2)
            ly += gb
            lk2 += 0.75 * h * gb
            jcbar += cb
            sbar += sb
            gb, cb, sb = self.rhs_vjp(t2, jc, lk2)               # k2 = f(y + h/2 k1)
            ly += gb
            lk1 += 0.5 * h * gb
            jcbar += cb
            sbar += sb
            gb, cb, sb = self.rhs_vjp(t1, jc, lk1)               # k1 = f(y)
            ly += gb
            jcbar += cb
            sbar += sb
            dt = kt[k + 1] - kt[k]                               # slope of segment k
            vbar[k + 1] += sbar / dt
            vbar[k] -= sbar / dt
            lam = ly
        return L, jcbar, vbar
