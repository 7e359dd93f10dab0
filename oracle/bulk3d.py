"""Oracle for the bulk (3D) problem in the magnetic-field formulation (TEST INFRASTRUCTURE ONLY).

Follows Section 3.1 of Prigozhin & Sokolovsky in float64 and in the paper's order:

  j = curl h (Ampere law), e = rho(|j|) j in the superconductor (Eq. 13), rho_out j elsewhere
  h_dot_in = -curl e on the conductor (Eq. 14, mu0 = 1)
  Phi[j] = F^-1{ (i/|k|^2) k x F(j) },  1/|k|^2 -> 0 at k = 0            (Eq. 17)
  iteration (Eq. 18): j_dot^i = curl h_dot^i, j_dot_in^i = j_dot^i on the conductor, 0 outside,
                      h_dot_out^{i+1} = h_e_dot + Phi[j_dot_in^i] on free space
  stop when mean over free-space nodes of |h_dot^{i+1} - h_dot^i| < delta_it max(|h_e_dot|, 1)
  all derivatives are Gaussian-smoothed spectral derivatives, sigma = sqrt(dx^2+dy^2+dz^2)
  (Section 3.1, last paragraph; Section 3.2).

Readings where the paper is silent:
  * odd multipliers i k_c are zero at the Nyquist index of axis c, in the curls and in Phi;
    Phi carries no Gaussian;
  * the conductor (mask 1 superconductor, mask 2 normal cutting layer) keeps h_dot_in and
    contributes to j_dot_in; the iteration updates free space (mask 0) only;
  * warm start from the most recent call (first call: h_e_dot), dropped after a call that fails
    with a residual above 1e3 times the threshold (or not finite); h_dot after the last update is
    returned on all of D;
  * iter_tol <= 0 runs exactly iter_max iterations and reports OK;
  * magnetization m = 1/2 sum dV r x j over the conductor.

Arrays are (3, nz, ny, nx), component-major (SoA).  Pinned by tests/test_oracle_bulk3d.py:
curl of trig fields, the closed-form centre field (2/3) m0 of a spherically symmetric Gaussian
magnetization for Phi, curl Phi[j] = j for divergence-free j, Ohmic linearity, invariants and
the Bean slab profile; by tests/test_oracle_power_law_pins.py: the exact jc and e0 scalings of
Eq. 13 with a lognormal jc map; by tests/test_oracle_laws.py: the elliptic law (gamma) through
the gamma^2-slower Ohmic decay of a mode whose current runs along z and the critical current
gamma jc of a slab carrying it, and the Kim law (b0) through |j| (1 + |h|/b0) = jc across a fully
penetrated slab.
"""
from __future__ import annotations

import math

import numpy as np

from . import _fft as dft
from .film2d import wavenumbers
from .waveform import Waveform

OK, NOCONV = 0, 3


class BulkProblem:
    def __init__(self, nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float,
                 mask: np.ndarray, *, n: float, rho_out: float, waveform: Waveform,
                 he_dir=(0.0, 0.0, 1.0), jc=1.0, e0: float = 1.0, sigma: float = 0.0,
                 iter_tol: float = 1e-4, iter_max: int = 100, gamma: float = 1.0,
                 b0: float = math.inf):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.L = (Lx, Ly, Lz)
        self.d = (2 * Lx / nx, 2 * Ly / ny, 2 * Lz / nz)
        self.mask = np.asarray(mask, dtype=np.uint8).reshape(nz, ny, nx)
        self.out = self.mask == 0
        self.conductor = ~self.out
        self.sc = self.mask == 1
        self.n, self.rho_out, self.e0 = float(n), float(rho_out), float(e0)
        self.jc = np.broadcast_to(np.asarray(jc, dtype=np.float64), (nz, ny, nx))
        self.sigma = sigma if sigma > 0 else math.sqrt(sum(x * x for x in self.d))
        self.iter_tol, self.iter_max = float(iter_tol), int(iter_max)
        self.gamma = float(gamma)          # anisotropy: the critical current along z is gamma jc
        self.b0 = float(b0)                # field dependence jc / (1 + |h|/b0); inf: none
        self.wf = waveform
        self.he_dir = np.asarray(he_dir, dtype=np.float64)

        kx, nqx = wavenumbers(nx, Lx)
        ky, nqy = wavenumbers(ny, Ly)
        kz, nqz = wavenumbers(nz, Lz)
        KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
        k2 = KX ** 2 + KY ** 2 + KZ ** 2
        self.G = np.exp(-k2 * self.sigma ** 2 / 2.0)
        # odd factors with the Nyquist index of their own axis removed
        kxo = np.where(np.broadcast_to(nqx[None, None, :], KX.shape), 0.0, KX)
        kyo = np.where(np.broadcast_to(nqy[None, :, None], KY.shape), 0.0, KY)
        kzo = np.where(np.broadcast_to(nqz[:, None, None], KZ.shape), 0.0, KZ)
        self.kodd = (kxo, kyo, kzo)
        self.D = tuple(1j * k * self.G for k in self.kodd)      # smoothed i k_c
        with np.errstate(divide="ignore"):
            self.inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
        self.warm = None
        self.last = {}

    # ---- operators -----------------------------------------------------------------------
    @staticmethod
    def _fft(v):
        return [dft.fftn(c) for c in v]

    @staticmethod
    def _ifft_re(vh):
        return np.stack([np.real(dft.ifftn(c)) for c in vh])

    def curl(self, v: np.ndarray) -> np.ndarray:
        """Gaussian-smoothed spectral curl of a vector field (3, nz, ny, nx)."""
        a = self._fft(v)
        Dx, Dy, Dz = self.D
        return self._ifft_re([Dy * a[2] - Dz * a[1], Dz * a[0] - Dx * a[2], Dx * a[1] - Dy * a[0]])

    def phi(self, j: np.ndarray) -> np.ndarray:
        """Eq. 17: Phi[j] = F^-1{ (i/|k|^2) k x F(j) }."""
        a = self._fft(j)
        kx, ky, kz = self.kodd
        f = 1j * self.inv_k2
        return self._ifft_re([f * (ky * a[2] - kz * a[1]), f * (kz * a[0] - kx * a[2]),
                              f * (kx * a[1] - ky * a[0])])

    def electric_field(self, j: np.ndarray, h: np.ndarray | None = None) -> np.ndarray:
        """Eq. 13 in the superconductor, Ohm law rho_out j elsewhere.  Other laws of the same
        family, which the paper's conclusion names as replacements: with gamma != 1 the
        elliptic power law j_eff = sqrt(j_x^2 + j_y^2 + (j_z/gamma)^2),
        e = rho(j_eff) (j_x, j_y, j_z/gamma^2); with a finite b0 the Kim-type critical current
        jc / (1 + |h|/b0), |h| the local field (the state h at the cell)."""
        g2 = self.gamma * self.gamma
        jeff = np.sqrt(j[0] ** 2 + j[1] ** 2 + j[2] ** 2 / g2)
        jc = self.jc
        if math.isfinite(self.b0):
            jc = jc / (1.0 + np.sqrt((np.asarray(h) ** 2).sum(axis=0)) / self.b0)
        rho_sc = (self.e0 / jc) * (jeff / jc) ** (self.n - 1.0)
        rho = np.where(self.sc, rho_sc, self.rho_out)
        e = rho[None] * j
        e[2] = e[2] * np.where(self.sc, 1.0 / g2, 1.0)
        return e

    def hdot_in(self, h: np.ndarray) -> np.ndarray:
        """Eq. 14: h_dot = -curl e on the conductor, with e from j = curl h."""
        e = self.electric_field(self.curl(h), h)
        return np.where(self.conductor[None], -self.curl(e), 0.0)

    # ---- the right-hand side -------------------------------------------------------------
    def rhs(self, t: float, h: np.ndarray, seg: int | None = None,
            force_iters: int | None = None) -> tuple[np.ndarray, int, int]:
        h = np.asarray(h, dtype=np.float64).reshape(3, self.nz, self.ny, self.nx)
        hed = self.wf.hedot(t, seg) * self.he_dir
        h_in = self.hdot_in(h)
        n_out = int(self.out.sum())
        if n_out == 0:
            self.last = dict(r=0.0)
            return h_in, 0, OK
        warm = self.warm if self.warm is not None else \
            np.broadcast_to(hed[:, None, None, None], h.shape)
        hd = np.where(self.out[None], warm, h_in)
        thresh = self.iter_tol * max(float(np.linalg.norm(hed)), 1.0)
        itmax = self.iter_max if force_iters is None else int(force_iters)
        fixed = self.iter_tol <= 0.0 and force_iters is None
        for i in range(itmax):
            jd = np.where(self.conductor[None], self.curl(hd), 0.0)       # j_dot_in^i
            hd_new = np.where(self.out[None], hed[:, None, None, None] + self.phi(jd), hd)  # Eq. 18
            diff = np.sqrt(((hd_new - hd) ** 2).sum(axis=0))
            r = diff[self.out].mean()
            hd = hd_new
            self.warm = hd.copy()
            if force_iters is not None or fixed:
                continue
            if r < thresh:
                break
        status = OK if (fixed or self.iter_tol <= 0.0 or r < thresh) else NOCONV
        if status == NOCONV and not (r < 1e3 * thresh):
            self.warm = None       # a diverged iterate is no warm start; the next call starts cold
        self.last = dict(r=r, thresh=thresh)
        return hd, i + 1, status

    # ---- readouts ------------------------------------------------------------------------
    def current(self, h: np.ndarray) -> np.ndarray:
        return self.curl(np.asarray(h).reshape(3, self.nz, self.ny, self.nx))

    def magnetization(self, h: np.ndarray) -> np.ndarray:
        """m = 1/2 sum dV r x j over the conductor."""
        j = self.current(h)
        Lx, Ly, Lz = self.L
        dx, dy, dz = self.d
        x = (-Lx + (np.arange(self.nx) + 0.5) * dx)[None, None, :]
        y = (-Ly + (np.arange(self.ny) + 0.5) * dy)[None, :, None]
        z = (-Lz + (np.arange(self.nz) + 0.5) * dz)[:, None, None]
        c = self.conductor
        dV = dx * dy * dz
        mx = 0.5 * dV * np.where(c, y * j[2] - z * j[1], 0.0).sum()
        my = 0.5 * dV * np.where(c, z * j[0] - x * j[2], 0.0).sum()
        mz = 0.5 * dV * np.where(c, x * j[1] - y * j[0], 0.0).sum()
        return np.array([mx, my, mz])
