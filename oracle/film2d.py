"""Oracle for the thin-film (2D) problem (TEST INFRASTRUCTURE ONLY).

Follows Section 2 of Prigozhin & Sokolovsky, FFT-based solution of 2D and 3D magnetization
problems in type-II superconductivity, in float64 and in the paper's order:

  Eq. 2   j = (d_y g, -d_x g)                      (stream function g, extended by 0 outside)
  Eq. 3   e = rho(|j|) j,  rho = (e0/jc) |j/jc|^(n-1) in the film; Ohm rho_out j elsewhere
          (Section 2.2: free space and filled holes)
  Eq. 4/9 h_z_dot = -curl e   on the conductor (film and filled holes)
  Section 2.2: derivatives are F^-1[i k exp(-|k|^2 sigma^2/2) F(.)], sigma = sqrt(dx^2+dy^2)
  Eq. 10  shift A on free space so that sum_D (h_dot - h_e_dot) = 0
  Eq. 11  g_dot^i = F^-1[(2/|k|) F h_dot^i] - C^i,  C^i = mean of the raw value over free space
  Eq. 12  h_dot_out^{i+1} = h_dot_out^i - lambda F^-1[(|k|/2) G F(g_dot^i_out)] - A^i
          (the same Gaussian smoothing G is used in Eq. 12, Section 2.2), lambda = 0.7
  stop    mean over free space of |g_dot^i| < tol = 2e-4 (Section 2.3), tested before the update
  h_z     h_z = h_e + F^-1[(|k|/2) F g]  (end of Section 2.1)

Readings where the paper is silent:
  * cell-centred grid x_i = -L + (i+1/2) dx; k = pi m / L with m in FFT order;
  * odd multipliers (i k_x, i k_y) are zero at the Nyquist index; even ones keep it;
  * 2/|k| and the A, C constants are zero/absent at k = 0;
  * the returned g_dot is zeroed on free space (g stays exactly 0 there);
  * the initial approximation is the free-space h_dot "from the previous time step" (Section
    2.2): the first evaluation of a step attempt (`begin_attempt()`) starts from the final
    iterate of the last evaluation of the integrator's most recent accepted step (`accept()`);
    the later stages of the attempt, and calls outside the integrator, start from the iterate
    of the most recent call (first call: h_e_dot); a call that fails with a residual above
    1e3 tol (or not finite) leaves no most-recent iterate;
  * the iteration stops without an update when it converges or reaches iter_max (then NOCONV);
  * iter_tol <= 0 runs exactly iter_max iterations and reports OK;
  * no free-space cells: a single pass with C = A = 0.

Pinned by tests/test_oracle_film2d.py: spectral derivatives and the Gaussian against trig
closed forms, 2/|k| and |k|/2 against the closed-form field of a Gaussian stream function,
Eq. 10/11 invariants, linearity of the Ohmic case, the exact decay rate 2 rho |k| of an
eddy-current mode of an unbounded Ohmic sheet, and Bean-limit flux fronts of a strip; by
tests/test_oracle_power_law_pins.py: the exact jc and e0 scalings of Eq. 3 with a lognormal jc
map, the Bean strip with a non-uniform jc (|j| = local jc in the penetrated zones), and Eq. 12's
multiplier as lambda times the smoothed field of the stray current; by
tests/test_oracle_direct_sums.py: every multiplier against O(N^2) Fourier sums; by
tests/test_oracle_laws.py: the elliptic law (gamma) through the gamma^2-slower Ohmic decay of a
mode whose current runs along y and the critical sheet current gamma jc of a strip along y.
"""
from __future__ import annotations

import math

import numpy as np

from . import _fft as dft
from .waveform import Waveform

OK, NOCONV = 0, 3


def wavenumbers(n: int, L: float) -> tuple[np.ndarray, np.ndarray]:
    """(k, is_nyquist) for n cells on [-L, L): k = 2 pi m / (2L), m in FFT order."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return np.pi * m / L, (m == -(n // 2))


class FilmProblem:
    """Method-of-lines right-hand side f(t, g) for a thin film (Section 2.2)."""

    def __init__(self, nx: int, ny: int, Lx: float, Ly: float, mask: np.ndarray, *, n: float,
                 rho_out: float, waveform: Waveform, jc=1.0, e0: float = 1.0,
                 sigma: float = 0.0, lam: float = 0.7, iter_tol: float = 2e-4,
                 iter_max: int = 100, gamma: float = 1.0):
        self.nx, self.ny, self.Lx, self.Ly = nx, ny, Lx, Ly
        self.dx, self.dy = 2.0 * Lx / nx, 2.0 * Ly / ny
        self.mask = np.asarray(mask, dtype=np.uint8).reshape(ny, nx)
        self.out = self.mask == 0
        self.conductor = ~self.out
        self.sc = self.mask == 1
        self.n, self.rho_out, self.e0 = float(n), float(rho_out), float(e0)
        self.jc = np.broadcast_to(np.asarray(jc, dtype=np.float64), (ny, nx))
        self.sigma = sigma if sigma > 0 else math.sqrt(self.dx ** 2 + self.dy ** 2)
        self.lam, self.iter_tol, self.iter_max = float(lam), float(iter_tol), int(iter_max)
        self.gamma = float(gamma)          # anisotropy: the critical current along y is gamma jc
        self.wf = waveform

        kx, nyq_x = wavenumbers(nx, Lx)
        ky, nyq_y = wavenumbers(ny, Ly)
        KX, KY = np.meshgrid(kx, ky)                   # [iy, ix]
        kabs = np.sqrt(KX ** 2 + KY ** 2)
        self.G = np.exp(-kabs ** 2 * self.sigma ** 2 / 2.0)
        self.Dx = 1j * KX * self.G
        self.Dx[:, nyq_x] = 0.0
        self.Dy = 1j * KY * self.G
        self.Dy[nyq_y, :] = 0.0
        with np.errstate(divide="ignore"):
            self.K1 = np.where(kabs > 0, 2.0 / np.where(kabs > 0, kabs, 1.0), 0.0)   # Eq. 11
        self.K2 = self.lam * (kabs / 2.0) * self.G                                  # Eq. 12
        self.Kh = kabs / 2.0                                                        # h_z readout
        self.warm = None          # free-space h_dot of the most recent call
        self.committed = None     # free-space h_dot of the previous (accepted) time step
        self.attempt_first = False    # the next call is the first of a step attempt
        self.last = {}

    # ---- spectral operators --------------------------------------------------------------
    @staticmethod
    def apply(mult: np.ndarray, f: np.ndarray) -> np.ndarray:
        """Re F^-1[mult F f] with the discrete Fourier transform."""
        return np.real(dft.ifft2(mult * dft.fft2(f)))

    def gradient(self, g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Gaussian-smoothed spectral gradient of g (Section 2.2)."""
        gh = dft.fft2(g)
        return np.real(dft.ifft2(self.Dx * gh)), np.real(dft.ifft2(self.Dy * gh))

    def sheet_current(self, g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Eq. 2: j_x = d_y g, j_y = -d_x g."""
        gx, gy = self.gradient(g)
        return gy, -gx

    def electric_field(self, jx: np.ndarray, jy: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Eq. 3 in the film, Ohm law rho_out j on free space and filled holes.  With gamma != 1
        the anisotropic (elliptic) law of the same family, one of the replacements the paper's
        conclusion names: j_eff = sqrt(j_x^2 + (j_y/gamma)^2), rho = (e0/jc)|j_eff/jc|^(n-1),
        e = rho (j_x, j_y/gamma^2) in the film (the critical current along y is gamma jc)."""
        g2 = self.gamma * self.gamma
        jeff = np.sqrt(jx * jx + jy * jy / g2)
        rho_sc = (self.e0 / self.jc) * (jeff / self.jc) ** (self.n - 1.0)
        rho = np.where(self.sc, rho_sc, self.rho_out)
        return rho * jx, rho * jy * np.where(self.sc, 1.0 / g2, 1.0)

    def hdot_in(self, g: np.ndarray) -> np.ndarray:
        """Eq. 4 / Eq. 9: h_z_dot = -(d_x e_y - d_y e_x) on the conductor, 0 elsewhere."""
        jx, jy = self.sheet_current(g)
        ex, ey = self.electric_field(jx, jy)
        curl = np.real(dft.ifft2(self.Dx * dft.fft2(ey) - self.Dy * dft.fft2(ex)))
        return np.where(self.conductor, -curl, 0.0)

    # ---- the right-hand side -------------------------------------------------------------
    def rhs(self, t: float, g: np.ndarray, seg: int | None = None,
            force_iters: int | None = None) -> tuple[np.ndarray, int, int]:
        """f(t, g): returns (g_dot, iterations, status) and updates the warm start."""
        g = np.asarray(g, dtype=np.float64).reshape(self.ny, self.nx)
        he_dot = self.wf.hedot(t, seg)
        N = self.nx * self.ny
        n_out = int(self.out.sum())
        h_in = self.hdot_in(g)

        if n_out == 0:                           # nothing to iterate: an unbounded film
            u = self.apply(self.K1, h_in)
            self.last = dict(C=0.0, A=0.0, r=0.0)
            return u, 1, OK

        # initial approximation (the previous time step's h_dot, Section 2.2) and the shift A^0
        # of Eq. 10
        first, self.attempt_first = self.attempt_first, False
        if first and self.committed is not None:
            warm = self.committed
        elif self.warm is not None:
            warm = self.warm
        else:
            warm = np.full((self.ny, self.nx), he_dot)
        hd = np.where(self.out, warm, h_in)
        A = (hd.sum() - N * he_dot) / n_out
        hd = np.where(self.out, hd - A, hd)
        self.warm = hd.copy()

        itmax = self.iter_max if force_iters is None else int(force_iters)
        fixed = self.iter_tol <= 0.0 and force_iters is None
        for i in range(itmax):
            u = self.apply(self.K1, hd)                                   # Eq. 11
            C = u[self.out].mean()
            gd = u - C
            r = np.abs(gd[self.out]).mean()                               # Section 2.3
            last = i == itmax - 1
            if force_iters is not None or fixed:
                stop = last
            else:
                stop = r < self.iter_tol or last
            if stop:
                break
            w = self.apply(self.K2, np.where(self.out, gd, 0.0))          # Eq. 12
            hd = np.where(self.out, hd - w, hd)
            A = (hd.sum() - N * he_dot) / n_out                           # Eq. 10
            hd = np.where(self.out, hd - A, hd)
            self.warm = hd.copy()
        status = OK if (fixed or self.iter_tol <= 0.0 or r < self.iter_tol) else NOCONV
        if status == NOCONV and not (r < 1e3 * self.iter_tol):
            self.warm = None       # a diverged iterate is no warm start; the next call starts cold
        self.last = dict(C=C, A=A, r=r, hdot=hd)
        return np.where(self.conductor, gd, 0.0), i + 1, status

    def accept(self) -> None:
        """The integrator accepted a step whose last evaluation was the most recent call: its
        free-space h_dot becomes the initial approximation of later calls."""
        if self.warm is not None:
            self.committed = self.warm.copy()

    def begin_attempt(self) -> None:
        """The integrator starts a step attempt: its first call starts from the accepted step."""
        self.attempt_first = True

    def reset_warm(self) -> None:
        self.warm = None
        self.committed = None
        self.attempt_first = False

    # ---- readouts ------------------------------------------------------------------------
    def hz(self, t: float, g: np.ndarray) -> np.ndarray:
        """h_z = h_e + F^-1[(|k|/2) F g] (end of Section 2.1)."""
        return self.wf.he(t) + self.apply(self.Kh, np.asarray(g).reshape(self.ny, self.nx))

    def magnetization(self, g: np.ndarray) -> float:
        """m_z = integral of g over the film (= 1/2 integral of r x j for g = 0 on the edge)."""
        return float(np.asarray(g).sum() * self.dx * self.dy)
