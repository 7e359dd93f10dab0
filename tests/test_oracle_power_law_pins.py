"""Pins of the power law's critical current density and e0 (Eq. 3 / Eq. 13) and of the multiplier
of the film's outside iteration (Eq. 12) that do not repeat the oracle's own formula.

* Exact scaling of the power law rho = (e0/jc) |j/jc|^(n-1):
    - jc -> c jc (map included), rho_out -> rho_out / c, state -> c state: j scales by c, |j/jc|
      and e = rho j are unchanged, so h_dot_in, the outside iteration and f are unchanged;
    - e0 -> c e0, rho_out -> c rho_out with a constant applied field: e scales by c, and the
      cold-started outside iteration is linear and homogeneous in h_dot_in, so f scales by c.
  Both hold for any n and any jc map, so they are run with n = 19 and a lognormal map.
* The Bean limit with a non-uniform jc: in the penetrated zones of a strip the sheet current
  density is the local jc (here 1.6 on one half of the strip, 0.8 on the other), which fixes
  where the map enters and that jc is the current scale of the law.
* Eq. 12: the free-space correction is lambda times the normal field that the stray sheet current
  (stream function g_dot on free space) produces (Eq. 7 / the h_z readout, pinned by a closed
  form in test_oracle_film2d.py), smoothed by the Gaussian of Section 2.2 (pinned by trig modes).

Each pin is a function of a problem class, so that the last tests can plant mistakes in copies
of the oracle (subclasses, on the CPU) and check that every pin catches its mistake.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.bs23 import BS23
from oracle.bulk3d import BulkProblem
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform


# ------------------------------------------------------------------------------------------
# pins, written against a problem class
# ------------------------------------------------------------------------------------------
def _film_case(cls, *, jc, rho_out, e0=1.0, wf=None, n=19.0):
    nn, L = 32, 2.0
    mask = W.film_mask(nn, nn, L, L, "disk", radius=1.2)
    wf = wf or Waveform((0.0, 1.0), (0.0, 0.6))
    return cls(nn, nn, L, L, mask, n=n, rho_out=rho_out, waveform=wf, jc=jc, e0=e0,
               iter_tol=0.0, iter_max=6), mask


def pin_film_jc_scaling(cls):
    c = 1.7
    jc = W.jc_map_lognormal((32, 32), seed=11, sigma=0.3)
    p, mask = _film_case(cls, jc=jc, rho_out=2.0)
    q, _ = _film_case(cls, jc=c * jc, rho_out=2.0 / c)
    g = W.film_state(mask, 2.0, 2.0, seed=12, amplitude=0.9)
    a, _, _ = p.rhs(0.4, g)
    b, _, _ = q.rhs(0.4, c * g)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a), np.linalg.norm(a - b) / np.linalg.norm(a)


def pin_film_e0_scaling(cls):
    c = 2.5
    jc = W.jc_map_lognormal((32, 32), seed=13, sigma=0.3)
    hold = Waveform((0.0, 1.0), (0.3, 0.3))            # constant h_e: h_e_dot = 0
    p, mask = _film_case(cls, jc=jc, rho_out=1.5, e0=1.0, wf=hold)
    q, _ = _film_case(cls, jc=jc, rho_out=1.5 * c, e0=c, wf=hold)
    g = W.film_state(mask, 2.0, 2.0, seed=14, amplitude=0.9)
    a, _, _ = p.rhs(0.4, g)
    b, _, _ = q.rhs(0.4, g)
    assert np.linalg.norm(c * a - b) <= 1e-11 * np.linalg.norm(b)


def _bulk_case(cls, *, jc, rho_out, e0=1.0, wf=None):
    nn, L = 16, 1.0
    mask = W.bulk_mask(nn, nn, nn, L, L, L, "box", ax=0.5, ay=0.4, az=0.3)
    wf = wf or Waveform((0.0, 1.0), (0.0, 0.4))
    return cls(nn, nn, nn, L, L, L, mask, n=19.0, rho_out=rho_out, waveform=wf, jc=jc, e0=e0,
               iter_tol=0.0, iter_max=3), mask


def pin_bulk_jc_scaling(cls):
    c = 1.7
    jc = W.jc_map_lognormal((16, 16, 16), seed=15, sigma=0.3)
    p, mask = _bulk_case(cls, jc=jc, rho_out=5.0)
    q, _ = _bulk_case(cls, jc=c * jc, rho_out=5.0 / c)
    h = W.bulk_state(mask, (1.0, 1.0, 1.0), seed=16, h0=0.3, depth=0.3)
    a, _, _ = p.rhs(0.4, h)
    b, _, _ = q.rhs(0.4, c * h)
    # e, h_dot_in and the iteration are unchanged, so h_dot is too
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a)


def pin_bulk_e0_scaling(cls):
    c = 2.5
    jc = W.jc_map_lognormal((16, 16, 16), seed=17, sigma=0.3)
    hold = Waveform((0.0, 1.0), (0.2, 0.2))
    p, mask = _bulk_case(cls, jc=jc, rho_out=5.0, e0=1.0, wf=hold)
    q, _ = _bulk_case(cls, jc=jc, rho_out=5.0 * c, e0=c, wf=hold)
    h = W.bulk_state(mask, (1.0, 1.0, 1.0), seed=18, h0=0.3, depth=0.3)
    a, _, _ = p.rhs(0.4, h)
    b, _, _ = q.rhs(0.4, h)
    assert np.linalg.norm(c * a - b) <= 1e-11 * np.linalg.norm(b)


def pin_bean_strip_nonuniform_jc(cls):
    """Strip |y| <= a across the periodic x direction, jc = 1.6 for y > 0 and 0.8 for y < 0,
    n = 50, h_e ramped to 0.7: in the penetrated zone next to each edge |j| is that edge's jc
    (n = 50 puts it a few per cent below jc at these electric fields)."""
    a, ny, Ly, nx = 0.5, 256, 2.0, 8
    Lx = nx * (2 * Ly / ny) / 2
    mask = W.film_mask(nx, ny, Lx, Ly, "rect", ax=10.0, ay=a)
    y = W.cell_centres(ny, Ly)
    jc_y = np.where(y > 0, 1.6, 0.8)
    jc = np.broadcast_to(jc_y[:, None], (ny, nx)).copy()
    wf = Waveform((0.0, 1.0), (0.0, 0.7))
    p = cls(nx, ny, Lx, Ly, mask, n=50.0, rho_out=1.0, waveform=wf, jc=jc, iter_tol=2e-4,
            iter_max=20000)
    s = BS23(p.rhs, wf, rtol=1e-4, atol=1e-4, on_accept=p.accept, on_attempt=p.begin_attempt)
    s.start(0.0, np.zeros((ny, nx)), 1.0)
    assert s.advance(1.0) == 0
    jx = p.sheet_current(s.y)[0][:, 0]
    edge = 4 * p.sigma
    for sign, jc_edge in ((1, 1.6), (-1, 0.8)):
        band = (sign * y > a - 0.17) & (sign * y < a - edge)
        assert band.sum() >= 4
        assert np.all(np.abs(np.abs(jx[band]) - jc_edge) < 0.07 * jc_edge), (jc_edge, jx[band])
        assert np.all(np.sign(jx[band]) == sign)                       # shielding sense


def pin_eq12_multiplier(cls):
    nn, L = 32, 2.0
    p = cls(nn, nn, L, L, np.ones((nn, nn), np.uint8), n=19.0, rho_out=1.0,
            waveform=Waveform((0.0, 1.0), (0.0, 0.5)), lam=0.7, sigma=0.11)
    f = W.rng(31).standard_normal((nn, nn))
    field = p.hz(0.3, p.apply(p.G, f)) - p.wf.he(0.3)       # normal field of the stray current
    np.testing.assert_allclose(p.apply(p.K2, f), 0.7 * field, atol=1e-12 * np.abs(field).max())
    # and Gaussian smoothing of a single Fourier mode is the factor exp(-|k|^2 sigma^2 / 2)
    x = W.cell_centres(nn, L)
    k = math.pi * 3 / L
    mode = np.cos(k * x)[None, :] + 0 * x[:, None]
    np.testing.assert_allclose(p.apply(p.G, mode), math.exp(-k * k * 0.11 ** 2 / 2) * mode, atol=1e-12)


# ------------------------------------------------------------------------------------------
# the pins on the oracle
# ------------------------------------------------------------------------------------------
def test_film_power_law_jc_scaling():
    pin_film_jc_scaling(FilmProblem)


def test_film_power_law_e0_scaling():
    pin_film_e0_scaling(FilmProblem)


def test_bulk_power_law_jc_scaling():
    pin_bulk_jc_scaling(BulkProblem)


def test_bulk_power_law_e0_scaling():
    pin_bulk_e0_scaling(BulkProblem)


@pytest.mark.slow
def test_bean_strip_with_nonuniform_jc():
    pin_bean_strip_nonuniform_jc(FilmProblem)


def test_eq12_multiplier_is_lambda_times_smoothed_field_of_stray_current():
    pin_eq12_multiplier(FilmProblem)


# ------------------------------------------------------------------------------------------
# mistakes planted in copies of the oracle (CPU only): every pin catches its mistake
# ------------------------------------------------------------------------------------------
class FilmJcBaseDropped(FilmProblem):          # rho = (e0/jc) |j|^(n-1)
    def electric_field(self, jx, jy):
        jabs = np.sqrt(jx * jx + jy * jy)
        rho = np.where(self.sc, (self.e0 / self.jc) * jabs ** (self.n - 1.0), self.rho_out)
        return rho * jx, rho * jy


class FilmJcExponent(FilmProblem):             # rho = e0 |j|^(n-1) / jc^(n-1)
    def electric_field(self, jx, jy):
        jabs = np.sqrt(jx * jx + jy * jy)
        rho = np.where(self.sc, self.e0 * (jabs / self.jc) ** (self.n - 1.0), self.rho_out)
        return rho * jx, rho * jy


class FilmE0Dropped(FilmProblem):              # rho = (1/jc) |j/jc|^(n-1)
    def electric_field(self, jx, jy):
        jabs = np.sqrt(jx * jx + jy * jy)
        rho = np.where(self.sc, (1.0 / self.jc) * (jabs / self.jc) ** (self.n - 1.0), self.rho_out)
        return rho * jx, rho * jy


class FilmJcTransposed(FilmProblem):           # the jc map read with x and y swapped
    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.jc = np.ascontiguousarray(np.asarray(self.jc).reshape(self.nx, self.ny).T)


class FilmK2NoGaussian(FilmProblem):
    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.K2 = self.lam * self.Kh


class FilmK2LambdaOne(FilmProblem):
    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.K2 = self.Kh * self.G


class BulkJcBaseDropped(BulkProblem):
    def electric_field(self, j, h=None):
        jabs = np.sqrt((j * j).sum(axis=0))
        rho = np.where(self.sc, (self.e0 / self.jc) * jabs ** (self.n - 1.0), self.rho_out)
        return rho[None] * j


class BulkE0Dropped(BulkProblem):
    def electric_field(self, j, h=None):
        jabs = np.sqrt((j * j).sum(axis=0))
        rho = np.where(self.sc, (1.0 / self.jc) * (jabs / self.jc) ** (self.n - 1.0), self.rho_out)
        return rho[None] * j


@pytest.mark.parametrize("pin,cls", [
    (pin_film_jc_scaling, FilmJcBaseDropped),
    (pin_film_jc_scaling, FilmJcExponent),
    (pin_film_e0_scaling, FilmE0Dropped),
    (pin_bulk_jc_scaling, BulkJcBaseDropped),
    (pin_bulk_e0_scaling, BulkE0Dropped),
    (pin_eq12_multiplier, FilmK2NoGaussian),
    (pin_eq12_multiplier, FilmK2LambdaOne),
])
def test_planted_mistake_is_caught(pin, cls):
    with pytest.raises(AssertionError):
        pin(cls)


@pytest.mark.slow
@pytest.mark.parametrize("cls", [FilmJcBaseDropped, FilmJcTransposed])
def test_planted_jc_mistake_is_caught_by_the_bean_strip(cls):
    with pytest.raises(AssertionError):
        pin_bean_strip_nonuniform_jc(cls)
