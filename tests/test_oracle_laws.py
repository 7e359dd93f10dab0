"""Pins of the oracle's other current-voltage laws (the paper's conclusion: the power law can be
replaced by anisotropic or field-dependent relations through the same method of lines).

* Anisotropic (elliptic) power law, e = rho(j_eff) (j_x, j_y, j_z / gamma^2) with
  j_eff^2 = j_x^2 + j_y^2 + (j_z / gamma)^2 (bulk; the film's anisotropy acts on j_y):
    - Ohmic limit n = 1: an eddy-current mode of an unbounded conductor whose current flows
      along the slow axis decays gamma^2 times slower (closed forms: 2 rho |k| G^2 for the sheet,
      Maxwell's receding image; rho |k|^2 G^2 for the bulk, the diffusion of h);
    - critical state: in the penetrated layer of a slab (current along z) or a strip (current
      along y) the current density is gamma jc.
* Field-dependent (Kim-type) critical current jc / (1 + |h| / b0) (bulk): in the critical
  state of a slab, |j| (1 + |h| / b0) = jc across the penetrated layer while |j| itself varies.
Mistakes planted in copies (the 1/gamma^2 factor of e dropped, gamma applied to the wrong
component, jc (1 + |h|/b0) in place of jc / (1 + |h|/b0)) fail these pins.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.bs23 import BS23
from oracle.bulk3d import BulkProblem
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform


def pin_film_aniso_ohmic_decay(cls):
    n, L, s, gam, rho = 32, 1.0, 0.05, 1.7, 1.3
    p = cls(n, n, L, L, np.ones((n, n), np.uint8), n=1.0, rho_out=1.0, jc=1.0 / rho, e0=1.0,
            waveform=Waveform((0.0, 1.0), (0.2, 0.2)), sigma=s, gamma=gam)
    x = W.cell_centres(n, L)[None, :] + 0 * W.cell_centres(n, L)[:, None]
    k = 2 * math.pi / L
    g = np.cos(k * x)                                   # j = (0, k sin kx): along y
    gd, _, _ = p.rhs(0.3, g)
    G = math.exp(-k * k * s * s / 2)
    np.testing.assert_allclose(gd, -2.0 * rho / gam ** 2 * k * G * G * g, atol=1e-12)


def pin_bulk_aniso_ohmic_decay(cls):
    n, L, s, gam, rho = 16, 1.0, 0.05, 1.7, 1.3
    p = cls(n, n, n, L, L, L, np.ones((n, n, n), np.uint8), n=1.0, rho_out=1.0, jc=1.0 / rho,
            e0=1.0, waveform=Waveform((0.0, 1.0), (0.0, 0.0)), sigma=s, gamma=gam)
    c = W.cell_centres(n, L)
    X = c[None, None, :] + 0 * c[None, :, None] + 0 * c[:, None, None]
    k = 2 * math.pi / L
    h = np.zeros((3, n, n, n))
    h[1] = np.cos(k * X)                                # j = curl h = (0, 0, -k sin kx): along z
    hd, _, _ = p.rhs(0.3, h)
    G = math.exp(-k * k * s * s / 2)
    want = np.zeros_like(h)
    want[1] = -rho / gam ** 2 * k * k * G * G * np.cos(k * X)
    np.testing.assert_allclose(hd, want, atol=1e-11)


def _slab(cls, he_dir, h_max, **law):
    """Slab |x| <= a (64 cells across the periodic box, 4 cells in y and z), n = 50, h_e
    ramped to h_max along he_dir.  In the periodic box the mean field is h_e, so the field
    outside rises above h_e while the slab shields."""
    a, nx, L = 0.5, 64, 1.0
    dx = 2 * L / nx
    nyz = 4
    Lyz = nyz * dx / 2
    mask = W.bulk_mask(nx, nyz, nyz, L, Lyz, Lyz, "slab", ax=a)
    wf = Waveform((0.0, 1.0), (0.0, h_max))
    p = cls(nx, nyz, nyz, L, Lyz, Lyz, mask, n=50.0, rho_out=5.0, waveform=wf, he_dir=he_dir,
            iter_tol=1e-4, iter_max=2000, **law)
    s = BS23(p.rhs, wf, rtol=1e-5, atol=1e-5)
    s.start(0.0, np.zeros((3, nyz, nyz, nx)), 1.0)
    assert s.advance(1.0) == 0
    x = W.cell_centres(nx, L)
    return p, s.y, p.current(s.y), x, a


def pin_bulk_aniso_critical_state(cls):
    gam = 2.0
    p, h, j, x, a = _slab(cls, (0.0, 1.0, 0.0), 0.6, gamma=gam)      # current along z
    jz = j[2, 0, 0, :]
    layer = (np.abs(x) < a - 2 * p.sigma) & (np.abs(x) > 0.16)       # penetrated, off the edge
    assert layer.sum() >= 10
    assert np.all(np.abs(np.abs(jz[layer]) - gam) < 0.1 * gam), jz[layer]


def pin_bulk_kim_critical_state(cls):
    b0 = 0.2
    p, h, j, x, a = _slab(cls, (0.0, 0.0, 1.0), 0.3, b0=b0)          # current along y
    jy = j[1, 0, 0, :]
    hm = np.sqrt((h[:, 0, 0, :] ** 2).sum(axis=0))
    layer = (np.abs(x) < a - 2 * p.sigma) & (np.abs(x) > 0.07)       # fully penetrated slab
    assert layer.sum() >= 14
    scaled = np.abs(jy[layer]) * (1.0 + hm[layer] / b0)
    assert np.all(np.abs(scaled - 1.0) < 0.1), scaled
    ja = np.abs(jy[layer])
    assert ja.max() < 0.8 and ja.max() > 1.2 * ja.min()               # |j| below jc, and varies


def pin_film_aniso_critical_state(cls):
    gam = 1.5
    a, nx, Lx, ny = 0.5, 256, 2.0, 8
    Ly = ny * (2 * Lx / nx) / 2
    mask = W.film_mask(nx, ny, Lx, Ly, "rect", ax=a, ay=10.0)            # strip along y
    wf = Waveform((0.0, 1.0), (0.0, 0.7))
    p = cls(nx, ny, Lx, Ly, mask, n=50.0, rho_out=1.0, waveform=wf, iter_tol=2e-4,
            iter_max=20000, gamma=gam)
    s = BS23(p.rhs, wf, rtol=1e-4, atol=1e-4, on_accept=p.accept, on_attempt=p.begin_attempt)
    s.start(0.0, np.zeros((ny, nx)), 1.0)
    assert s.advance(1.0) == 0
    jy = p.sheet_current(s.y)[1][0, :]
    x = W.cell_centres(nx, Lx)
    band = (np.abs(x) > a - 0.17) & (np.abs(x) < a - 4 * p.sigma)
    assert band.sum() >= 4
    assert np.all(np.abs(np.abs(jy[band]) - gam) < 0.07 * gam), jy[band]


def test_film_anisotropic_ohmic_decay():
    pin_film_aniso_ohmic_decay(FilmProblem)


def test_bulk_anisotropic_ohmic_decay():
    pin_bulk_aniso_ohmic_decay(BulkProblem)


@pytest.mark.slow
def test_bulk_anisotropic_critical_state():
    pin_bulk_aniso_critical_state(BulkProblem)


@pytest.mark.slow
def test_bulk_kim_critical_state():
    pin_bulk_kim_critical_state(BulkProblem)


@pytest.mark.slow
def test_film_anisotropic_critical_state():
    pin_film_aniso_critical_state(FilmProblem)


class FilmNoGammaSquared(FilmProblem):
    def electric_field(self, jx, jy):
        g2 = self.gamma * self.gamma
        jeff = np.sqrt(jx * jx + jy * jy / g2)
        rho = np.where(self.sc, (self.e0 / self.jc) * (jeff / self.jc) ** (self.n - 1.0), self.rho_out)
        return rho * jx, rho * jy


class BulkGammaOnX(BulkProblem):
    def electric_field(self, j, h=None):
        g2 = self.gamma * self.gamma
        jeff = np.sqrt(j[0] ** 2 / g2 + j[1] ** 2 + j[2] ** 2)
        rho = np.where(self.sc, (self.e0 / self.jc) * (jeff / self.jc) ** (self.n - 1.0), self.rho_out)
        e = rho[None] * j
        e[0] = e[0] * np.where(self.sc, 1.0 / g2, 1.0)
        return e


class BulkKimInverted(BulkProblem):
    def electric_field(self, j, h=None):
        jabs = np.sqrt((j * j).sum(axis=0))
        jc = self.jc * (1.0 + np.sqrt((np.asarray(h) ** 2).sum(axis=0)) / self.b0)
        rho = np.where(self.sc, (self.e0 / jc) * (jabs / jc) ** (self.n - 1.0), self.rho_out)
        return rho[None] * j


@pytest.mark.parametrize("pin,cls", [(pin_film_aniso_ohmic_decay, FilmNoGammaSquared),
                                     (pin_bulk_aniso_ohmic_decay, BulkGammaOnX)])
def test_planted_law_mistake_is_caught(pin, cls):
    with pytest.raises(AssertionError):
        pin(cls)


@pytest.mark.slow
@pytest.mark.parametrize("pin,cls", [(pin_bulk_kim_critical_state, BulkKimInverted),
                                     (pin_bulk_aniso_critical_state, BulkGammaOnX)])
def test_planted_critical_state_mistake_is_caught(pin, cls):
    with pytest.raises(AssertionError):
        pin(cls)
