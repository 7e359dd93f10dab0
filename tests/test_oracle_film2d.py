"""Pins of the thin-film oracle (Section 2) against closed forms, invariants and physics."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.bs23 import BS23
from oracle.film2d import NOCONV, OK, FilmProblem
from oracle.waveform import Waveform


def _grid(n, L):
    return W.cell_centres(n, L)


def _film(nx, ny, Lx, Ly, mask, **kw):
    kw.setdefault("n", 19.0)
    kw.setdefault("rho_out", 1.0)
    kw.setdefault("waveform", Waveform((0.0, 1.0), (0.0, 0.5)))
    return FilmProblem(nx, ny, Lx, Ly, mask, **kw)


def test_smoothed_gradient_of_trig_mode():
    nx, ny, Lx, Ly = 32, 16, 2.0, 1.0
    p = _film(nx, ny, Lx, Ly, np.ones((ny, nx), np.uint8), sigma=0.07)
    x = _grid(nx, Lx)[None, :]
    y = _grid(ny, Ly)[:, None]
    kx, ky = math.pi * 3 / Lx, math.pi * 2 / Ly
    g = np.cos(kx * x + 0.3) * np.sin(ky * y)
    gx, gy = p.gradient(g)
    G = math.exp(-(kx * kx + ky * ky) * 0.07 ** 2 / 2)
    np.testing.assert_allclose(gx, -kx * G * np.sin(kx * x + 0.3) * np.sin(ky * y), atol=1e-12)
    np.testing.assert_allclose(gy, ky * G * np.cos(kx * x + 0.3) * np.cos(ky * y), atol=1e-12)
    jx, jy = p.sheet_current(g)                        # Eq. 2
    np.testing.assert_allclose(jx, gy, atol=0)
    np.testing.assert_allclose(jy, -gx, atol=0)


def test_odd_multiplier_zero_at_nyquist():
    p = _film(16, 8, 1.0, 1.0, np.ones((8, 16), np.uint8))
    g = np.tile((-1.0) ** np.arange(16), (8, 1))       # pure x-Nyquist mode
    gx, gy = p.gradient(g)
    assert np.abs(gx).max() < 1e-14 and np.abs(gy).max() < 1e-14


def test_inverse_pair_of_biot_savart_multipliers():
    p = _film(32, 32, 2.0, 2.0, np.ones((32, 32), np.uint8))
    f = W.rng(3).standard_normal((32, 32))
    np.testing.assert_allclose(p.apply(p.Kh * p.K1, f), f - f.mean(), atol=1e-13)


def test_field_of_gaussian_stream_function_closed_form():
    # continuous transform of Eq. 7 for g = exp(-r^2/2s^2):
    #   h_z(0) - h_e = (1/4pi^2) int (|k|/2) 2 pi s^2 e^{-k^2 s^2/2} d^2k = sqrt(2 pi) / (4 s)
    # (worked by hand); the bump is centred on a cell centre and the box is large, so the only
    # differences are periodic images and the k = 0 mode, both far below the tolerance.
    n, L, s = 256, 2.0, 0.1
    p = _film(n, n, L, L, np.ones((n, n), np.uint8))
    x = _grid(n, L)
    c = x[n // 2]
    r2 = (x[None, :] - c) ** 2 + (x[:, None] - c) ** 2
    g = np.exp(-r2 / (2 * s * s))
    hz = p.hz(0.0, g)
    assert hz[n // 2, n // 2] == pytest.approx(math.sqrt(2 * math.pi) / (4 * s), rel=1e-3)
    # away from the bump: the radial Hankel transform of the same closed form,
    #   h_z(r) = (s^2/2) int_0^inf k^2 e^{-k^2 s^2/2} J0(k r) dk,
    # plus the periodic images, which are point dipoles of moment m = 2 pi s^2 at that distance
    from scipy.integrate import quad
    from scipy.special import j0
    i = n // 2 + 38
    rr = x[i] - c
    iso = quad(lambda k: 0.5 * s * s * k * k * math.exp(-k * k * s * s / 2) * j0(k * rr),
               0, 400, limit=2000)[0]
    m = 2 * math.pi * s * s
    images = sum(-m / (4 * math.pi * math.hypot(rr - 2 * L * a, 2 * L * b) ** 3)
                 for a in range(-40, 41) for b in range(-40, 41) if (a, b) != (0, 0))
    assert hz[n // 2, i] == pytest.approx(iso + images, rel=1e-3)


def test_eddy_current_mode_decays_at_two_rho_k():
    # unbounded Ohmic sheet (whole box is conductor, n = 1): Maxwell's receding image gives a
    # decay rate 2 rho |k| (mu0 = 1); with smoothed derivatives both carry G(k)
    n, L = 32, 1.0
    p = _film(n, n, L, L, np.ones((n, n), np.uint8), n=1.0, jc=1.0, sigma=0.05)
    x = _grid(n, L)[None, :] + 0 * _grid(n, L)[:, None]
    k = math.pi * 2 / L
    g = np.cos(k * x)
    gd, it, st = p.rhs(0.3, g)
    G = math.exp(-k * k * 0.05 ** 2 / 2)
    np.testing.assert_allclose(gd, -2.0 * k * G * G * g, atol=1e-12)
    assert st == OK


def _square(n=64, L=2.0):
    return W.film_mask(n, n, L, L, "rect", ax=1.0, ay=1.0)


def test_rhs_invariants_on_square_film():
    n, L = 64, 2.0
    mask = _square(n, L)
    # a cold start converges slowly (the Meissner-like edge singularity), hence the high cap
    p = _film(n, n, L, L, mask, n=19.0, rho_out=1.0, iter_tol=2e-3, iter_max=5000)
    g = W.film_state(mask, L, L, seed=7, amplitude=0.6)
    t = 0.4
    gd, it, st = p.rhs(t, g)
    assert st == OK and it >= 1
    out = mask == 0
    assert np.all(gd[out] == 0.0)                                     # g stays 0 outside
    hd = p.last["hdot"]
    hed = p.wf.hedot(t)
    assert abs((hd - hed).sum()) < 1e-9 * np.abs(hd).sum()           # Eq. 10
    np.testing.assert_allclose(hd[~out], p.hdot_in(g)[~out], atol=0)  # h_dot_in untouched
    raw = p.apply(p.K1, hd) - p.last["C"]                             # Eq. 11
    assert abs(raw[out].mean()) < 1e-12
    assert np.abs(raw[out]).mean() < 2e-3                             # stop test met
    np.testing.assert_allclose(gd[~out], raw[~out], atol=1e-12)


def test_iteration_failure_and_fixed_count():
    n, L = 32, 2.0
    mask = W.film_mask(n, n, L, L, "rect", ax=1.0, ay=1.0)
    g = W.film_state(mask, L, L, seed=2, amplitude=0.6)
    p = _film(n, n, L, L, mask, iter_tol=1e-14, iter_max=2)
    _, it, st = p.rhs(0.1, g)
    assert st == NOCONV and it == 2
    p = _film(n, n, L, L, mask, iter_tol=0.0, iter_max=5)
    _, it, st = p.rhs(0.1, g)
    assert st == OK and it == 5


def test_ohmic_rhs_is_linear_for_a_fixed_iteration_count():
    # n = 1 and constant h_e: every step of Eqs. 9-12 is linear in g when the iteration starts
    # cold (initial guess h_e_dot = 0) and runs a fixed number of times
    n, L = 32, 2.0
    mask = W.film_mask(n, n, L, L, "disk", radius=1.0)
    kw = dict(n=1.0, rho_out=3.0, iter_tol=0.0, iter_max=7,
              waveform=Waveform((0.0, 1.0), (0.3, 0.3)))
    g1 = W.film_state(mask, L, L, seed=1)
    g2 = W.film_state(mask, L, L, seed=2, amplitude=0.3)
    f = lambda g: _film(n, n, L, L, mask, **kw).rhs(0.5, g)
    a, b = 0.7, -1.3
    r12, it, s1 = f(a * g1 + b * g2)
    r1, _, _ = f(g1)
    r2, _, _ = f(g2)
    assert s1 == OK and it == 7
    np.testing.assert_allclose(r12, a * r1 + b * r2, atol=1e-12 * np.abs(r12).max())


def test_bean_strip_critical_state():
    # strip |y| <= a across the periodic x direction in a rising field.  Bean limit for a thin
    # strip (sheet-current units): flux front b = a / cosh(pi h_e); inside the front
    # |j| = (2/pi) arctan(c |y| / sqrt(b^2 - y^2)), c = sqrt(1 - b^2/a^2), and h_z = 0;
    # |j| = 1 between the front and the edge.  n = 50 and the Gaussian filter smear the front
    # over ~3 sigma, which the masks below leave out.
    a, ny, Ly = 0.5, 512, 4.0
    nx = 8
    Lx = nx * (2 * Ly / ny) / 2
    mask = W.film_mask(nx, ny, Lx, Ly, "rect", ax=10.0, ay=a)
    he_end = 0.3
    wf = Waveform((0.0, 1.0), (0.0, he_end))
    p = FilmProblem(nx, ny, Lx, Ly, mask, n=50.0, rho_out=1.0, waveform=wf,
                    iter_tol=2e-4, iter_max=20000)
    s = BS23(p.rhs, wf, rtol=1e-5, atol=1e-5, on_accept=p.accept, on_attempt=p.begin_attempt)
    s.start(0.0, np.zeros((ny, nx)), 1.0)
    assert s.advance(1.0) == OK
    j = p.sheet_current(s.y)[0][:, 0]
    hz = p.hz(1.0, s.y)[:, 0]
    y = W.cell_centres(ny, Ly)
    b = a / math.cosh(math.pi * he_end)
    c = math.sqrt(1 - b * b / (a * a))
    core = np.abs(y) < b - 3 * p.sigma
    pen = (np.abs(y) > b + 3 * p.sigma) & (np.abs(y) < a - 3 * p.sigma)
    bean = (2 / math.pi) * np.arctan(c * np.abs(y[core]) / np.sqrt(b * b - y[core] ** 2))
    assert np.abs(np.abs(j[core]) - bean).max() < 0.05
    assert np.all((np.abs(j[pen]) > 0.85) & (np.abs(j[pen]) < 1.05)), j[pen]
    assert np.all(np.sign(j[pen]) == np.sign(y[pen]))                  # shielding sense
    assert np.abs(hz[core]).max() < 0.01 * he_end
    assert hz[pen].min() > 0.3 * he_end


def test_attempts_start_from_the_accepted_step():
    """Reading of 'the previous time step' (Section 2.2): after an accepted step the first
    evaluation of the next attempt starts from that step's final free-space h_dot, whatever the
    most recent call left; the later stages of an attempt start from the preceding stage."""
    n, L = 32, 2.0
    mask = W.film_mask(n, n, L, L, "rect", ax=1.0, ay=1.0)
    wf = Waveform((0.0, 1.0), (0.0, 0.5))
    kw = dict(n=19.0, rho_out=1.0, waveform=wf, iter_tol=2e-4, iter_max=3000)
    p = FilmProblem(n, n, L, L, mask, **kw)
    s = BS23(p.rhs, wf, rtol=1e-6, atol=1e-6, on_accept=p.accept, on_attempt=p.begin_attempt)
    g0 = W.film_state(mask, L, L, seed=21, amplitude=0.3)
    s.start(0.0, g0, 1.0)
    while s.attempt(1.0) != 1:
        pass
    # the accepted step's last evaluation (k4) left its iterate as the committed start
    assert p.committed is not None and np.array_equal(p.committed, p.warm)
    committed = p.committed.copy()
    # a stage outside an attempt start ignores the committed field ...
    p.warm = np.full_like(p.warm, 0.37)
    q = FilmProblem(n, n, L, L, mask, **kw)
    q.warm = p.warm.copy()
    a, _, _ = p.rhs(s.t, s.y, None, 3)
    b, _, _ = q.rhs(s.t, s.y, None, 3)
    assert np.array_equal(a, b)
    # ... while the first evaluation of an attempt starts from it
    p.warm = np.full_like(p.warm, 0.37)
    p.begin_attempt()
    a, _, _ = p.rhs(s.t, s.y, None, 3)
    q = FilmProblem(n, n, L, L, mask, **kw)
    q.warm = committed
    b, _, _ = q.rhs(s.t, s.y, None, 3)
    assert np.array_equal(a, b)
    assert p.attempt_first is False


def test_film_without_conductor_is_the_applied_field():
    """No superconductor, hence no sheet current: the field is the applied one everywhere, so the
    outside iteration ends at h_dot = h_e_dot on all of D (Eq. 10 with nothing to shift, Eq. 11
    with nothing to source) and f = 0 (g = 0 outside the film, reading 5); h_z = h_e."""
    n, L = 32, 2.0
    p = _film(n, n, L, L, np.zeros((n, n), np.uint8), waveform=Waveform((0.0, 1.0), (0.0, 0.5)))
    g = 0.01 * W.rng(3).standard_normal((n, n))
    for t in (0.1, 0.6):
        gd, it, st = p.rhs(t, g)
        assert st == OK and not gd.any()
        np.testing.assert_allclose(p.last["hdot"], 0.5, rtol=0, atol=1e-15)
    np.testing.assert_allclose(p.hz(0.6, np.zeros((n, n))), 0.3, rtol=0, atol=1e-15)
