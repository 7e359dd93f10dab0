"""Pins of the bulk (3D) oracle (Section 3.1) against closed forms, identities and physics."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.bs23 import BS23
from oracle.bulk3d import NOCONV, OK, BulkProblem
from oracle.waveform import Waveform


def _bulk(N, L, mask=None, **kw):
    kw.setdefault("n", 25.0)
    kw.setdefault("rho_out", 5.0)
    kw.setdefault("waveform", Waveform((0.0, 1.0), (0.0, 0.5)))
    if mask is None:
        mask = np.ones((N, N, N), np.uint8)
    return BulkProblem(N, N, N, L, L, L, mask, **kw)


def _xyz(n, L):
    c = W.cell_centres(n, L)
    return c[None, None, :], c[None, :, None], c[:, None, None]


def test_smoothed_curl_of_trig_field():
    n, L, s = 16, 1.0, 0.05
    p = _bulk(n, L, sigma=s)
    x, y, z = _xyz(n, L)
    k = math.pi / L
    kx, ky, kz = 2 * k, 1 * k, 3 * k
    v = np.zeros((3, n, n, n))
    v[0] = np.sin(ky * y) + 0 * x + 0 * z          # curl = (0, 0, -ky cos(ky y))
    v[2] = np.cos(kx * x) * np.sin(kz * z) + 0 * y  # curl = (0, kx sin(kx x) sin(kz z), 0)
    c = p.curl(v)
    G1 = math.exp(-ky * ky * s * s / 2)
    G2 = math.exp(-(kx * kx + kz * kz) * s * s / 2)
    np.testing.assert_allclose(c[0], 0 * c[0], atol=1e-12)
    np.testing.assert_allclose(c[1], G2 * kx * np.sin(kx * x) * np.sin(kz * z) + 0 * y, atol=1e-12)
    np.testing.assert_allclose(c[2], -G1 * ky * np.cos(ky * y) + 0 * x + 0 * z, atol=1e-12)


def _gaussian_magnetization_current(n, L, s, m0):
    """j = curl M for M = m0 z_hat exp(-r^2/2s^2) centred on a cell centre, evaluated exactly."""
    x, y, z = _xyz(n, L)
    c = W.cell_centres(n, L)[n // 2]
    X, Y, Z = x - c, y - c, z - c
    Mz = m0 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * s * s))
    j = np.zeros((3, n, n, n))
    j[0] = -Y / (s * s) * Mz              # d_y M_z
    j[1] = X / (s * s) * Mz               # -d_x M_z
    return j, Mz


def test_biot_savart_operator_centre_of_gaussian_magnetization():
    # Phi[curl M] has Fourier transform M_hat - k_hat (k_hat . M_hat).  For M = m0 z_hat g(|r|)
    # the cubic lattice of wavevectors makes the lattice sum of k_hat_z^2 over each shell 1/3,
    # so on the periodic box with k = 0 removed:  Phi_z(0) = (2/3) (m0 - m_tot / V)  exactly up
    # to aliasing (here < 1e-12), where m_tot = sum M dV.  (Uniformly magnetized ball analogue:
    # B/mu0 = M + H with H = -M/3 at the centre.)
    n, L, s, m0 = 48, 1.0, 0.12, 1.7
    p = _bulk(n, L)
    j, Mz = _gaussian_magnetization_current(n, L, s, m0)
    h = p.phi(j)
    dV = (2 * L / n) ** 3
    expect = (2.0 / 3.0) * (m0 - Mz.sum() * dV / (2 * L) ** 3)
    c = n // 2
    assert h[2, c, c, c] == pytest.approx(expect, rel=1e-9)
    assert abs(h[0, c, c, c]) < 1e-12 and abs(h[1, c, c, c]) < 1e-12


def test_curl_of_phi_is_identity_on_divergence_free_current():
    # the paper's identity curl Phi[j] = j (Section 3.1), with the Gaussian switched off
    n, L, s, m0 = 32, 1.0, 0.15, 1.0
    p = _bulk(n, L, sigma=1e-30)
    j, _ = _gaussian_magnetization_current(n, L, s, m0)
    np.testing.assert_allclose(p.curl(p.phi(j)), j, atol=1e-9 * np.abs(j).max())


def test_rhs_invariants_and_conductor_unchanged():
    n, L = 16, 1.0
    mask = W.bulk_mask(n, n, n, L, L, L, "box", ax=0.5, ay=0.5, az=0.5)
    p = _bulk(n, L, mask, iter_tol=1e-4, iter_max=500)
    h = W.bulk_state(mask, (L, L, L), seed=4)
    hd, it, st = p.rhs(0.3, h)
    assert st == OK and it >= 1
    out = mask == 0
    np.testing.assert_allclose(hd[:, ~out], p.hdot_in(h)[:, ~out], atol=0)
    # converged: one more application of Eq. 18 moves free space by less than the tolerance
    hed = p.wf.hedot(0.3) * p.he_dir
    jd = np.where(p.conductor[None], p.curl(hd), 0.0)
    again = hed[:, None, None, None] + p.phi(jd)
    diff = np.sqrt(((again - hd) ** 2).sum(axis=0))[out].mean()
    assert diff < 1e-4 * max(np.linalg.norm(hed), 1.0)


def test_fixed_count_and_failure():
    n, L = 16, 1.0
    mask = W.bulk_mask(n, n, n, L, L, L, "box", ax=0.5, ay=0.5, az=0.5)
    h = W.bulk_state(mask, (L, L, L), seed=5)
    p = _bulk(n, L, mask, iter_tol=1e-15, iter_max=2)
    assert p.rhs(0.2, h)[1:] == (2, NOCONV)
    p = _bulk(n, L, mask, iter_tol=0.0, iter_max=3)
    assert p.rhs(0.2, h)[1:] == (3, OK)


def test_ohmic_rhs_is_linear_for_a_fixed_iteration_count():
    n, L = 16, 1.0
    mask = W.bulk_mask(n, n, n, L, L, L, "ball", r_out=0.6)
    kw = dict(n=1.0, rho_out=4.0, iter_tol=0.0, iter_max=4,
              waveform=Waveform((0.0, 1.0), (0.2, 0.2)))
    h1 = W.bulk_state(mask, (L, L, L), seed=1)
    h2 = W.bulk_state(mask, (L, L, L), seed=2)
    f = lambda h: _bulk(16, L, mask, **kw).rhs(0.5, h)[0]
    a, b = -0.4, 1.9
    np.testing.assert_allclose(f(a * h1 + b * h2), a * f(h1) + b * f(h2), atol=1e-12)


def test_bean_slab_profile():
    # slab |x| <= a, periodic in y and z, h_e along z: the Bean profile has |d h_z/dx| = 1 (jc)
    # in the penetrated layer and a flux-free core; h_z on the slab surface is computed (the
    # periodic k = 0 removal shifts the outside level), the depth is that surface value.
    a, nx, L = 0.5, 64, 1.0
    dx = 2 * L / nx
    nyz = 4
    Lyz = nyz * dx / 2
    mask = W.bulk_mask(nx, nyz, nyz, L, Lyz, Lyz, "slab", ax=a)
    wf = Waveform((0.0, 1.0), (0.0, 0.25))
    p = BulkProblem(nx, nyz, nyz, L, Lyz, Lyz, mask, n=50.0, rho_out=5.0, waveform=wf,
                    iter_tol=1e-4, iter_max=2000)
    s = BS23(p.rhs, wf, rtol=1e-5, atol=1e-5)
    s.start(0.0, np.zeros((3, nyz, nyz, nx)), 1.0)
    assert s.advance(1.0) == OK
    h = s.y
    hz = h[2, 0, 0, :]
    jy = p.current(h)[1, 0, 0, :]
    x = W.cell_centres(nx, L)
    inside = np.abs(x) <= a
    hs = hz[np.abs(x) > a + 0.2].mean()                  # level outside the slab
    depth = hs - hz[nx // 2]                             # Bean: slope 1 from h_s to the core
    assert 0.25 < depth < 0.45
    front = a - depth
    layer = inside & (np.abs(x) > front + 2 * p.sigma) & (np.abs(x) < a - 2 * p.sigma)
    core = np.abs(x) < front - 2 * p.sigma
    assert layer.sum() >= 3 and core.sum() >= 1
    assert np.all(np.abs(np.abs(jy[layer]) - 1.0) < 0.1), jy[layer]
    assert np.all(np.sign(jy[layer]) == -np.sign(x[layer]))        # j_y = -d h_z / dx
    assert np.abs(jy[core]).max() < 0.5
    assert np.abs(jy[np.abs(x) > a + 0.1]).max() < 0.01            # no stray current outside


def test_body_without_conductor_follows_the_applied_field():
    """No superconductor: Eq. 18 adds to h_e_dot the field of the currents in Omega, and there are
    none, so h_dot = h_e_dot along the applied direction on all of D, on the ramp and after its
    knot; BS23 integrates that piecewise-constant rate exactly, so a ramp from h = 0 stays at
    h_e(t) times the direction, and the moment stays 0."""
    d = np.array([0.6, 0.0, 0.8])
    wf = Waveform((0.0, 0.5, 1.0), (0.0, 0.25, 0.25))
    p = _bulk(16, 1.0, mask=np.zeros((16, 16, 16), np.uint8), waveform=wf, he_dir=tuple(d),
              iter_tol=1e-4)
    h = 0.01 * W.rng(4).standard_normal((3, 16, 16, 16))
    for t, rate in ((0.1, 0.5), (0.7, 0.0)):
        hd, it, st = p.rhs(t, h)
        assert st == OK
        np.testing.assert_allclose(hd, np.broadcast_to(rate * d[:, None, None, None], hd.shape),
                                   rtol=0, atol=1e-15)
    p = _bulk(16, 1.0, mask=np.zeros((16, 16, 16), np.uint8), waveform=wf, he_dir=tuple(d),
              iter_tol=1e-4)
    s = BS23(p.rhs, wf, rtol=1e-6, atol=1e-6)
    s.start(0.0, np.zeros((3, 16, 16, 16)), 1.0)
    s.advance(1.0)
    assert s.t == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(s.y, np.broadcast_to(0.25 * d[:, None, None, None], s.y.shape),
                               rtol=0, atol=1e-14)
    assert not p.magnetization(s.y).any()
