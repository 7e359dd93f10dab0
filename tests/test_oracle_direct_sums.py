"""Pins of the oracle's Fourier machinery that do not go through numpy.fft: plain O(N^2) sums
of the discrete Fourier series on tiny grids (cell-centred points, k = pi m / L; they catch a
wrong wavenumber scale, ordering, normalisation or component), the symmetry Parseval's identity
gives every real even multiplier and the antisymmetry of the derivatives, and the moment
identity 1/2 int r x j = int g (films) / int M (bulk), which fixes the sign of the sheet
current (Eq. 2) and of the curl.  (Keeping or zeroing the Nyquist term of an odd multiplier
gives the same real part here, so these pins do not decide that reading.)"""
import numpy as np

import workloads as W
from oracle.bulk3d import BulkProblem
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform

WF = Waveform((0.0, 1.0), (0.0, 0.5))


def _modes(n, L):
    """Cell centres x_j and the wavenumbers k_m = pi m / L, m = -n/2 .. n/2 - 1 (Section 2.2)."""
    x = -L + (np.arange(n) + 0.5) * (2.0 * L / n)
    m = np.arange(-(n // 2), n // 2)
    return x, np.pi * m / L, m == -(n // 2)


def _direct_2d(f, Lx, Ly, mult):
    """Re of (1/N) sum_k mult(kx, ky) [sum_x f(x) e^{-i k.x}] e^{i k.x}, term by term."""
    ny, nx = f.shape
    x, kx, nqx = _modes(nx, Lx)
    y, ky, nqy = _modes(ny, Ly)
    Ex = np.exp(-1j * np.outer(kx, x))            # [m, j]
    Ey = np.exp(-1j * np.outer(ky, y))
    fh = Ey @ f @ Ex.T                              # [my, mx]
    KX, KY = np.meshgrid(kx, ky)
    NX, NY = np.meshgrid(nqx, nqy)
    gh = mult(KX, KY, NX, NY) * fh
    return np.real(Ey.conj().T @ gh @ Ex.conj()) / (nx * ny)


def test_film_operators_equal_direct_fourier_sums():
    nx, ny, Lx, Ly, s = 8, 6, 1.3, 0.7, 0.2
    p = FilmProblem(nx, ny, Lx, Ly, np.ones((ny, nx), np.uint8), n=19.0, rho_out=1.0,
                    waveform=WF, sigma=s)
    f = W.rng(21).standard_normal((ny, nx))
    G = lambda kx, ky: np.exp(-(kx * kx + ky * ky) * s * s / 2)
    gx, gy = p.gradient(f)
    np.testing.assert_allclose(gx, _direct_2d(f, Lx, Ly, lambda kx, ky, nx_, ny_:
                                              np.where(nx_, 0, 1j * kx * G(kx, ky))), atol=1e-12)
    np.testing.assert_allclose(gy, _direct_2d(f, Lx, Ly, lambda kx, ky, nx_, ny_:
                                              np.where(ny_, 0, 1j * ky * G(kx, ky))), atol=1e-12)
    kab = lambda kx, ky: np.sqrt(kx * kx + ky * ky)
    k1 = lambda kx, ky, a, b: np.where(kab(kx, ky) > 0, 2 / np.maximum(kab(kx, ky), 1e-300), 0)
    np.testing.assert_allclose(p.apply(p.K1, f), _direct_2d(f, Lx, Ly, k1), atol=1e-12)
    # Eq. 12's multiplier lambda (|k|/2) exp(-|k|^2 sigma^2/2), lambda = 0.7 (Section 2.2)
    np.testing.assert_allclose(p.apply(p.K2, f), _direct_2d(f, Lx, Ly, lambda kx, ky, a, b:
                                                           0.7 * kab(kx, ky) / 2 * G(kx, ky)), atol=1e-12)
    np.testing.assert_allclose(p.hz(0.4, f) - WF.he(0.4),
                               _direct_2d(f, Lx, Ly, lambda kx, ky, a, b: kab(kx, ky) / 2), atol=1e-12)


def _direct_3d(v, L, mult):
    """The same O(N^2) sums for a scalar field on (nz, ny, nx)."""
    nz, ny, nx = v.shape
    (x, kx, qx), (y, ky, qy), (z, kz, qz) = _modes(nx, L[0]), _modes(ny, L[1]), _modes(nz, L[2])
    Ex, Ey, Ez = (np.exp(-1j * np.outer(k, c)) for k, c in ((kx, x), (ky, y), (kz, z)))
    vh = np.einsum("az,by,cx,zyx->abc", Ez, Ey, Ex, v)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    QZ, QY, QX = np.meshgrid(qz, qy, qx, indexing="ij")
    wh = mult(KX, KY, KZ, QX, QY, QZ) * vh
    return np.real(np.einsum("az,by,cx,abc->zyx", Ez.conj(), Ey.conj(), Ex.conj(), wh)) / v.size


def test_bulk_curl_and_biot_savart_operator_equal_direct_fourier_sums():
    nx, ny, nz, L, s = 6, 4, 8, (0.9, 0.6, 1.1), 0.15
    p = BulkProblem(nx, ny, nz, *L, np.ones((nz, ny, nx), np.uint8), n=25.0, rho_out=5.0,
                    waveform=WF, sigma=s)
    v = W.rng(22).standard_normal((3, nz, ny, nx))
    G = lambda kx, ky, kz: np.exp(-(kx * kx + ky * ky + kz * kz) * s * s / 2)
    odd = lambda k, q: np.where(q, 0.0, k)

    def comp(c, smooth, scale):
        # component c of (i k x v_hat) times the scalar factor
        def mult_for(a, b, sign):
            def m(kx, ky, kz, qx, qy, qz):
                ks = (odd(kx, qx), odd(ky, qy), odd(kz, qz))
                f = G(kx, ky, kz) if smooth else 1.0
                return sign * 1j * ks[a] * f * scale(kx, ky, kz)
            return m
        a, b = [(1, 2), (2, 0), (0, 1)][c]
        return (_direct_3d(v[b], L, mult_for(a, b, 1.0)) +
                _direct_3d(v[a], L, mult_for(b, a, -1.0)))

    one = lambda kx, ky, kz: 1.0
    k2 = lambda kx, ky, kz: kx * kx + ky * ky + kz * kz
    inv = lambda kx, ky, kz: np.where(k2(kx, ky, kz) > 0, 1 / np.maximum(k2(kx, ky, kz), 1e-300), 0)
    c, ph = p.curl(v), p.phi(v)
    for i in range(3):
        np.testing.assert_allclose(c[i], comp(i, True, one), atol=1e-12)
        np.testing.assert_allclose(ph[i], comp(i, False, inv), atol=1e-12)


def test_parseval_symmetry_of_film_operators():
    n, L = 16, 1.0
    p = FilmProblem(n, n, L, L, np.ones((n, n), np.uint8), n=19.0, rho_out=1.0, waveform=WF)
    r = W.rng(23)
    a, b = r.standard_normal((n, n)), r.standard_normal((n, n))
    for K in (p.K1, p.K2, p.Kh, p.G):                          # real even multipliers
        assert abs(np.vdot(a, p.apply(K, b)) - np.vdot(p.apply(K, a), b)) < 1e-12 * n * n
    ax, _ = p.gradient(a)
    bx, _ = p.gradient(b)
    _, ay = p.gradient(a)
    _, by = p.gradient(b)
    assert abs(np.vdot(a, bx) + np.vdot(ax, b)) < 1e-12 * n * n   # d/dx is antisymmetric
    assert abs(np.vdot(a, by) + np.vdot(ay, b)) < 1e-12 * n * n


def test_parseval_symmetry_of_bulk_operators():
    n, L = 8, 1.0
    p = BulkProblem(n, n, n, L, L, L, np.ones((n, n, n), np.uint8), n=25.0, rho_out=5.0,
                    waveform=WF)
    r = W.rng(24)
    a, b = r.standard_normal((3, n, n, n)), r.standard_normal((3, n, n, n))
    for op in (p.curl, p.phi):                                  # both are symmetric
        assert abs(np.vdot(a, op(b)) - np.vdot(op(a), b)) < 1e-11 * a.size


def test_film_moment_equals_half_moment_of_sheet_current():
    """m_z = int g dA = 1/2 int (x j_y - y j_x) dA for g vanishing near the box edge (Eq. 2,
    by parts); the Gaussian smoothing keeps both integrals.  A sign error in j flips it."""
    n, L, s = 128, 2.0, 0.15
    p = FilmProblem(n, n, L, L, np.ones((n, n), np.uint8), n=19.0, rho_out=1.0, waveform=WF)
    x = W.cell_centres(n, L)
    X, Y = np.meshgrid(x, x)
    g = np.exp(-((X - 0.2) ** 2 + (Y + 0.1) ** 2) / (2 * s * s)) * (1 + 0.5 * X)
    jx, jy = p.sheet_current(g)
    dA = p.dx * p.dy
    half = 0.5 * (X * jy - Y * jx).sum() * dA
    assert abs(half - p.magnetization(g)) < 1e-9 * abs(p.magnetization(g))


def test_bulk_moment_equals_integral_of_magnetization():
    """1/2 int r x (curl M) dV = int M dV for M vanishing near the box edge: the oracle's moment
    readout of the field h = M must return the integral of M."""
    n, L, s = 32, 1.0, 0.12
    p = BulkProblem(n, n, n, L, L, L, np.ones((n, n, n), np.uint8), n=25.0, rho_out=5.0,
                    waveform=WF)
    c = W.cell_centres(n, L)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    bump = np.exp(-(X ** 2 + (Y - 0.1) ** 2 + (Z + 0.05) ** 2) / (2 * s * s))
    M = np.stack([0.3 * bump, -0.2 * bump * (1 + X), bump * (1 + 0.5 * Y)])
    dV = (2 * L / n) ** 3
    want = M.sum(axis=(1, 2, 3)) * dV
    # summation by parts on the sampled bump holds to ~1e-6 here; a wrong sign or factor of the
    # curl or of the moment is an O(1) error
    np.testing.assert_allclose(p.magnetization(M), want, rtol=1e-5)
