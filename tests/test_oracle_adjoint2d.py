"""Pins of the film-solve adjoint oracle: consistency with the forward oracle, the dot-product
test of the transposed outside iteration, and central finite differences of the map."""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint2d import FilmAdjoint
from oracle.film2d import FilmProblem
from oracle.waveform import Waveform

N, L = 32, 2.0
KT, KV = [0.0, 0.5, 1.0], [0.0, 0.3, 0.45]


def _setup(n_power=19.0, iters=4, seed=31, amplitude=1.6, gamma=1.0):
    # amplitude 1.6 on this grid puts |j| just below jc (the smoothing rounds the critical-state
    # slope), where the power law is sensitive to jc
    mask = W.film_mask(N, N, L, L, "rect", ax=1.0, ay=0.75)
    jc = W.jc_map_lognormal((N, N), seed=seed, sigma=0.05)
    p = FilmProblem(N, N, L, L, mask, n=n_power, rho_out=1.0, waveform=Waveform(KT, KV), jc=jc,
                    iter_tol=0.0, iter_max=iters, gamma=gamma)
    g0 = W.film_state(mask, L, L, seed=seed, amplitude=amplitude)
    return p, FilmAdjoint(p, iters), g0, np.array(p.jc)


@pytest.mark.parametrize("gamma", [1.0, 1.6])
def test_forward_rhs_equals_the_film_oracle(gamma):
    """Cold start and a fixed iteration count: the adjoint's f is FilmProblem.rhs (with the
    elliptic law too)."""
    p, a, g0, jc = _setup(gamma=gamma)
    s = p.wf.hedot(0.2)
    ref, it, _ = p.rhs(0.2, g0, None, a.I)
    got, _ = a.rhs(g0, jc, s)
    assert it == a.I
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_transposed_outside_iteration_dot_product():
    p, a, _, _ = _setup(iters=5)
    r = W.rng(32)
    hin = np.where(p.conductor, r.standard_normal((N, N)), 0.0)
    s = 0.37
    v = r.standard_normal((N, N))
    hb, sb = a.P_T(v)
    lhs = float((a.P(hin, s) * v).sum())
    rhs = float((hin * hb).sum()) + s * sb
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def _fd(fun, x, d, eps):
    return (fun(x + eps * d) - fun(x - eps * d)) / (2 * eps)


@pytest.mark.parametrize("gamma", [1.0, 1.6])
def test_rhs_vjp_matches_finite_differences(gamma):
    p, a, g0, jc = _setup(gamma=gamma)
    r = W.rng(33)
    s = 0.3
    v = r.standard_normal((N, N))
    _, tape = a.rhs(g0, jc, s)
    gb, cb, sb = a.rhs_vjp(tape, jc, v)
    dg = np.where(p.conductor, r.standard_normal((N, N)), 0.0)
    dc = np.where(p.sc, r.standard_normal((N, N)), 0.0)
    fg = _fd(lambda x: float((a.rhs(x, jc, s)[0] * v).sum()), g0, dg, 1e-6)
    fc = _fd(lambda x: float((a.rhs(g0, x, s)[0] * v).sum()), jc, dc, 1e-6)
    fs = _fd(lambda x: float((a.rhs(g0, jc, x)[0] * v).sum()), s, 1.0, 1e-6)
    assert abs(fg - (gb * dg).sum()) < 1e-6 * abs(fg)
    assert abs(fc - (cb * dc).sum()) < 1e-6 * abs(fc)
    assert abs(fs - sb) < 1e-6 * abs(fs)


def test_warm_chain_equals_the_film_oracle():
    """Calls in a row, each from the previous call's last iterate with its own count: the
    adjoint's forward is FilmProblem.rhs called the same way (its most recent call's warm start)."""
    p, a, g0, jc = _setup()
    p.reset_warm()
    warm = None
    r = W.rng(35)
    for t, it in ((0.2, 3), (0.21, 1), (0.23, 5)):
        g = g0 + 0.01 * np.where(p.conductor, r.standard_normal((N, N)), 0.0)
        s = p.wf.hedot(t)
        ref, it_o, _ = p.rhs(t, g, None, it)
        w = np.full((N, N), s) if warm is None else warm
        got, warm, _ = a.call(g, jc, s, w, it)
        assert it_o == it
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        np.testing.assert_allclose(warm, p.warm, rtol=0, atol=1e-13 * np.abs(p.warm).max())


def test_warm_outside_iteration_dot_product():
    """<P(h_in, s, w), (v, omega)> = <h_in, hbar> + s sbar + <w, wbar> for all three inputs and
    both outputs (g_dot on the conductor, last iterate on free space)."""
    p, a, _, _ = _setup()
    r = W.rng(36)
    out = p.out.astype(float)
    for iters in (1, 2, 6):
        hin = np.where(p.conductor, r.standard_normal((N, N)), 0.0)
        w = out * r.standard_normal((N, N))
        s = 0.41
        v = r.standard_normal((N, N))
        om = out * r.standard_normal((N, N))
        gd, last = a.P_warm(hin, s, w, iters)
        hb, sb, wb = a.P_T_warm(v, om, iters)
        lhs = float((gd * v).sum() + (last * om).sum())
        rhs = float((hin * hb).sum() + s * sb + (w * wb).sum())
        assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0), (iters, lhs, rhs)
        assert np.all(wb[p.conductor] == 0.0) and np.all(hb[p.out] == 0.0)


def test_call_vjp_matches_finite_differences_with_warm_start():
    p, a, g0, jc = _setup()
    r = W.rng(37)
    s, it = 0.3, 3
    out = p.out.astype(float)
    w0 = out * (0.2 + 0.05 * r.standard_normal((N, N)))
    v = r.standard_normal((N, N))
    om = out * r.standard_normal((N, N))

    def J(g, c, s_, w):
        gd, last, _ = a.call(g, c, s_, w, it)
        return float((gd * v).sum() + (last * om).sum())
    _, _, tape = a.call(g0, jc, s, w0, it)
    gb, cb, sb, wb = a.call_vjp(tape, jc, it, v, om)
    dg = np.where(p.conductor, r.standard_normal((N, N)), 0.0)
    dc = np.where(p.sc, r.standard_normal((N, N)), 0.0)
    dw = out * r.standard_normal((N, N))
    fg = _fd(lambda x: J(x, jc, s, w0), g0, dg, 1e-6)
    fc = _fd(lambda x: J(g0, x, s, w0), jc, dc, 1e-6)
    fs = _fd(lambda x: J(g0, jc, x, w0), s, 1.0, 1e-6)
    fw = _fd(lambda x: J(g0, jc, s, x), w0, dw, 1e-6)
    assert abs(fg - (gb * dg).sum()) < 1e-6 * abs(fg)
    assert abs(fc - (cb * dc).sum()) < 1e-6 * abs(fc)
    assert abs(fs - sb) < 1e-6 * abs(fs)
    assert abs(fw - (wb * dw).sum()) < 1e-6 * abs(fw)


STEPS = [(0.1 + 0.002 * i, 0.002) for i in range(6)]
ITERS = [4, 2, 3, 1, 2, 2, 3, 1, 1, 2, 3, 2, 1, 1, 2, 2, 2, 3]


def check_solve_gradient(a, p, g0, jc, warm0=None):
    target = W.rng(34).standard_normal((N, N)) * 0.01
    Lv, cb, vb, wb = a.gradient(g0, jc, KT, KV, STEPS, target, ITERS, warm0)
    assert Lv == pytest.approx(a.loss(g0, jc, KT, KV, STEPS, target, ITERS, warm0), rel=1e-14)
    kv = np.array(KV)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        fd = _fd(lambda x: a.loss(g0, jc, KT, x, STEPS, target, ITERS, warm0), kv, e, 1e-5)
        assert abs(fd - vb[k]) <= 1e-6 * max(abs(fd), 1e-12) + 1e-14, (k, fd, vb[k])
    # the most sensitive cell and cells across the film (edge, core, corner)
    film = np.argwhere(p.sc)
    picks = [np.unravel_index(np.argmax(np.abs(cb)), cb.shape)]
    picks += [tuple(film[i]) for i in (0, len(film) // 3, len(film) // 2, -1)]
    scale = np.abs(cb).max()
    assert scale > 1e-4
    for iy, ix in picks:
        e = np.zeros((N, N))
        e[iy, ix] = 1.0
        fd = _fd(lambda x: a.loss(g0, x, KT, KV, STEPS, target, ITERS, warm0), jc, e, 1e-5)
        assert abs(fd - cb[iy, ix]) <= 1e-6 * abs(fd) + 1e-8 * scale, (iy, ix, fd, cb[iy, ix])
    assert np.all(cb[~p.sc] == 0.0)
    if warm0 is not None:
        dw = p.out * W.rng(38).standard_normal((N, N))
        fd = _fd(lambda x: a.loss(g0, jc, KT, KV, STEPS, target, ITERS, x), warm0, dw, 1e-5)
        assert abs(fd - (wb * dw).sum()) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("n_power", [1.0, 19.0])
def test_solve_gradient_matches_finite_differences(n_power):
    """dL/djc and dL/dv of the frozen-step, frozen-count solve (warm start carried from call to
    call, cold first call) against central differences of L, for the Ohmic sheet (rho = 1/jc)
    and a power-law film in a near-critical state."""
    p, a, g0, jc = _setup(n_power=n_power)
    check_solve_gradient(a, p, g0, jc)


def test_solve_gradient_with_a_given_first_warm_start():
    p, a, g0, jc = _setup()
    warm0 = p.out * (0.25 + 0.05 * W.rng(39).standard_normal((N, N)))
    check_solve_gradient(a, p, g0, jc, warm0)


class WarmCouplingDropped(FilmAdjoint):
    """A planted mistake: the warm start treated as a constant of every call."""
    def call_vjp(self, tape, jc, iters, v, wbar):
        gb, cb, sb, wb = super().call_vjp(tape, jc, iters, v, None)
        return gb, cb, sb, np.zeros_like(wb)


def test_planted_warm_coupling_mistake_is_caught():
    p, _, g0, jc = _setup()
    with pytest.raises(AssertionError):
        check_solve_gradient(WarmCouplingDropped(p, 4), p, g0, jc)


def test_checkpointed_reverse_sweep_gives_the_same_gradient():
    p, a, g0, jc = _setup()
    target = W.rng(40).standard_normal((N, N)) * 0.01
    full = a.gradient(g0, jc, KT, KV, STEPS, target, ITERS)
    for C in (1, 2, 4):
        ck = a.gradient(g0, jc, KT, KV, STEPS, target, ITERS, ckpt_every=C)
        assert ck[0] == full[0]
        np.testing.assert_array_equal(ck[1], full[1])
        np.testing.assert_array_equal(ck[2], full[2])
