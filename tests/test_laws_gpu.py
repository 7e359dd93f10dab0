"""The other current-voltage laws on the GPU against the FP64 oracle, through the C ABI.

The conclusion of the paper names anisotropic and field-dependent relations as replacements for
the power law in the same method of lines.  The library carries two of them (mf_params.gamma,
mf_params.b0), both acting in the superconductor:
  * the elliptic power law e = rho(s) A j, s^2 = j^T A j, A = diag(1, 1/gamma^2) for a film and
    diag(1, 1, 1/gamma^2) for a bulk body;
  * the Kim-type critical current jc / (1 + |h| / b0) of a bulk body, |h| the stage field.
Checked here: the electric-field readout, right-hand sides with forced and converged outside
iterations, lock-step film and bulk ramps, and the film's vector-Jacobian
product with the elliptic law (the oracle's pins of these laws are in test_oracle_laws.py and
test_oracle_adjoint2d.py).
"""
import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of, rel_l2
from oracle.adjoint2d import FilmAdjoint
from oracle.bs23 import BS23, LogEntry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

TOL64 = 1e-9
TOL32 = 2e-4


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _film(precision, gamma=1.7):
    wl = film_workload(256, 64, L=(4.0, 1.0), shape="disk", radius=0.8, hole=(0.3, 0.1, 0.25),
                       n=30.0, rho_out=5.0, precision=precision, gamma=gamma)
    wl.jc_map = W.jc_map_lognormal((64, 256), seed=9)
    return wl


def _bulk(precision, gamma=2.0, b0=0.3, nn=32):
    m = W.bulk_mask(nn, nn, nn, 1.0, 1.0, 1.0, "box", ax=0.5, ay=0.4, az=0.3)
    wl = W.Workload(f"bulk_law_{nn}", 3, nn, nn, nn, 1.0, 1.0, 1.0, m, n=25.0, rho_out=5.0,
                    precision=precision, t0=0.0, t1=1.0, he_knots=((0.0, 0.5, 1.0), (0.0, 0.25, 0.25)),
                    iter_tol=1e-4, gamma=gamma, b0=b0, vector_he=(0.3, 0.0, 1.0))
    wl.jc_map = W.jc_map_lognormal((nn, nn, nn), seed=19)
    return wl


@pytest.mark.parametrize("precision", [0, 1])
def test_film_elliptic_law_electric_field_readout(precision):
    wl = _film(precision)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=31, amplitude=0.8)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((2, wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_E, out=out, t=0.3, y=dev(g))
    ex, ey = o.electric_field(*o.sheet_current(g))
    iso = oracle_of(wl, gamma=1.0).electric_field(*o.sheet_current(g))
    assert rel_l2(np.stack([ex, ey]), np.stack(iso)) > 0.1          # the law is not the isotropic one
    err = rel_l2(out.cpu().numpy(), np.stack([ex, ey]))
    assert err < (TOL64 if precision == 0 else TOL32), err


@pytest.mark.parametrize("precision", [0, 1])
def test_bulk_elliptic_and_kim_laws_electric_field_readout(precision):
    wl = _bulk(precision)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=20, h0=0.3, depth=0.3)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((3, wl.nz, wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_E, out=out, t=0.1, y=dev(h))
    ref = o.electric_field(o.current(h), h)
    assert rel_l2(ref, oracle_of(wl, gamma=1.0).electric_field(o.current(h), h)) > 0.1
    assert rel_l2(ref, o.electric_field(o.current(h), 0.0 * h)) > 0.1
    err = rel_l2(out.cpu().numpy(), ref)
    assert err < (TOL64 if precision == 0 else TOL32), err


def _rhs_pair(wl, y0, times, force, tol):
    o = oracle_of(wl)
    p = native.from_workload(wl)
    y = dev(y0)
    out = torch.zeros_like(y)
    for t in times:
        ref, it_o, st_o = o.rhs(t, y0, None, force)
        it_g, st_g = p.mf_rhs(t, y, out, force_iters=force or 0, allow_noconv=True)
        assert (it_g, st_g) == (it_o, st_o), (t, it_g, it_o, st_g, st_o)
        err = rel_l2(out.cpu().numpy(), ref)
        assert err < tol, (t, err)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32)])
def test_film_elliptic_law_rhs(precision, tol):
    wl = _film(precision)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=32, amplitude=0.9)
    _rhs_pair(wl, g, [0.2, 0.6], 4, tol)
    if precision == 0:
        _rhs_pair(wl, g, [0.2, 0.2 + 1e-3, 0.6], None, tol)      # converged, warm-started


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32)])
def test_bulk_elliptic_and_kim_laws_rhs(precision, tol):
    wl = _bulk(precision)
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=41, h0=0.3, depth=0.3)
    _rhs_pair(wl, h, [0.1, 0.3], 3, tol)
    if precision == 0:
        _rhs_pair(wl, h, [0.1, 0.1 + 1e-3, 0.7], None, tol)


def test_film_elliptic_law_ramp_lock_step():
    """A 64^2 film in a 128^2 grid with gamma = 1.5, n = 19, h_e 0 -> 0.5 on [0, 0.5]: the GPU's
    ramp replayed by the oracle with the GPU's steps, decisions and iteration counts."""
    wl = W.square_film_128(precision=0)
    wl.gamma, wl.t1 = 1.5, 0.5
    wl.he_knots = ((0.0, 0.5), (0.0, 0.5))
    p = native.from_workload(wl)
    m, hz = p.mf_run_ramp(np.array([0.25, 0.5]), want_fields=True)
    log = p.mf_get_log()
    o = oracle_of(wl)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    s.start(wl.t0, np.zeros((128, 128)), wl.t1)
    s.replay([LogEntry(*e) for e in log])
    assert s.t == pytest.approx(0.5, abs=1e-14)
    g = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    p.mf_get_state(g)
    assert rel_l2(g.cpu().numpy(), s.y) < 1e-6
    assert m[-1, 0] == pytest.approx(o.magnetization(s.y), rel=1e-6)
    # the anisotropy shows: the sheet current along y is gamma times stronger at the x edges
    jx, jy = o.sheet_current(s.y)
    assert np.abs(jy).max() > 1.3 * np.abs(jx).max()


def test_bulk_kim_law_ramp_lock_step():
    """A box in a 32^3 grid with the elliptic and Kim laws through the ramp knot at t = 0.5: the
    GPU's ramp replayed by the oracle with the GPU's steps, decisions and iteration counts."""
    wl = _bulk(0, nn=32)
    t_out = np.array([0.25, 0.55])
    p = native.from_workload(wl)
    m, j = p.mf_run_ramp(t_out, want_fields=True)
    log = p.mf_get_log()
    o = oracle_of(wl)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol)
    s.start(0.0, np.zeros((3, 32, 32, 32)), 1.0)
    s.replay([LogEntry(*e) for e in log])
    assert s.t == pytest.approx(0.55, abs=1e-14)
    y = torch.zeros((3, 32, 32, 32), dtype=torch.float64, device="cuda")
    p.mf_get_state(y)
    assert rel_l2(y.cpu().numpy(), s.y) < 1e-6
    np.testing.assert_allclose(m[-1], o.magnetization(s.y), rtol=1e-6, atol=1e-12)
    assert rel_l2(j[-1].cpu().numpy().reshape(3, 32, 32, 32), o.current(s.y)) < 1e-6


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 2e-4)])
def test_film_elliptic_law_rhs_vjp(precision, tol):
    wl = W.square_film_128(precision=precision)
    wl.gamma = 1.6
    wl.jc_map = W.jc_map_lognormal((wl.ny, wl.nx), seed=44, sigma=0.05)
    o = oracle_of(wl)
    iters = 4
    adj = FilmAdjoint(o, iters)
    jc = np.array(o.jc)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=45, amplitude=1.0)
    v = W.rng(46).standard_normal((wl.ny, wl.nx))
    _, tape = adj.rhs(g, jc, 0.3)
    gb_ref, cb_ref, sb_ref = adj.rhs_vjp(tape, jc, v)
    p = native.from_workload(wl)
    gb, cb, sb = p.mf_film_rhs_vjp(dev(g), dev(v), iters)
    assert rel_l2(gb.cpu().numpy(), gb_ref) < tol
    assert rel_l2(cb.cpu().numpy(), cb_ref) < tol
    assert abs(sb - sb_ref) <= tol * abs(sb_ref)
