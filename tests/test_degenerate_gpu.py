"""Degenerate inputs of the method on the GPU, through the C ABI: a film or a body without any
superconductor.

With an empty Omega nothing carries current.  The film's right-hand side (Eqs. 10-12, the return
value zero outside the film) is then exactly 0 for any g; the bulk iteration (Eq. 18) ends at
h_dot = h_e_dot on all of D, because the update only adds the field of currents in Omega.  A bulk
ramp from h = 0 therefore follows h(t) = h_e(t) z exactly, and both moments stay 0.  The FP64
oracle gives the same values and iteration counts.
"""
import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("precision", [0, 1])
def test_film_without_conductor(precision):
    wl = film_workload(64, 64, precision=precision)
    wl.mask = np.zeros((64, 64), np.uint8)
    g = 0.01 * np.random.default_rng(1).standard_normal((64, 64))
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.full((64, 64), 7.0, dtype=torch.float64, device="cuda")
    for t in (0.1, 0.3):
        ref, it_o, st_o = o.rhs(t, g)
        it, st = p.mf_rhs(t, dev(g), out)
        assert (it, st) == (it_o, st_o) and not ref.any()
        assert not out.cpu().numpy().any()
    q = native.from_workload(wl)
    m, hz = q.mf_run_ramp(np.array([0.5, 1.0]), want_fields=True)
    assert not m.any()
    info = q.mf_get_info()
    assert info["t"] == 1.0 and info["n_noconv"] == 0
    # h_z = h_e + the field of the (absent) currents
    np.testing.assert_allclose(hz.cpu().numpy(), [[0.25] * 4096, [0.5] * 4096], rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_bulk_without_conductor(precision):
    wl = W.Workload("empty_bulk_16", 3, 16, 16, 16, 1.0, 1.0, 1.0, np.zeros((16, 16, 16), np.uint8),
                    n=25.0, rho_out=5.0, precision=precision, t0=0.0, t1=1.0,
                    he_knots=((0.0, 0.5, 1.0), (0.0, 0.25, 0.25)), iter_tol=1e-4)
    h = 0.01 * np.random.default_rng(2).standard_normal((3, 16, 16, 16))
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((3, 16, 16, 16), dtype=torch.float64, device="cuda")
    for t, he_dot in ((0.1, 0.5), (0.7, 0.0)):          # on the ramp, then past the knot
        ref, it_o, st_o = o.rhs(t, h)
        it, st = p.mf_rhs(t, dev(h), out)
        assert (it, st) == (it_o, st_o)
        np.testing.assert_allclose(ref[2], he_dot, rtol=0, atol=1e-15)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[2], he_dot, rtol=0, atol=1e-12)
        np.testing.assert_allclose(got[:2], 0.0, rtol=0, atol=1e-12)
    q = native.from_workload(wl)
    m, j = q.mf_run_ramp(np.array([0.25, 1.0]), want_fields=True)
    assert not m.any()                                   # a sum over the (empty) conductor
    # j = curl of a uniform field: zero up to the transforms' rounding
    np.testing.assert_allclose(j.cpu().numpy(), 0.0, rtol=0, atol=1e-12 if precision == 0 else 2e-5)
    y = torch.zeros((3, 16, 16, 16), dtype=torch.float64, device="cuda")
    q.mf_get_state(y)
    y = y.cpu().numpy()
    np.testing.assert_allclose(y[2], 0.25, rtol=0, atol=1e-12)
    np.testing.assert_allclose(y[:2], 0.0, rtol=0, atol=1e-12)
