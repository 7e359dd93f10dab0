"""The film right-hand side that allocates nothing (mf_film_rhs_noalloc), through the C ABI.

Some callers cannot allocate device memory (an application whose pool owns every device byte
and forbids cudaMalloc, or a latency-critical loop that must not take an allocation's implicit
device synchronisation).  This entry point runs the same kernel out of a static device array.
Two calls in a row must each match the regular entry point (mf_rhs on a fresh problem, which
also starts its outside iteration cold) within the FP64 tolerance of the other parity tests,
and a grid beyond the static limit must be refused with a clear message.  The file is named
to be collected last.
"""
import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

TOL64 = 1e-9


def _regular(wl, t, g, force):
    p = native.from_workload(wl)
    y = torch.as_tensor(g, device="cuda")
    out = torch.zeros_like(y)
    it, st = p.mf_rhs(t, y, out, force_iters=force, allow_noconv=True)
    return out.cpu().numpy(), it, st


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    wl = W.square_film_128(precision=0)
    p = native.from_workload(wl)                       # parameters only; its workspace is unused
    cases = [(0.2, W.film_state(wl.mask, wl.Lx, wl.Ly, seed=31, amplitude=0.5), 5),
             (0.45, W.film_state(wl.mask, wl.Lx, wl.Ly, seed=32, amplitude=0.3), 0)]
    for t, g, force in cases:
        y = torch.as_tensor(g, device="cuda")
        out = torch.full_like(y, np.nan)
        st, it, msg = native.mf_film_rhs_noalloc(p, t, y, out, force_iters=force)
        ref, it_ref, st_ref = _regular(wl, t, g, force)
        assert st == st_ref and it == it_ref, (st, st_ref, it, it_ref, msg)
        assert rel_l2(out.cpu().numpy(), ref) < TOL64


def test_noalloc_fp32_and_size_limit():
    wl = W.square_film_128(precision=1)
    p = native.from_workload(wl)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=33, amplitude=0.4)
    y = torch.as_tensor(g, device="cuda")
    out = torch.zeros_like(y)
    st, it, _ = native.mf_film_rhs_noalloc(p, 0.3, y, out, force_iters=4)
    ref, it_ref, st_ref = _regular(wl, 0.3, g, 4)
    assert st == st_ref and it == it_ref == 4
    assert rel_l2(out.cpu().numpy(), ref) < TOL64

    big = W.rect_film_2048(precision=1, n_grid=512)
    pb = native.from_workload(big)
    yb = torch.zeros((512, 512), dtype=torch.float64, device="cuda")
    st, _, msg = native.mf_film_rhs_noalloc(pb, 0.1, yb, torch.zeros_like(yb))
    assert st == native.MF_ERR_WORKSPACE and "exceeds the static scratch limit" in msg


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_nonsquare_grid_with_jc_map(precision):
    """A 256 x 128 grid (non-square tables), a lognormal jc map (converted to the transform
    precision inside the static array) and more than 32 knots of h_e: two calls in a row, each
    against the regular entry point and the FP64 oracle."""
    kt = np.linspace(0.0, 1.0, 40)
    wl = film_workload(256, 128, L=(4.0, 2.0), shape="disk", radius=1.5, precision=precision,
                       n=30.0, he_knots=(tuple(kt), tuple(0.5 * kt ** 1.5)))
    wl.jc_map = W.jc_map_lognormal((128, 256), seed=34)
    p = native.from_workload(wl)
    tol = TOL64 if precision == 0 else 2e-4
    for t, seed in ((0.33, 35), (0.71, 36)):
        g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=seed, amplitude=0.6)
        y = torch.as_tensor(g, device="cuda")
        out = torch.full_like(y, np.nan)
        st, it, msg = native.mf_film_rhs_noalloc(p, t, y, out, force_iters=4)
        ref, it_ref, st_ref = _regular(wl, t, g, 4)
        assert st == st_ref and it == it_ref == 4, msg
        assert rel_l2(out.cpu().numpy(), ref) < (TOL64 if precision == 0 else 1e-6)
        want, _, _ = oracle_of(wl).rhs(t, g, None, 4)
        assert rel_l2(out.cpu().numpy(), want) < tol
