"""mf_advance_batch: several films advanced together on their own streams give exactly the
states of the same films advanced one at a time (the kernels are deterministic)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402


def _state(p, n):
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t, h = p.mf_get_state(y)
    return t, h, y


def test_batch_equals_one_at_a_time():
    wls = W.film_batch(4, seed=7, max_side=96, precision=1)
    t_end = [0.05, 0.08, 0.05, 0.1]
    batch = [native.from_workload(wl, stream=torch.cuda.Stream()) for wl in wls]
    for p in batch:
        p.mf_set_state(0.0, None, h=1e-3)
    st = native.advance_batch(batch, t_end)
    assert st == [0] * len(wls)
    for wl, pb, te in zip(wls, batch, t_end):
        ps = native.from_workload(wl)
        ps.mf_set_state(0.0, None, h=1e-3)
        ps.mf_advance(te)
        n = wl.nx * wl.ny
        tb, hb, yb = _state(pb, n)
        ts, hs, ys = _state(ps, n)
        assert tb == ts == pytest.approx(te, abs=1e-12)
        assert hb == hs
        assert torch.equal(yb, ys)
        ib, is_ = pb.mf_get_info(), ps.mf_get_info()
        for k in ("n_attempts", "n_rhs", "n_iters"):
            assert ib[k] == is_[k], k


def test_batch_reports_each_status():
    # a problem whose outside iteration cannot converge (impossible tolerance, one iteration)
    # fails with step underflow; the other problem of the batch still completes
    wls = W.film_batch(2, seed=8, max_side=64, precision=1)
    good = native.from_workload(wls[0], stream=torch.cuda.Stream())
    bad = native.from_workload(wls[1], stream=torch.cuda.Stream(), iter_tol=1e-30, iter_max=1)
    for p in (good, bad):
        p.mf_set_state(0.0, None, h=1e-3)
    with pytest.raises(native.MFError):
        native.advance_batch([good, bad], [0.02, 0.02], max_attempts=200)
    t, _, _ = _state(good, wls[0].nx * wls[0].ny)
    assert t == pytest.approx(0.02, abs=1e-12)
