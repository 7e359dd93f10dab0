"""mf_advance_batch: films advanced together in one shared persistent launch (each on its own
range of CTAs) give exactly the states of the same films advanced one at a time: the items and
the order of every reduction do not depend on how many CTAs run a film."""
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


def _check_equal_to_one_at_a_time(wls, t_end, streams=True):
    batch = [native.from_workload(wl, stream=torch.cuda.Stream() if streams else None) for wl in wls]
    for p in batch:
        p.mf_set_state(0.0, None, h=1e-3)
    st = native.advance_batch(batch, t_end)
    assert st == [0] * len(wls)
    for wl, pb, te in zip(wls, batch, t_end):
        ps = native.from_workload(wl)
        ps.mf_set_state(0.0, None, h=1e-3)
        ps.mf_advance(te)
        n = wl.nx * wl.ny * wl.nz * (3 if wl.dim == 3 else 1)
        tb, hb, yb = _state(pb, n)
        ts, hs, ys = _state(ps, n)
        assert tb == ts == pytest.approx(te, abs=1e-12)
        assert hb == hs
        assert torch.equal(yb, ys)
        ib, is_ = pb.mf_get_info(), ps.mf_get_info()
        for k in ("n_attempts", "n_rhs", "n_iters"):
            assert ib[k] == is_[k], k


def test_batch_equals_one_at_a_time():
    _check_equal_to_one_at_a_time(W.film_batch(4, seed=7, max_side=96, precision=1),
                                  [0.05, 0.08, 0.05, 0.1])


@pytest.mark.parametrize("streams", [False, True])
def test_mixed_batch_equals_one_at_a_time(streams):
    """Films of both precisions (shared launches per precision), a 1024^2 film whose own launch
    fills the GPU (launched alone) and a bulk cube (its own launch) in one call: each equals its
    one-at-a-time run."""
    films = W.film_batch(5, seed=9, max_side=160, precision=1)
    films[1].precision = 0
    films[3].precision = 0
    big = W.rect_film_2048(precision=1, n_grid=1024)
    cube = W.cube_bulk(16, precision=1)
    _check_equal_to_one_at_a_time([big] + films + [cube], [0.005, 0.04, 0.03, 0.05, 0.03, 0.04, 0.02],
                                  streams=streams)


def test_many_small_films_one_launch():
    """40 films of 64..128 cells (grids 128^2 and 256^2): more films than fit one CTA range each
    at their own launch widths, so every film runs on fewer CTAs than alone."""
    wls = W.film_batch(40, seed=11, max_side=128, precision=1)
    _check_equal_to_one_at_a_time(wls, [0.02] * len(wls), streams=False)


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


def test_batch_refuses_a_repeated_problem_and_runs_nothing():
    """The same problem twice in one call would run twice at once on one workspace: refused with
    MF_ERR_ARG before any work (the problem's state is untouched); no problems: nothing to do."""
    wl = W.film_batch(1, seed=8, max_side=64, precision=1)[0]
    p = native.from_workload(wl)
    p.mf_set_state(0.0, None, h=1e-3)
    with pytest.raises(native.MFError) as e:
        native.advance_batch([p, p], [0.02, 0.02])
    assert e.value.status == native.MF_ERR_ARG
    t, h, _ = _state(p, wl.nx * wl.ny)
    assert (t, h) == (0.0, 1e-3) and p.mf_get_info()["n_attempts"] == 0
    assert native.advance_batch([], []) == []
