"""Failure detection, repeatability and checkpoint/resume through the C ABI.

Faults are made on the host: a NaN written into the state, an iteration limit that cannot be
met.  Nothing here faults or stalls the GPU; every failure comes back as a status code.
"""
import math

import numpy as np
import pytest

import workloads as W
from helpers import film_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _nan_film(**kw):
    wl = film_workload(64, 64, precision=0, ax=1.0, ay=1.0, **kw)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=61, amplitude=0.3)
    g[32, 32] = np.nan
    return wl, g


@pytest.mark.parametrize("dim", [2, 3, "3_bulk_copies"])
def test_barrier_wait_that_runs_out_returns_a_status(dim):
    """A grid-barrier time limit of 1 ns makes the first CTA to reach a barrier give up before
    the others arrive: the launch raises its abort flag, every CTA leaves, and the call returns
    MF_ERR_BARRIER (a bounded wait that returns, not a fault).  With the default limit restored
    the same problem computes the oracle's right-hand side."""
    from helpers import oracle_of
    if dim == 2:
        wl = film_workload(128, 128, precision=0, ax=1.0, ay=1.0)
        y0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=62, amplitude=0.4)
    elif dim == "3_bulk_copies":
        # y and z lines of 256 points: their gathers are bulk copies on an mbarrier, whose
        # waits give up at the same limit and then drain the copies before the CTA leaves
        m = W.bulk_mask(16, 256, 256, 0.5, 2.0, 2.0, "box", ax=0.3, ay=1.0, az=1.0)
        wl = W.Workload("box_16x256x256", 3, 16, 256, 256, 0.5, 2.0, 2.0, m, n=25.0, rho_out=5.0,
                        precision=0, t0=0.0, t1=1.0, he_knots=((0.0, 1.0), (0.0, 0.5)), iter_tol=1e-4)
        y0 = W.bulk_state(m, (0.5, 2.0, 2.0), seed=64, h0=0.3, depth=0.3)
    else:
        m = W.bulk_mask(32, 32, 32, 1.0, 1.0, 1.0, "box", ax=0.5, ay=0.5, az=0.5)
        wl = W.Workload("cube32", 3, 32, 32, 32, 1.0, 1.0, 1.0, m, n=25.0, rho_out=5.0, precision=0,
                        t0=0.0, t1=1.0, he_knots=((0.0, 1.0), (0.0, 0.5)), iter_tol=1e-4)
        y0 = W.bulk_state(m, (1.0, 1.0, 1.0), seed=63)
    p = native.from_workload(wl)
    assert p.mf_get_info()["grid"] > 1
    y = dev(y0)
    out = torch.zeros_like(y)
    p.mf_set_barrier_timeout(1e-9)
    with pytest.raises(native.MFError) as e:
        p.mf_rhs(0.2, y, out, force_iters=3)
    assert e.value.status == native.MF_ERR_BARRIER
    with pytest.raises(native.MFError) as e:
        p.mf_advance(0.5, max_attempts=2)
    assert e.value.status == native.MF_ERR_BARRIER
    p.mf_set_barrier_timeout(0.0)                       # back to the default limit
    p.mf_reset_warm()
    it, st = p.mf_rhs(0.2, y, out, force_iters=3, allow_noconv=True)
    ref, it_o, _ = oracle_of(wl).rhs(0.2, y0, None, 3)
    assert it == it_o == 3
    err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-9, err


def test_nan_state_is_rejected_until_step_underflow():
    """The outside iteration cannot converge on a NaN state: every attempt is rejected (outcome
    2) and halves h, until h < h_min ends the run with MF_ERR_STEP_UNDERFLOW.  The state is
    never replaced."""
    wl, g = _nan_film(iter_max=3)
    p = native.from_workload(wl)
    p.mf_set_state(0.1, dev(g), h=1e-3)
    with pytest.raises(native.MFError) as e:
        p.mf_advance(0.2)
    assert e.value.status == native.MF_ERR_STEP_UNDERFLOW
    info = p.mf_get_info()
    halvings = math.ceil(math.log2(1e-3 / 1e-12))         # h_min = 1e-12
    assert info["n_attempts"] == info["n_rejected"] == info["n_noconv"] == halvings
    assert info["n_accepted"] == 0 and info["n_rhs"] == halvings
    assert all(e[3] == 2 and e[4][0] == 3 for e in p.mf_get_log())
    y = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    t, h = p.mf_get_state(y)
    assert t == 0.1 and h < 1e-12
    np.testing.assert_array_equal(y.cpu().numpy(), g)


def test_nan_state_with_fixed_iterations_is_nonfinite():
    """With a fixed iteration count (no stop test) the NaN reaches the derivative: mf_rhs and
    mf_advance return MF_ERR_NONFINITE, and the integrator stops before its first attempt."""
    wl, g = _nan_film(iter_max=3, iter_tol=0.0)
    p = native.from_workload(wl)
    out = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(native.MFError) as e:
        p.mf_rhs(0.1, dev(g), out)
    assert e.value.status == native.MF_ERR_NONFINITE
    p.mf_set_state(0.1, dev(g), h=1e-3)
    with pytest.raises(native.MFError) as e:
        p.mf_advance(0.2)
    assert e.value.status == native.MF_ERR_NONFINITE
    info = p.mf_get_info()
    assert info["n_attempts"] == 0 and info["n_rhs"] == 2 and info["t"] == 0.1


@pytest.mark.parametrize("precision", [0, 1])
def test_repeat_runs_are_bitwise_identical(precision):
    """Fixed-order reductions, no float atomics: two problems built alike give the same bits."""
    wl = W.square_film_128(precision=precision)
    runs = []
    for _ in range(2):
        p = native.from_workload(wl)
        p.mf_set_state(0.0, None, h=1e-3)
        p.mf_advance(0.3)
        y = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
        p.mf_get_state(y)
        runs.append((y, p.mf_get_log(), p.mf_get_info()["n_iters"]))
    assert torch.equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1] and runs[0][2] == runs[1][2]


def _run_on(p, t, n):
    p.mf_advance(t)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    p.mf_get_state(y)
    i = p.mf_get_info()
    return y, p.mf_get_log(), (i["n_attempts"], i["n_rhs"], i["n_iters"], i["t"], i["h"])


@pytest.mark.parametrize("case,where", [("film_fp32", "device"), ("film_fp32", "host"),
                                        ("cube_fp64", "device")])
def test_checkpoint_resume_is_exact(case, where):
    """A checkpoint taken mid-ramp and restored into a fresh problem (and into the same one)
    continues bit for bit like the original: warm start, first-same-as-last derivative, step
    size, counters and log included."""
    if case == "film_fp32":
        wl, t_mid, t_end = W.square_film_128(precision=1), 0.3, 0.6
        n = 128 * 128
    else:
        wl, t_mid, t_end = W.cube_bulk(16, precision=0), 0.2, 0.6   # through the knot at 0.5
        n = 3 * 16 ** 3
    p = native.from_workload(wl)
    p.mf_set_state(0.0, None, h=1e-3)
    p.mf_advance(t_mid)
    blob = torch.empty(native.load().mf_checkpoint_bytes(p.h), dtype=torch.uint8,
                       device="cuda" if where == "device" else "cpu")
    p.mf_checkpoint_save(blob)
    ya, la, ca = _run_on(p, t_end, n)
    q = native.from_workload(wl)
    q.mf_checkpoint_restore(blob)
    yb, lb, cb = _run_on(q, t_end, n)
    assert torch.equal(ya, yb) and la == lb and ca == cb
    p.mf_checkpoint_restore(blob)
    yc, lc, cc = _run_on(p, t_end, n)
    assert torch.equal(ya, yc) and la == lc and ca == cc


def test_checkpoint_of_another_grid_is_refused():
    a = native.from_workload(W.square_film_128(precision=1))
    b = native.from_workload(film_workload(64, 64, precision=1))
    blob = a.mf_checkpoint_save()
    y0 = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    b.mf_get_state(y0)
    with pytest.raises(native.MFError) as e:
        b.mf_checkpoint_restore(blob)
    assert e.value.status == native.MF_ERR_ARG
    y1 = torch.zeros_like(y0)
    b.mf_get_state(y1)
    assert torch.equal(y0, y1)
