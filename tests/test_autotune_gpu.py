"""mf_autotune: the chosen work-item shape and launch width is one the kernels accept, the state
is kept, and the tuned problem still matches the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

BATCH = 4096


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _valid_shape(wl, tu):
    rb, zs = tu["rows_per_item"], tu["zs_per_item"]
    assert rb >= 2 and rb & (rb - 1) == 0 and wl.ny % rb == 0
    if wl.dim == 2:
        assert rb <= 2 * BATCH // wl.nx
    else:
        assert 3 * wl.nx * (rb // 2) <= BATCH and 3 * wl.ny * zs <= BATCH and zs <= wl.nz
    assert tu["grid"] >= 1 and tu["candidates"] >= 2
    assert 0 < tu["ms_per_rhs"] <= tu["ms_per_rhs_default"]


@pytest.mark.parametrize("case", ["film_256_fp64", "film_512x128_fp32", "cube_32_fp64"])
def test_tuned_problem_matches_oracle(case):
    if case == "film_256_fp64":
        wl = film_workload(256, 256, precision=0, ax=1.0, ay=0.6)
        y0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=51, amplitude=0.4)
        tol = 1e-9
    elif case == "film_512x128_fp32":
        wl = film_workload(512, 128, L=(4.0, 1.0), precision=1, ax=3.0, ay=0.5)
        y0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=52, amplitude=0.4)
        tol = 2e-4
    else:
        wl = W.cube_bulk(32, precision=0)
        y0 = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=53)
        tol = 1e-9
    p = native.from_workload(wl)
    p.mf_set_state(0.15, dev(y0), h=2e-3)
    before = p.mf_get_info()
    tu = p.mf_autotune(reps=2, force_iters=2)
    _valid_shape(wl, tu)
    info = p.mf_get_info()
    assert info["rows_per_item"] == tu["rows_per_item"] and info["grid"] == tu["grid"]
    # state, step size and counters kept
    y = torch.zeros_like(dev(y0))
    t, h = p.mf_get_state(y)
    assert (t, h) == (0.15, 2e-3)
    assert torch.equal(y, dev(y0))
    for k in ("n_rhs", "n_iters", "n_attempts"):
        assert info[k] == before[k], k
    # the tuned configuration against the oracle, starting cold like a fresh oracle
    o = oracle_of(wl)
    out = torch.zeros_like(y)
    for t_eval in (0.15, 0.2):
        ref, it_o, st_o = o.rhs(t_eval, y0, None, 4)
        it_g, st_g = p.mf_rhs(t_eval, y, out, force_iters=4, allow_noconv=True)
        assert (it_g, st_g) == (it_o, st_o)
        assert rel_l2(out.cpu().numpy(), ref) < tol


def test_tuned_advance_matches_untuned():
    """The item shape changes only the order of the sums: an FP64 film advanced after tuning
    agrees with the untuned one to rounding, step for step."""
    wl = film_workload(256, 256, precision=0, ax=1.0, ay=1.0)
    a, b = native.from_workload(wl), native.from_workload(wl)
    for p in (a, b):
        p.mf_set_state(0.0, None, h=1e-3)
    a.mf_autotune(reps=1, force_iters=1)
    a.mf_advance(0.05)
    b.mf_advance(0.05)
    ya = torch.zeros((256, 256), dtype=torch.float64, device="cuda")
    yb = torch.zeros_like(ya)
    ta, _ = a.mf_get_state(ya)
    tb, _ = b.mf_get_state(yb)
    assert ta == tb == pytest.approx(0.05, abs=1e-12)
    ia, ib = a.mf_get_info(), b.mf_get_info()
    assert ia["n_attempts"] == ib["n_attempts"] and ia["n_rhs"] == ib["n_rhs"]
    assert rel_l2(ya.cpu().numpy(), yb.cpu().numpy()) < 1e-9
