"""The film right-hand side's vector-Jacobian product on the GPU — the transposed outside
iteration alone and the whole product — against the adjoint oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of, rel_l2
from oracle.adjoint2d import FilmAdjoint

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402


def _workload(case):
    if case == "square_fp64":
        return W.square_film_128(precision=0), 1e-9
    if case == "square_fp32":
        return W.square_film_128(precision=1), 2e-4
    return film_workload(256, 64, L=(4.0, 1.0), shape="disk", radius=0.8, hole=(0.3, 0.1, 0.25),
                         n=30.0, rho_out=5.0), 1e-9


@pytest.mark.parametrize("iters", [1, 3, 6])
@pytest.mark.parametrize("case", ["square_fp64", "square_fp32", "disk_hole_nonsquare_fp64"])
def test_transposed_outside_iteration_matches_oracle(case, iters):
    wl, tol = _workload(case)
    o = oracle_of(wl)
    adj = FilmAdjoint(o, iters)
    v = W.rng(41 + iters).standard_normal((wl.ny, wl.nx))
    hb_ref, sb_ref = adj.P_T(v)
    p = native.from_workload(wl)
    hb, sb = p.mf_film_outside_vjp(torch.as_tensor(v, device="cuda"), iters)
    hb = hb.cpu().numpy()
    assert rel_l2(hb, hb_ref) < tol
    assert abs(sb - sb_ref) <= tol * abs(sb_ref)
    assert np.all(hb[wl.mask == 0] == 0.0)
    # the dot-product identity with the oracle's forward iteration, on the GPU's transpose
    r = W.rng(50 + iters)
    x = np.where(wl.mask != 0, r.standard_normal((wl.ny, wl.nx)), 0.0)
    s = 0.3
    lhs = float((adj.P(x, s) * v).sum())
    assert abs(lhs - (float((x * hb).sum()) + s * sb)) <= 10 * tol * (abs(lhs) + 1.0)


@pytest.mark.parametrize("case", ["square_fp64", "square_fp32", "disk_hole_nonsquare_fp64"])
def test_rhs_vjp_matches_oracle(case):
    """Cotangents of g, of the jc map and of h_e_dot, with a jc map and a near-critical state so
    that the linearised power law (n - 1 = 18 or 29) carries the result."""
    wl, tol = _workload(case)
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
    gb, cb, sb = p.mf_film_rhs_vjp(torch.as_tensor(g, device="cuda"), torch.as_tensor(v, device="cuda"),
                                   iters)
    gb, cb = gb.cpu().numpy(), cb.cpu().numpy()
    assert np.abs(cb_ref).max() > 1e-3 * np.abs(gb_ref).max()      # the jc term is not negligible
    assert rel_l2(gb, gb_ref) < tol
    assert rel_l2(cb, cb_ref) < tol
    assert np.all(cb[wl.mask != 1] == 0.0)
    assert abs(sb - sb_ref) <= tol * abs(sb_ref)


@pytest.mark.parametrize("case", ["square_fp64", "square_fp32", "disk_hole_nonsquare_fp64"])
def test_warm_started_rhs_vjp_matches_oracle(case):
    """One warm-started call (the integrator's: from the previous call's last iterate) with a
    cotangent on its last iterate: cotangents of g, jc, h_e_dot and the warm start."""
    wl, tol = _workload(case)
    wl.jc_map = W.jc_map_lognormal((wl.ny, wl.nx), seed=44, sigma=0.05)
    o = oracle_of(wl)
    adj = FilmAdjoint(o)
    jc = np.array(o.jc)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=45, amplitude=1.0)
    r = W.rng(51)
    out = (wl.mask == 0).astype(float)
    v = r.standard_normal((wl.ny, wl.nx))
    om = out * r.standard_normal((wl.ny, wl.nx))
    for iters in (1, 3):
        _, _, tape = adj.call(g, jc, 0.3, out * 0.2, iters)
        gb_ref, cb_ref, sb_ref, wb_ref = adj.call_vjp(tape, jc, iters, v, om)
        p = native.from_workload(wl)
        dv = lambda a: torch.as_tensor(a, device="cuda")
        gb, cb, wb, sb = p.mf_film_rhs_vjp_warm(dv(g), dv(v), iters, dv(om))
        assert rel_l2(gb.cpu().numpy(), gb_ref) < tol
        assert rel_l2(cb.cpu().numpy(), cb_ref) < tol
        assert rel_l2(wb.cpu().numpy(), wb_ref) < tol
        assert abs(sb - sb_ref) <= tol * abs(sb_ref) + tol * np.abs(wb_ref).sum()
        assert np.all(wb.cpu().numpy()[wl.mask != 0] == 0.0)


KNOTS = ((0.0, 0.5, 1.0), (0.0, 0.3, 0.45))
STEPS = [(0.1 + 0.002 * i, 0.002) for i in range(6)]
ITERS = [5, 2, 3, 1, 2, 2, 3, 1, 1, 2, 3, 2, 1, 1, 2, 2, 2, 3]


def _solve_case(precision):
    wl = W.square_film_128(precision=precision)
    wl.he_knots = KNOTS
    wl.jc_map = W.jc_map_lognormal((wl.ny, wl.nx), seed=47, sigma=0.05)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=48, amplitude=1.0)
    target = W.rng(49).standard_normal((wl.ny, wl.nx)) * 0.01
    return wl, g0, target


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_solve_gradient_matches_oracle(precision, tol):
    """Loss, dL/djc and dL/d(knot values) of a frozen-decision solve (6 steps, given counts per
    call, warm start carried from call to call, cold first call; n = 19, lognormal jc map,
    near-critical start) against FilmAdjoint.gradient.  FP32 transforms: each evaluation is
    within 2e-4 and a step sums three products and three forward evaluations, so 1e-3."""
    wl, g0, target = _solve_case(precision)
    o = oracle_of(wl)
    L_ref, cb_ref, vb_ref, _ = FilmAdjoint(o).gradient(g0, np.array(o.jc), KNOTS[0], KNOTS[1], STEPS,
                                                       target, ITERS)
    p = native.from_workload(wl)
    L, cb, vb, _ = p.mf_film_solve_gradient(torch.as_tensor(g0, device="cuda"),
                                            torch.as_tensor(target, device="cuda"), STEPS, ITERS,
                                            ckpt_every=4)
    assert abs(L - L_ref) <= tol * abs(L_ref)
    assert rel_l2(cb.cpu().numpy(), cb_ref) < tol
    np.testing.assert_allclose(vb, vb_ref, rtol=tol, atol=tol * np.abs(vb_ref).max())
    L2, cb2, vb2, _ = p.mf_film_solve_gradient(torch.as_tensor(g0, device="cuda"),
                                               torch.as_tensor(target, device="cuda"), STEPS, ITERS,
                                               ckpt_every=4, grad=False)
    assert L2 == L and cb2 is None and vb2 is None                # the forward alone


def test_solve_gradient_with_a_given_first_warm_start():
    wl, g0, target = _solve_case(0)
    o = oracle_of(wl)
    warm0 = (wl.mask == 0) * (0.25 + 0.05 * W.rng(52).standard_normal((wl.ny, wl.nx)))
    L_ref, cb_ref, vb_ref, wb_ref = FilmAdjoint(o).gradient(g0, np.array(o.jc), KNOTS[0], KNOTS[1],
                                                            STEPS, target, ITERS, warm0)
    p = native.from_workload(wl)
    dv = lambda a: torch.as_tensor(a, device="cuda")
    L, cb, vb, wb = p.mf_film_solve_gradient(dv(g0), dv(target), STEPS, ITERS, ckpt_every=2,
                                             warm0=dv(warm0), warm0_grad=True)
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert rel_l2(cb.cpu().numpy(), cb_ref) < 1e-9
    assert rel_l2(wb.cpu().numpy(), wb_ref) < 1e-9
    np.testing.assert_allclose(vb, vb_ref, rtol=1e-9, atol=1e-9 * np.abs(vb_ref).max())


def test_checkpoint_interval_does_not_change_the_gradient():
    """The reverse sweep recomputes each segment from its checkpoint exactly as the forward ran
    it: every interval gives the same bits."""
    wl, g0, target = _solve_case(1)
    p = native.from_workload(wl)
    dv = lambda a: torch.as_tensor(a, device="cuda")
    ref = p.mf_film_solve_gradient(dv(g0), dv(target), STEPS, ITERS, ckpt_every=6)
    for C in (1, 4):
        got = p.mf_film_solve_gradient(dv(g0), dv(target), STEPS, ITERS, ckpt_every=C)
        assert got[0] == ref[0] and got[2] == ref[2]
        assert torch.equal(got[1], ref[1])


def test_knot_count_mismatch_is_refused():
    wl, g0, target = _solve_case(0)
    p = native.from_workload(wl)
    with pytest.raises(ValueError):
        p.mf_set_knot_values([0.0, 0.3])
    assert p.lib.mf_set_knot_values(p.h, (native.ctypes.c_double * 2)(0.0, 0.3), 2) == native.MF_ERR_ARG


def test_autograd_wrapper_and_central_differences_of_the_gpu_map():
    """jc.grad and knots.grad through torch.autograd equal the oracle's gradient, for a jc given on
    the CPU (the gradient comes back there), and central differences of the GPU map itself
    (parameters changed in place with mf_set_jc_map and mf_set_knot_values) agree with them."""
    from paper_1801_04869_gb300.adjoint import film_solve_loss
    wl, g0, target = _solve_case(0)
    o = oracle_of(wl)
    _, cb_ref, vb_ref, _ = FilmAdjoint(o).gradient(g0, np.array(o.jc), KNOTS[0], KNOTS[1], STEPS,
                                                   target, ITERS)
    p = native.from_workload(wl)
    g0d = torch.as_tensor(g0, device="cuda")
    td = torch.as_tensor(target, device="cuda")
    jc = torch.tensor(wl.jc_map, dtype=torch.float64, requires_grad=True)          # on the CPU
    kv = torch.tensor(KNOTS[1], dtype=torch.float64, requires_grad=True)
    loss = film_solve_loss(jc, kv, p, g0d, td, STEPS, ITERS)
    loss.backward()
    assert jc.grad.device.type == "cpu"
    assert rel_l2(jc.grad.numpy(), cb_ref) < 1e-9
    np.testing.assert_allclose(kv.grad.numpy(), vb_ref, rtol=1e-9, atol=1e-12)

    def L(jcv, kvv):
        with torch.no_grad():
            return float(film_solve_loss(jcv, kvv, p, g0d, td, STEPS, ITERS))

    eps = 1e-5
    i = int(np.argmax(np.abs(cb_ref)))
    e = torch.zeros_like(jc).view(-1)
    e[i] = eps
    e = e.view_as(jc)
    fd = (L(jc.detach() + e, kv.detach()) - L(jc.detach() - e, kv.detach())) / (2 * eps)
    assert abs(fd - cb_ref.reshape(-1)[i]) <= 1e-6 * abs(fd)
    d = torch.tensor([0.0, eps, 0.0], dtype=torch.float64)
    fd = (L(jc.detach(), kv.detach() + d) - L(jc.detach(), kv.detach() - d)) / (2 * eps)
    assert abs(fd - vb_ref[1]) <= 1e-6 * abs(fd)


def test_refused_for_bulk_and_for_films_without_free_space():
    cube = native.from_workload(W.cube_bulk(16, precision=0))
    v = torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(native.MFError) as e:
        cube.mf_film_outside_vjp(v, 2)
    assert e.value.status == native.MF_ERR_ARG
    wl = film_workload(32, 32, L=(1.0, 1.0), ax=5.0, ay=5.0)         # the film fills the box
    assert (wl.mask != 0).all()
    p = native.from_workload(wl)
    with pytest.raises(native.MFError) as e:
        p.mf_film_outside_vjp(torch.zeros((32, 32), dtype=torch.float64, device="cuda"), 2)
    assert e.value.status == native.MF_ERR_ARG
