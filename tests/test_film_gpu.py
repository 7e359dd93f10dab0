"""Parity of the CUDA thin-film path (Section 2) with the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import workloads as W
from helpers import film_workload, oracle_of, rel_l2
from oracle.bs23 import BS23, LogEntry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

TOL64 = 1e-9        # FP64 path: per right-hand side, relative L2
TOL32 = 2e-4        # FP32 transforms: per right-hand side and per ramp, relative L2


def gpu_of(wl, **over):
    return native.from_workload(wl, **over)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 64), (128, 128), (256, 32), (512, 512), (2048, 2048)])
@pytest.mark.parametrize("precision", [0, 1])
def test_hz_readout_round_trip(nx, ny, precision):
    """h_z = h_e + F^-1[(|k|/2) F g]: x pass, y pass with multiplier, inverse passes."""
    wl = film_workload(nx, ny, L=(2.0, 1.5), precision=precision, ax=1.0, ay=0.7)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=nx + ny) + 0.05 * W.rng(3).standard_normal((ny, nx))
    o = oracle_of(wl)
    p = gpu_of(wl)
    out = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_HZ, out=out, t=0.3, y=dev(g))
    ref = o.hz(0.3, g)
    err = rel_l2(out.cpu().numpy(), ref)
    assert err < (1e-13 if precision == 0 else 2e-6), err
    m = p.mf_readout(native.MF_READ_MOMENT, t=0.3, y=dev(g))
    assert m[0] == pytest.approx(o.magnetization(g), rel=1e-12)


@pytest.mark.parametrize("case", ["square_n19", "disk_hole_jc_map"])
@pytest.mark.parametrize("precision", [0, 1])
def test_electric_field_readout(case, precision):
    """e = rho(|j|) j (Eq. 3) with j = (g_y, -g_x) (Eq. 2), Ohm law outside the film: the
    MF_READ_E readout against the oracle's electric field."""
    if case == "square_n19":
        wl = film_workload(128, 128, precision=precision, ax=1.0, ay=1.0)
    else:
        wl = film_workload(256, 64, L=(4.0, 1.0), shape="disk", radius=0.8, hole=(0.3, 0.1, 0.25),
                           n=30.0, rho_out=5.0, precision=precision)
        wl.jc_map = W.jc_map_lognormal((64, 256), seed=9)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=31, amplitude=0.8)
    o = oracle_of(wl)
    p = gpu_of(wl)
    out = torch.zeros((2, wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_E, out=out, t=0.3, y=dev(g))
    ex, ey = o.electric_field(*o.sheet_current(g))
    err = rel_l2(out.cpu().numpy(), np.stack([ex, ey]))
    assert err < (TOL64 if precision == 0 else TOL32), err


def _rhs_pair(wl, g, times, force=None, precision_tol=TOL64):
    o = oracle_of(wl)
    p = gpu_of(wl)
    y = dev(g)
    out = torch.zeros_like(y)
    for t in times:
        ref, it_o, st_o = o.rhs(t, g, None, force)
        it_g, st_g = p.mf_rhs(t, y, out, force_iters=force or 0, allow_noconv=True)
        assert it_g == it_o and st_g == st_o, (t, it_g, it_o, st_g, st_o)
        err = rel_l2(out.cpu().numpy(), ref)
        assert err < precision_tol, (t, err)
    return p, o


def test_rhs_fp64_forced_iterations_config1_geometry():
    wl = W.square_film_128(precision=0)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=11, amplitude=0.5)
    _rhs_pair(wl, g, [0.1, 0.2, 0.35], force=6)


def test_rhs_fp64_converged_iterations_with_warm_start():
    wl = W.square_film_128(precision=0)
    wl.iter_tol = 2e-3
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=12, amplitude=0.4)
    _rhs_pair(wl, g, [0.2, 0.2 + 1e-3, 0.2 + 2e-3])


@pytest.mark.parametrize("case", ["disk_hole_nonsquare", "jc_map", "ohmic_n1"])
def test_rhs_fp64_variants(case):
    if case == "disk_hole_nonsquare":
        wl = film_workload(256, 64, L=(4.0, 1.0), shape="disk", radius=0.8, hole=(0.3, 0.1, 0.25),
                           n=30.0, rho_out=5.0)
    elif case == "jc_map":
        wl = film_workload(128, 128, ax=1.0, ay=0.6)
        wl.jc_map = W.jc_map_lognormal((128, 128), seed=5)
    else:
        wl = film_workload(64, 64, shape="disk", radius=1.0, n=1.0, rho_out=3.0)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=21, amplitude=0.5)
    _rhs_pair(wl, g, [0.05, 0.3], force=5)


def test_rhs_unbounded_ohmic_sheet_closed_form():
    """No free space: f is linear; a cosine mode decays at 2 rho |k| G^2 (thin-sheet eddy currents)."""
    nx = ny = 32
    wl = film_workload(nx, ny, L=(1.0, 1.0), ax=5.0, ay=5.0, n=1.0, rho_out=1.0)
    assert (wl.mask == 1).all()
    wl.sigma = 0.05
    x = W.cell_centres(nx, 1.0)[None, :] + 0 * W.cell_centres(ny, 1.0)[:, None]
    k = 2 * math.pi
    g = np.cos(k * x)
    p = gpu_of(wl)
    out = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    p.mf_rhs(0.2, dev(g), out)
    G = math.exp(-k * k * 0.05 ** 2 / 2)
    np.testing.assert_allclose(out.cpu().numpy(), -2 * k * G * G * g, atol=1e-11)


def test_rhs_noconv_status_and_output():
    wl = W.square_film_128(precision=0)
    wl.iter_tol = 1e-14
    wl.iter_max = 3
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=13, amplitude=0.5)
    o = oracle_of(wl)
    p = gpu_of(wl)
    out = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    it, st = p.mf_rhs(0.4, dev(g), out, allow_noconv=True)
    ref, it_o, st_o = o.rhs(0.4, g)
    assert st == native.MF_ERR_NOCONV == st_o and it == 3 == it_o
    assert rel_l2(out.cpu().numpy(), ref) < TOL64


def test_rhs_fp32_precision_form():
    wl = W.square_film_128(precision=1)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=14, amplitude=0.5)
    _rhs_pair(wl, g, [0.1, 0.3], force=6, precision_tol=TOL32)


@pytest.mark.slow
def test_rhs_full_size_rect_film_2048_fp32():
    """The 2048^2 workload (1024x512 film), FP32 transforms, against the FP64 oracle."""
    wl = W.rect_film_2048(precision=1)
    g = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=15, amplitude=0.4)
    _rhs_pair(wl, g, [0.05], force=3, precision_tol=TOL32)


@pytest.mark.slow
def test_step_full_size_rect_film_2048_fp32_as_benchmarked():
    """The benchmark's launch: the 2048^2 film from the bench's start state, one persistent
    mf_advance launch of one BS23 attempt (4 right-hand sides with converged outside
    iterations).  The FP64 oracle replays it with the GPU's step size and per-stage iteration
    counts; the state increment and the h_z increment agree within the precision form's 2e-4."""
    wl = W.rect_film_2048(precision=1)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=100, amplitude=0.3)
    p = gpu_of(wl)
    p.mf_set_state(0.05, dev(g0), h=2e-5)
    p.mf_advance(1.0, max_attempts=1)
    log = p.mf_get_log()
    assert len(log) == 1 and log[0][3] == 1 and min(log[0][4]) >= 1
    g = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    t1, _ = p.mf_get_state(g)
    # the oracle runs the logged iteration counts; a stop-test tolerance it always meets keeps
    # its status (and so its warm start) that of the converged GPU stages
    o = oracle_of(wl, iter_tol=1.0)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    s.start(0.05, g0, 1.0)
    s.replay([LogEntry(*e) for e in log])
    assert s.t == t1
    dg_gpu = g.cpu().numpy() - g0
    dg_ref = s.y - g0
    assert rel_l2(dg_gpu, dg_ref) < TOL32
    dhz = o.hz(t1, s.y) - o.hz(0.05, g0)
    dhz_gpu = o.hz(t1, g.cpu().numpy()) - o.hz(0.05, g0)
    assert rel_l2(dhz_gpu, dhz) < TOL32


def _replay(o, wl, log, y0):
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    s.start(wl.t0, y0, wl.t1)
    entries = [LogEntry(t, h, tn, oc, it, err) for (t, h, tn, oc, it, err) in log]
    s.replay(entries)
    return s


def test_ramp_fp64_lock_step_config1():
    """Square film 64^2 in 128^2, n = 19, h_e 0 -> 0.5: the GPU ramp replayed by the oracle with the
    GPU's step sizes, decisions and iteration counts."""
    wl = W.square_film_128(precision=0)
    p = gpu_of(wl)
    t_out = np.linspace(0.1, 1.0, 10)
    m, hz = p.mf_run_ramp(t_out, want_fields=True)
    log = p.mf_get_log()
    info = p.mf_get_info()
    assert info["n_accepted"] > 10 and info["n_noconv"] == 0
    assert abs(info["t"] - 1.0) < 1e-15
    o = oracle_of(wl)
    s = _replay(o, wl, log, np.zeros((128, 128)))
    assert s.t == pytest.approx(1.0, abs=1e-14)
    g = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    p.mf_get_state(g)
    assert rel_l2(g.cpu().numpy(), s.y) < 1e-6
    assert rel_l2(hz[-1].cpu().numpy().reshape(128, 128), o.hz(1.0, s.y)) < 1e-6
    assert m[-1, 0] == pytest.approx(o.magnetization(s.y), rel=1e-6)
    # accept/reject decisions the oracle would take on the replayed steps
    acc = [e for e in s.log if e.outcome == 1]
    assert all(e.err <= 1.0 + 1e-6 for e in acc)


def test_ramp_fp32_free_running_config1():
    """FP32 transforms with FP64 state: h_z and m_z(t) within 2e-4 of the free-running oracle."""
    wl = W.square_film_128(precision=1)
    p = gpu_of(wl)
    t_out = np.array([0.25, 0.5, 0.75, 1.0])
    m, hz = p.mf_run_ramp(t_out, want_fields=True)
    o = oracle_of(wl)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol, on_accept=o.accept, on_attempt=o.begin_attempt)
    s.start(0.0, np.zeros((128, 128)), 1.0)
    for k, t in enumerate(t_out):
        s.advance(t)
        assert abs(m[k, 0] - o.magnetization(s.y)) <= TOL32 * abs(o.magnetization(s.y))
        assert rel_l2(hz[k].cpu().numpy().reshape(128, 128), o.hz(t, s.y)) < TOL32


def test_step_and_state_round_trip():
    wl = W.square_film_128(precision=0)
    p = gpu_of(wl)
    g0 = W.film_state(wl.mask, wl.Lx, wl.Ly, seed=16, amplitude=0.2)
    p.mf_set_state(0.2, dev(g0), h=1e-3)
    t, h = p.mf_get_state()
    assert t == 0.2 and h == 1e-3
    assert p.mf_step(1.0) in (True, False)
    t1, _ = p.mf_get_state()
    assert t1 >= 0.2
    info = p.mf_get_info()
    assert info["n_attempts"] == 1


def test_binding_refuses_tensors_the_library_cannot_take():
    """The C calls take bare pointers; the binding refuses, before any call, a tensor that is too
    short, not float64, not contiguous or not on the problem's device."""
    wl = film_workload(32, 32)
    p = gpu_of(wl)
    y = torch.zeros((32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        p.mf_rhs(0.1, y[:16], torch.zeros_like(y))
    with pytest.raises(TypeError):
        p.mf_rhs(0.1, y.float(), torch.zeros_like(y))
    with pytest.raises(ValueError):
        p.mf_rhs(0.1, y.t(), torch.zeros_like(y))                        # a transposed view
    with pytest.raises(ValueError):
        p.mf_set_state(0.0, y.cpu())
    with pytest.raises(ValueError):
        p.mf_readout(native.MF_READ_E, out=torch.zeros_like(y))          # e has 2 fields
    with pytest.raises(ValueError):
        p.mf_checkpoint_restore(torch.zeros(16, dtype=torch.uint8, device="cuda"))
    assert p.mf_get_info()["n_rhs"] == 0
