"""Parity of the CUDA bulk path (Section 3.1, Eqs. 13-18) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as W
from helpers import oracle_of, rel_l2
from oracle.bs23 import BS23, LogEntry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1801_04869_gb300 import native  # noqa: E402

TOL64 = 1e-9
TOL32 = 2e-4


def bulk_workload(nx, ny, nz, L=(1.0, 1.0, 1.0), shape="box", precision=0, **kw):
    dims = {k: kw.pop(k) for k in ("ax", "ay", "az", "r_in", "r_out") if k in kw}
    m = W.bulk_mask(nx, ny, nz, *L, shape, **dims)
    base = dict(n=25.0, rho_out=5.0, precision=precision, t0=0.0, t1=1.0,
                he_knots=((0.0, 0.5, 1.0), (0.0, 0.25, 0.25)), iter_tol=1e-4)
    base.update(kw)
    return W.Workload(f"bulk_{nx}x{ny}x{nz}", 3, nx, ny, nz, *L, m, **base)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("dims", [(8, 8, 8), (32, 16, 8), (16, 64, 32), (64, 64, 64), (128, 128, 128)])
@pytest.mark.parametrize("precision", [0, 1])
def test_current_readout_round_trip(dims, precision):
    """j = curl h: x, y, z passes with the smoothed curl, inverse passes; and the moment."""
    nx, ny, nz = dims
    wl = bulk_workload(nx, ny, nz, L=(1.0, 0.8, 1.2), precision=precision, ax=0.5, ay=0.4, az=0.6)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=nx + 3 * ny + 7 * nz)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_J, out=out, t=0.1, y=dev(h))
    err = rel_l2(out.cpu().numpy(), o.current(h))
    assert err < (1e-13 if precision == 0 else 2e-6), err
    m = p.mf_readout(native.MF_READ_MOMENT, t=0.1, y=dev(h))
    np.testing.assert_allclose(m, o.magnetization(h), rtol=1e-11 if precision == 0 else 2e-5,
                               atol=1e-13 if precision == 0 else 1e-7)


@pytest.mark.parametrize("precision", [0, 1])
def test_electric_field_readout(precision):
    """e = rho(|j|) j (Eq. 13) with j = curl h, Ohm law outside: MF_READ_E against the oracle."""
    wl = bulk_workload(32, 32, 32, precision=precision, ax=0.5, ay=0.4, az=0.3)
    wl.jc_map = W.jc_map_lognormal((32, 32, 32), seed=19)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=20, h0=0.3, depth=0.3)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((3, 32, 32, 32), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_E, out=out, t=0.1, y=dev(h))
    err = rel_l2(out.cpu().numpy(), o.electric_field(o.current(h)))
    assert err < (TOL64 if precision == 0 else TOL32), err


def _rhs_pair(wl, h, times, force=None, tol=TOL64):
    o = oracle_of(wl)
    p = native.from_workload(wl)
    y = dev(h)
    out = torch.zeros_like(y)
    for t in times:
        ref, it_o, st_o = o.rhs(t, h, None, force)
        it_g, st_g = p.mf_rhs(t, y, out, force_iters=force or 0, allow_noconv=True)
        assert (it_g, st_g) == (it_o, st_o), (t, it_g, it_o, st_g, st_o)
        err = rel_l2(out.cpu().numpy(), ref)
        assert err < tol, (t, err)


def test_rhs_fp64_cube_forced_and_converged():
    wl = bulk_workload(32, 32, 32)
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=41)
    _rhs_pair(wl, h, [0.1, 0.3], force=3)
    _rhs_pair(wl, h, [0.1, 0.1 + 1e-3, 0.7])          # warm starts, then past the knot


@pytest.mark.parametrize("case", ["ball_cut_layer", "jc_map", "ohmic_n1", "nonsquare"])
def test_rhs_fp64_variants(case):
    if case == "ball_cut_layer":
        wl = bulk_workload(32, 32, 32, L=(1.5, 1.5, 1.5), shape="ball", r_in=0.5, r_out=1.0, n=30.0)
        z = W.cell_centres(32, 1.5)[:, None, None]
        y = W.cell_centres(32, 1.5)[None, :, None]
        layer = (np.abs(z) <= 0.1) & (np.abs(y) < 0.4) & (wl.mask == 0)
        wl.mask = np.where(layer, 2, wl.mask).astype(np.uint8)
    elif case == "jc_map":
        wl = bulk_workload(32, 32, 32)
        wl.jc_map = W.jc_map_lognormal((32, 32, 32), seed=6)
    elif case == "ohmic_n1":
        wl = bulk_workload(16, 16, 16, n=1.0, rho_out=2.0)
    else:
        wl = bulk_workload(64, 32, 16, L=(2.0, 1.0, 0.5), ax=1.0, ay=0.5, az=0.25)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=42)
    _rhs_pair(wl, h, [0.05, 0.4], force=2)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("dims", [(32, 256, 256), (16, 512, 256)])
def test_rhs_with_bulk_copied_lines(dims, precision, tol):
    """y and z lines of 256 or more points arrive by bulk copies (tensor memory accelerator) into
    the staging buffer, shorter ones by per-thread asynchronous copies: a forced-iteration right-
    hand side and the current readout on grids that take the bulk copies on one or both axes,
    in both precisions (FP64: 16-byte values, twice the bytes per line)."""
    nx, ny, nz = dims
    wl = bulk_workload(nx, ny, nz, L=(0.5, 2.0, 2.0), precision=precision, ax=0.3, ay=1.0, az=1.0)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=71, h0=0.3, depth=0.3)
    _rhs_pair(wl, h, [0.2], force=2, tol=tol)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    out = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_J, out=out, t=0.2, y=dev(h))
    assert rel_l2(out.cpu().numpy(), o.current(h)) < (1e-13 if precision == 0 else 2e-6)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("dims", [(512, 64, 32), (16, 16, 512)])
def test_rhs_at_the_maximum_axis_length(dims, precision, tol):
    """512 points, the largest axis the bulk path accepts, along x (x-pass items of 4 rows of
    three fields, 257-point half spectra) and along z (z lines of 512 points by bulk copies):
    a forced-iteration right-hand side and the current readout against the oracle."""
    nx, ny, nz = dims
    L = (2.0, 0.25, 0.125) if nx == 512 else (0.125, 0.125, 2.0)
    ext = dict(ax=1.0, ay=0.1, az=0.05) if nx == 512 else dict(ax=0.08, ay=0.06, az=1.0)
    wl = bulk_workload(nx, ny, nz, L=L, precision=precision, **ext)
    h = W.bulk_state(wl.mask, (wl.Lx, wl.Ly, wl.Lz), seed=73, h0=0.3, depth=0.05, noise=0.01)
    _rhs_pair(wl, h, [0.2], force=2, tol=tol)
    o = oracle_of(wl)
    p = native.from_workload(wl)
    if nx == 512:
        assert p.mf_get_info()["rows_per_item"] == 4
    out = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    p.mf_readout(native.MF_READ_J, out=out, t=0.2, y=dev(h))
    assert rel_l2(out.cpu().numpy(), o.current(h)) < (1e-13 if precision == 0 else 2e-6)


def test_rhs_no_free_space_single_pass():
    wl = bulk_workload(16, 16, 16, ax=5.0, ay=5.0, az=5.0)
    assert (wl.mask == 1).all()
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=43)
    _rhs_pair(wl, h, [0.2])


def test_rhs_fp32_precision_form():
    wl = bulk_workload(32, 32, 32, precision=1)
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=44)
    _rhs_pair(wl, h, [0.1, 0.3], force=3, tol=TOL32)


@pytest.mark.slow
def test_rhs_full_size_cube_128_fp32():
    """The cube workload (64^3 cells in a 128^3 grid), FP32 transforms, against the FP64 oracle."""
    wl = W.cube_bulk(128, precision=1)
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=45)
    _rhs_pair(wl, h, [0.2], force=2, tol=TOL32)


@pytest.mark.slow
def test_rhs_full_size_cube_256_fp32():
    """The larger cube workload (128^3 cells in a 256^3 grid), FP32 transforms, against the FP64
    oracle (one forced outside iteration: the oracle takes about half a minute)."""
    wl = W.cube_bulk(256, precision=1)
    h = W.bulk_state(wl.mask, (1.0, 1.0, 1.0), seed=46)
    _rhs_pair(wl, h, [0.2], force=1, tol=TOL32)


def test_ramp_fp64_lock_step_small_cube():
    """Cube 16^3 cells in a 32^3 grid through the ramp knot at t = 0.5, replayed by the oracle."""
    wl = W.cube_bulk(32, precision=0)
    p = native.from_workload(wl)
    t_out = np.array([0.25, 0.5, 0.6])
    m, j = p.mf_run_ramp(t_out, want_fields=True)
    log = p.mf_get_log()
    o = oracle_of(wl)
    s = BS23(o.rhs, o.wf, rtol=wl.rtol, atol=wl.atol)
    s.start(0.0, np.zeros((3, 32, 32, 32)), 1.0)
    s.replay([LogEntry(*e[:3], e[3], e[4], e[5]) for e in log])
    assert s.t == pytest.approx(0.6, abs=1e-14)
    y = torch.zeros((3, 32, 32, 32), dtype=torch.float64, device="cuda")
    p.mf_get_state(y)
    assert rel_l2(y.cpu().numpy(), s.y) < 1e-6
    np.testing.assert_allclose(m[-1], o.magnetization(s.y), rtol=1e-6, atol=1e-12)
    assert rel_l2(j[-1].cpu().numpy().reshape(3, 32, 32, 32), o.current(s.y)) < 1e-6
    # the first attempt after the knot recomputes k1 (h_e_dot jumps there)
    after = [e for e in log if e[0] == 0.5]
    assert after and after[0][4][0] >= 0


def test_ramp_with_an_output_time_one_ulp_before_a_knot():
    """Output times from numpy.linspace put 0.49999999999999994 one ulp before the knot at 0.5:
    the sliver step to the knot is accepted and the next step starts from the step size the
    sliver replaced (it once collapsed to 5 x 5.6e-17 and stopped with step underflow)."""
    wl = bulk_workload(32, 32, 32, precision=1)
    p = native.from_workload(wl)
    t_out = np.linspace(0.05, 1.0, 20)
    m, _ = p.mf_run_ramp(t_out)
    info = p.mf_get_info()
    assert info["t"] == 1.0 and info["n_noconv"] == 0
    log = p.mf_get_log()
    slivers = [e for e in log if e[3] == 1 and e[1] < 1e-12]
    assert len(slivers) == 1 and slivers[0][2] == 0.5
